"""Pin of the transparent boundary condition (reading of the boundary "exterior values": p+ = 0,
v+ = 0 with the upwind penalties realises p - rho c n.v = 0): a plane pulse leaves the bar through a
transparent end without reflection, while a rigid end sends it back."""

import numpy as np
import pytest

from oracle.dg_rhs import energy
from oracle.mrab import MRAB
from oracle.rtm import full_rhs, make_problem
from tests import plane_wave as pw


@pytest.mark.parametrize("end_code, lo, hi", [(2, 0.0, 1e-4), (3, 0.99, 1.0)])
def test_plane_pulse_at_transparent_and_rigid_ends(end_code, lo, hi):
    xyz, tets, fb = pw.bar(end_code)
    K = len(tets)
    prob = make_problem(xyz, tets, np.full(K, pw.C), np.full(K, pw.RHO), 3, face_bc=fb, n_levels_max=1)
    dt = prob.dt_local
    x = prob.geo.x
    S = MRAB(prob.geo, prob.levels, prob.n_levels, dt)
    S.set_state(pw.state(x, 0.0))
    S.set_history(full_rhs(prob, pw.state(x, -dt)), full_rhs(prob, pw.state(x, -2 * dt)))
    e0 = energy(S.q, prob.geo)
    for _ in range(int(np.ceil(pw.T_END / dt))):
        S.global_step()
    ratio = energy(S.q, prob.geo) / e0
    assert lo <= ratio <= hi, ratio  # transparent: about 6e-7 left; rigid: about 0.9993
