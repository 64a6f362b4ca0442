"""The library's transparent and rigid boundaries on a plane pulse (see tests/plane_wave.py): the
pulse leaves through a transparent end and is reflected by a rigid one, in FP64 and FP32, and the
FP64 fields match the oracle's run step for step."""

import numpy as np
import pytest

from oracle.mrab import MRAB
from oracle.rtm import full_rhs, make_problem
from paper_1506_00907_gb300 import ridg
from tests import plane_wave as pw
from tests.parity_cases import TOL

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("end_code, lo, hi", [(2, 0.0, 1e-4), (3, 0.99, 1.0)])
def test_plane_pulse_at_transparent_and_rigid_ends(dtype, end_code, lo, hi):
    xyz, tets, fb = pw.bar(end_code)
    K = len(tets)
    mesh = ridg.Mesh(xyz, tets, face_bc=fb)
    s = ridg.Solver(mesh, 3, np.full(K, pw.C), np.full(K, pw.RHO), dtype=dtype, n_levels_max=1)
    x = s.nodes()
    dt = s.info.dt_local
    s.set_state(pw.state(x, 0.0))
    s.set_history(s.eval_rhs(pw.state(x, -dt)), s.eval_rhs(pw.state(x, -2 * dt)))
    e0 = s.energy()
    n = int(np.ceil(pw.T_END / dt))
    s.step(n)
    ratio = s.energy() / e0
    assert lo <= ratio <= hi, ratio
    if dtype == "f64":
        prob = make_problem(xyz, tets, np.full(K, pw.C), np.full(K, pw.RHO), 3, face_bc=fb, n_levels_max=1)
        S = MRAB(prob.geo, prob.levels, prob.n_levels, prob.dt_local)
        S.set_state(pw.state(prob.geo.x, 0.0))
        S.set_history(full_rhs(prob, pw.state(prob.geo.x, -dt)), full_rhs(prob, pw.state(prob.geo.x, -2 * dt)))
        for _ in range(n):
            S.global_step()
        # relative to the initial fields: after the transparent exit the remaining fields are tiny
        err = np.linalg.norm(s.get_state() - S.q) / np.linalg.norm(pw.state(x, 0.0))
        assert err < 10 * TOL["f64"], err
