"""Pin of the oracle's source term and wave propagation against the free-space Green's function
(reading of Eq. waveSyst1 vs Eq. sourceTerm: the source enters dp/dt with unit weight, M_k w =
l(x0)): the pressure at a receiver 0.49 away from a Ricker point source in a homogeneous medium
follows f'(t - r/c) / (4 pi c^2 r) to discretisation accuracy; the other scaling would be
rho c^2 = 4.5 times too large."""

import numpy as np

from oracle.mrab import MRAB
from oracle.rtm import make_problem
from oracle.wavelet import ricker
from tests import green


def test_point_source_matches_greens_function():
    xyz, tets = green.cube(8)
    K = len(tets)
    prob = make_problem(xyz, tets, np.full(K, green.C), np.full(K, green.RHO), 3, default_bc=2, cfl=0.15,
                        n_levels_max=1)
    geo = prob.geo
    ks, rs = geo.locate(green.SOURCE)
    kr, rr = geo.locate(green.RECEIVER)
    w = geo.source_weights(ks, rs)
    row = geo.interpolation_row(rr)
    S = MRAB(geo, prob.levels, prob.n_levels, prob.dt_local, direction=+1, tau0=0)
    S.injections = [(ks, w, lambda tau: float(ricker(tau * prob.dt_local, green.F0, green.T_PEAK, 1.0)))]
    n_g = int(np.ceil(green.t_end() / prob.dt_global))
    ps = [row @ S.q[kr, 0]]
    for _ in range(n_g):
        S.global_step()
        ps.append(row @ S.q[kr, 0])
    ps = np.array(ps)
    pa = green.pressure(prob.dt_global * np.arange(n_g + 1))
    err = np.linalg.norm(ps - pa) / np.linalg.norm(pa)
    assert err < 0.1, err  # 8 hexes per side, N = 3: about 6.6 %
    assert 0.95 < np.abs(ps).max() / np.abs(pa).max() < 1.08
