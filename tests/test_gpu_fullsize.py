"""GPU checks at the full size of the benchmark workload (layered 2 x 2 x 1 km model, 190,608
tetrahedra, N = 4, FP32, three multi-rate levels), in the launch configuration the benchmark
times: fused step launches over every active level, one wavefield forward and two (source and
receiver, with the images) backward.

* One global multi-rate step (all three levels, half-step traces, every boundary condition in
  the model) against the FP64 oracle, element by element, at the FP32 tolerance.
* Whole-shot properties that hold at any size (the oracle cannot run a full shot of this model):
  the method is linear in the source amplitude and in the observed data, so traces scale with
  the amplitude and the images with the product of the two scalings.
"""

import numpy as np
import pytest

from oracle.mrab import MRAB
from oracle.rtm import make_problem
from paper_1506_00907_gb300 import ridg
from synth import config2_layered_rtm, random_state
from tests.parity_cases import TOL, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def workload():
    return config2_layered_rtm()


@pytest.fixture(scope="module")
def solver(workload):
    w = workload
    mesh = ridg.Mesh(w.xyz, w.tets, default_bc=w.default_bc)
    return ridg.Solver(mesh, w.N, w.c, w.rho, dtype="f32", cfl=w.cfl, n_levels_max=w.n_levels_max)


def test_full_size_global_step_parity(workload, solver):
    w, s = workload, solver
    assert s.info.K == 190_608 and s.info.n_levels == 3
    prob = make_problem(w.xyz, w.tets, w.c, w.rho, w.N, default_bc=w.default_bc, cfl=w.cfl,
                        n_levels_max=w.n_levels_max)
    assert np.array_equal(s.levels(), prob.levels)
    Np = s.Np
    q = random_state(w.K, Np, seed=21)
    r1 = random_state(w.K, Np, seed=22, scale=1e3)
    r2 = random_state(w.K, Np, seed=23, scale=1e3)
    s.set_state(q)
    s.set_history(r1, r2)
    s.step(1)
    q_gpu = s.get_state()
    st = MRAB(prob.geo, prob.levels, prob.n_levels, prob.dt_local)
    st.set_state(q)
    st.set_history(r1, r2)
    st.global_step()
    assert rel_l2(q_gpu, st.q) < TOL["f32"]
    # element by element: no element (first, last, padded block tails, level boundaries) is off, against
    # its own norm (loose) and with the largest element error against the largest element norm
    err_k = np.linalg.norm((q_gpu - st.q).reshape(w.K, -1), axis=1)
    ref_k = np.linalg.norm(st.q.reshape(w.K, -1), axis=1)
    assert (err_k / ref_k).max() < 100 * TOL["f32"]
    assert err_k.max() / ref_k.max() < 10 * TOL["f32"]


def test_full_size_shot_is_linear(workload, solver):
    w, s = workload, solver
    t_final = 0.0012  # 12 global steps: every level, the overshoot, record and replay, images
    tr1, ip1, iq1 = s.rtm_shot(w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, t_final)
    assert np.isfinite(tr1).all() and np.isfinite(ip1).all() and np.isfinite(iq1).all()
    assert np.abs(tr1).max() > 0 and np.abs(ip1).max() > 0
    # source amplitude x2: traces x2; the receiver data are the shot's own traces, so images x4
    tr2, ip2, iq2 = s.rtm_shot(w.source_xyz, w.f0, w.t_peak, 2.0, w.receivers, t_final)
    assert rel_l2(tr2, 2.0 * tr1) < 1e-6
    assert rel_l2(ip2, 4.0 * ip1) < 1e-6
    assert rel_l2(iq2, 4.0 * iq1) < 1e-6
    # observed data x3 with the source unchanged: images x3
    tr3, ip3, iq3 = s.rtm_shot(w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, t_final, observed=3.0 * tr1)
    assert rel_l2(tr3, tr1) < 1e-6
    assert rel_l2(ip3, 3.0 * ip1) < 1e-6
    assert rel_l2(iq3, 3.0 * iq1) < 1e-6
