"""RTM procedure of the oracle (Sec. 2, Sec. 3.3, Sec. 4.3): boundary-trace replay
reconstructs the source wavefield, and a whole shot runs with finite images."""

import numpy as np

from oracle.dg_rhs import energy
from oracle.mrab import MRAB
from oracle.rtm import make_problem, rtm_shot
from synth import tiny_layered_rtm


def _pulse_problem():
    w = tiny_layered_rtm(N=3)
    prob = make_problem(w.xyz, w.tets, w.c, w.rho, 3, default_bc=2, cfl=0.15)
    g = prob.geo
    q0 = np.zeros((g.K, 4, g.ref.Np))
    q0[:, 0] = np.exp(-((g.x - np.array([100.0, 100.0, 50.0])) ** 2).sum(-1) / (2 * 20.0 ** 2))
    return prob, q0


def _forward_then_backward(prob, q0, n_global, replay):
    g = prob.geo
    S = MRAB(g, prob.levels, prob.n_levels, prob.dt_local, +1)
    S.set_state(q0)
    S.record = {}
    states = [S.q.copy()]
    for _ in range(n_global):
        S.global_step()
        states.append(S.q.copy())
    tau_f, nl = S.tau, S.n_local
    saved = {}
    for _ in range(2 * nl):
        tau = S.tau
        S.fine_step()
        for l, st in S.stride.items():
            if tau == tau_f + 2 * st:
                E = S.level_elems[l]
                saved[l] = (S.hist[1][E].copy(), S.hist[0][E].copy())
    S.phase_rhs()
    E = S.level_elems[1]
    saved[1] = (S.hist[1][E].copy(), S.hist[0][E].copy())
    B = MRAB(g, prob.levels, prob.n_levels, prob.dt_local, -1, tau0=tau_f)
    B.set_state(states[-1])
    for l, (r1, r2) in saved.items():
        E = B.level_elems[l]
        B.hist[0][E], B.hist[1][E] = r1, r2
    if replay:
        B.replay = S.record
    for _ in range(n_global):
        B.global_step()
    return np.linalg.norm(B.q - states[0]) / np.linalg.norm(states[0])


def test_replayed_boundary_traces_reconstruct_the_source_wavefield():
    """Recorded forward traces as the exterior state of boundary faces: after 200 global steps
    (28 ms: the pulse has reached the transparent faces 50 m away), the backward run returns
    to the initial state within a few percent; without the replay the waves that left do not come
    back and the error is an order of magnitude larger."""
    prob, q0 = _pulse_problem()
    e_replay = _forward_then_backward(prob, q0, 200, True)
    e_plain = _forward_then_backward(prob, q0, 200, False)
    assert e_replay < 4e-2
    assert e_plain > 5 * e_replay


def test_tiny_shot_runs():
    w = tiny_layered_rtm(N=2, t_final=0.01)
    prob = make_problem(w.xyz, w.tets, w.c, w.rho, 2, default_bc=2, cfl=0.15)
    res = rtm_shot(prob, w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final)
    assert res.traces.shape == (len(w.receivers), res.n_global + 1)
    assert np.all(np.isfinite(res.image_p)) and np.all(np.isfinite(res.image_q))
    assert np.abs(res.image_p).max() > 0 and np.abs(res.traces).max() > 0
    assert res.dof_updates > 0
