"""Source signals of the oracle (Sec. 5.1): the sampled form is the cubic Lagrange interpolant of
its samples (exact on cubics, equal to the samples on the nodes, fourth-order accurate, zero away
from the record), and a forward run driven by the samples of a Ricker pulse matches the run driven
by the pulse itself."""

import numpy as np

from oracle.rtm import forward, make_problem, rtm_shot
from oracle.wavelet import ricker, sampled
from synth import tiny_layered_rtm


def test_sampled_signal_on_the_nodes_and_outside():
    s = np.random.default_rng(2).standard_normal(12)
    dt = 0.37
    for n in range(12):
        assert abs(sampled(n * dt, s, dt, 2.0) - 2.0 * s[n]) < 1e-13
    for t in (-2.01 * dt, -10.0, 13.5 * dt, 100.0):
        assert sampled(t, s, dt) == 0.0


def test_sampled_signal_is_exact_on_cubics():
    dt = 0.25
    c = (0.3, -1.2, 0.7, 0.45)
    p = lambda t: c[0] + c[1] * t + c[2] * t ** 2 + c[3] * t ** 3  # noqa: E731
    s = np.array([p(n * dt) for n in range(20)])
    for t in np.linspace(dt, 17 * dt, 101):
        assert abs(sampled(t, s, dt) - p(t)) < 1e-11 * max(1.0, abs(p(t)))


def test_sampled_ricker_converges_at_fourth_order():
    f0, tp = 25.0, 0.05
    t = np.linspace(0.01, 0.09, 333)
    err = []
    for dt in (2e-3, 1e-3):
        s = ricker(np.arange(200) * dt, f0, tp)
        err.append(max(abs(sampled(x, s, dt) - ricker(x, f0, tp)) for x in t))
    assert 12.0 < err[0] / err[1] < 20.0


def test_forward_traces_equal_the_shot_traces_and_the_sampled_pulse():
    w = tiny_layered_rtm(N=2, t_final=0.003)
    prob = make_problem(w.xyz, w.tets, w.c, w.rho, 2, default_bc=w.default_bc, cfl=w.cfl,
                        n_levels_max=w.n_levels_max)
    tr = forward(prob, w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final)
    shot = rtm_shot(prob, w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final)
    assert np.array_equal(tr, shot.traces) and np.abs(tr).max() > 0
    # the same pulse given by samples at a spacing unrelated to the time step
    dt_s = 0.3 * prob.dt_local
    s = ricker(np.arange(int((w.t_final + 2 * prob.dt_global) / dt_s)) * dt_s, w.f0, w.t_peak)
    tr_s = forward(prob, w.source_xyz, 0.0, 0.0, 1.0, w.receivers, w.t_final, wavelet=s, wavelet_dt=dt_s)
    assert np.linalg.norm(tr_s - tr) < 1e-4 * np.linalg.norm(tr)
