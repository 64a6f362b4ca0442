"""Misfit gradient of the oracle (discrete adjoint of single-rate AB3, velocity in rho c^2 with
tau, level and time step frozen): the assembled operator reproduces the right-hand side, and the
adjoint gradient matches central finite differences of the oracle's own forward misfit."""

import numpy as np

from oracle.adjoint import assemble_operator, frozen_geometry, misfit_gradient, shot_misfit
from oracle.dg_rhs import rhs, traces
from oracle.rtm import make_problem
from synth import adjoint_box_small


def _case():
    w = adjoint_box_small()
    prob = make_problem(w.xyz, w.tets, w.c, w.rho, w.N, default_bc=w.default_bc, cfl=w.cfl, n_levels_max=1)
    obs = shot_misfit(prob, w.c_observed, w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final, 0.0).traces
    return w, prob, obs


def test_assembled_operator_is_the_rhs():
    w, prob, _ = _case()
    c = w.c * (1.0 + 0.1 * np.random.default_rng(4).standard_normal(w.K))
    g = frozen_geometry(prob.geo, c)
    A = assemble_operator(g)
    x = np.random.default_rng(3).standard_normal((w.K, 4, prob.geo.ref.Np))
    y = rhs(np.arange(w.K), x, traces(x, g), g)
    assert np.linalg.norm(A @ x.reshape(-1) - y.reshape(-1)) < 1e-12 * np.linalg.norm(y)


def test_adjoint_gradient_matches_finite_differences():
    w, prob, obs = _case()
    J, grad = misfit_gradient(prob, w.c, w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final, obs)
    assert J > 0 and np.all(np.isfinite(grad))
    for k in np.random.default_rng(2).choice(w.K, 4, replace=False):
        d = 1e-4 * w.c[k]
        cp, cm = w.c.copy(), w.c.copy()
        cp[k] += d
        cm[k] -= d
        Jp = shot_misfit(prob, cp, w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final, obs).misfit
        Jm = shot_misfit(prob, cm, w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final, obs).misfit
        fd = (Jp - Jm) / (2 * d)
        assert abs(fd - grad[k]) < 1e-5 * abs(grad[k]) + 1e-9 * np.abs(grad).max(), (k, fd, grad[k])
