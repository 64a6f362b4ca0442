"""Misfit gradient of the oracle (discrete adjoint of single-rate AB3, velocity in rho c^2 with
tau, level and time step frozen): the assembled operator reproduces the right-hand side, and the
adjoint gradient matches central finite differences of the oracle's own forward misfit.  The
multi-rate gradient (reverse accumulation over the fine steps of Algorithm 1) matches the
single-rate adjoint on one level and central finite differences on two and three."""

import numpy as np

import pytest

from oracle.adjoint import assemble_operator, frozen_geometry, misfit_gradient, misfit_gradient_levels, shot_misfit
from oracle.dg_rhs import rhs, traces
from oracle.rtm import make_problem
from synth import adjoint_box_small, adjoint_box_three_level, adjoint_box_two_level


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


def _two_level_case(n_levels_max):
    w = adjoint_box_two_level()
    prob = make_problem(w.xyz, w.tets, w.c, w.rho, w.N, default_bc=w.default_bc, cfl=w.cfl,
                        n_levels_max=n_levels_max)
    args = (w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final)
    obs = shot_misfit(prob, w.c_observed, *args, 0.0).traces
    return w, prob, args, obs


def test_multirate_gradient_reduces_to_the_single_rate_adjoint():
    """One level: the fine-step reverse accumulation over the full state and the recursion on q
    with the transposed operator are two derivations of one gradient."""
    w, prob, args, obs = _two_level_case(1)
    assert prob.n_levels == 1
    J1, g1 = misfit_gradient(prob, w.c, *args, obs)
    J, g = misfit_gradient_levels(prob, w.c, *args, obs)
    assert abs(J - J1) <= 1e-14 * J1
    assert np.linalg.norm(g - g1) < 1e-12 * np.linalg.norm(g1)


def test_multirate_gradient_matches_finite_differences():
    """Two levels (12 + 12 elements): central differences of the forward misfit, elements of both
    levels; a state without the stored half-step traces misses by 1e-3 to 2e-2 here."""
    w, prob, args, obs = _two_level_case(2)
    assert prob.n_levels == 2 and set(np.unique(prob.levels)) == {1, 2}
    J, grad = misfit_gradient_levels(prob, w.c, *args, obs)
    assert J > 0 and np.all(np.isfinite(grad))
    ks = [0, 5, 13, 20]
    assert {int(prob.levels[k]) for k in ks} == {1, 2}
    for k in ks:
        d = 1e-4 * w.c[k]
        cp, cm = w.c.copy(), w.c.copy()
        cp[k] += d
        cm[k] -= d
        fd = (shot_misfit(prob, cp, *args, obs).misfit - shot_misfit(prob, cm, *args, obs).misfit) / (2 * d)
        assert abs(fd - grad[k]) < 1e-5 * abs(grad[k]) + 1e-9 * np.abs(grad).max(), (k, fd, grad[k])


def test_single_rate_adjoint_refuses_several_levels():
    w, prob, args, obs = _two_level_case(2)
    with pytest.raises(ValueError):
        misfit_gradient(prob, w.c, *args, obs)


def test_multirate_gradient_matches_finite_differences_on_three_levels():
    """Three levels (10 + 8 + 6 elements): nested half steps and the coupling of the two finer
    levels; central differences on elements of every level."""
    w = adjoint_box_three_level()
    prob = make_problem(w.xyz, w.tets, w.c, w.rho, w.N, default_bc=w.default_bc, cfl=w.cfl, n_levels_max=3)
    assert prob.n_levels == 3
    args = (w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final)
    obs = shot_misfit(prob, w.c_observed, *args, 0.0).traces
    J, grad = misfit_gradient_levels(prob, w.c, *args, obs)
    assert J > 0 and np.all(np.isfinite(grad))
    ks = [int(np.nonzero(prob.levels == l)[0][0]) for l in (1, 2, 3)] + [5, 15]
    for k in ks:
        d = 1e-4 * w.c[k]
        cp, cm = w.c.copy(), w.c.copy()
        cp[k] += d
        cm[k] -= d
        fd = (shot_misfit(prob, cp, *args, obs).misfit - shot_misfit(prob, cm, *args, obs).misfit) / (2 * d)
        assert abs(fd - grad[k]) < 1e-5 * abs(grad[k]) + 1e-9 * np.abs(grad).max(), (k, fd, grad[k])
