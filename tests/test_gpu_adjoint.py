"""Velocity gradient through the library's adjoint kernels (``ridg_set_velocity``,
``ridg_eval_adjoint_rhs``, ``ridg_misfit_forward`` / ``_backward``), against the oracle:

* the transposed operator equals the transpose of the oracle's assembled right-hand-side operator,
  element by element, with every boundary condition;
* <A^T x, y> = <x, A y> with the library's own A (pinned to the oracle elsewhere) at N = 1..6, on
  a multi-block mesh with a ragged tail, in both precisions;
* the misfit and its gradient equal the oracle's on a small box;
* on the 648-element adjoint box (N = 3, one level, 16 checkpoints) the gradient matches central
  finite differences of the misfit on 20 random elements, does not depend on the number of
  checkpoints, and reaches torch through ``ridg.misfit`` (a torch.autograd.Function);
* on two rate levels the misfit and the gradient equal the oracle's multi-rate gradient (reverse
  accumulation over the fine steps of Algorithm 1), independently of the number of checkpoints."""

import functools

import numpy as np
import pytest

from oracle.adjoint import assemble_operator, frozen_geometry, misfit_gradient, misfit_gradient_levels, shot_misfit
from oracle.rtm import make_problem
from paper_1506_00907_gb300 import ridg
from synth import (adjoint_box, adjoint_box_small, adjoint_box_three_level, adjoint_box_two_level,
                   adjoint_observed_velocity, random_state, tiny_layered_rtm)
from tests.parity_cases import TOL, mixed_bc, rel_l2

pytestmark = pytest.mark.gpu


def _solver(w, dtype="f64", face_bc=None, N=None, n_levels_max=1):
    mesh = ridg.Mesh(w.xyz, w.tets, face_bc=face_bc, default_bc=w.default_bc)
    return ridg.Solver(mesh, w.N if N is None else N, w.c, w.rho, dtype=dtype, cfl=w.cfl, n_levels_max=n_levels_max)


@pytest.mark.parametrize("dtype,N", [("f64", 2), ("f64", 3), ("f32", 2), ("f32", 3), ("f32", 4)])
def test_adjoint_rhs_is_the_transpose_of_the_oracle_operator(dtype, N):
    """A^T against the transpose of the oracle's assembled operator, in both precisions."""
    w = adjoint_box_small()
    fb = mixed_bc(w)
    c = w.c_observed  # a velocity other than the reference one: tau stays that of w.c
    prob = make_problem(w.xyz, w.tets, w.c, w.rho, N, face_bc=fb, default_bc=w.default_bc, cfl=w.cfl, n_levels_max=1)
    AT = assemble_operator(frozen_geometry(prob.geo, c)).T.tocsr()
    s = _solver(w, dtype=dtype, face_bc=fb, N=N)
    s.set_velocity(c)
    lam = random_state(w.K, s.Np, seed=41)
    if dtype == "f32":
        lam = lam.astype(np.float32).astype(np.float64)  # the FP32 solver's own input
    ref = (AT @ lam.reshape(-1)).reshape(lam.shape)
    out = s.eval_adjoint_rhs(lam)
    assert rel_l2(out, ref) < TOL[dtype]
    per = np.linalg.norm((out - ref).reshape(w.K, -1), axis=1) / np.linalg.norm(ref.reshape(w.K, -1), axis=1)
    assert per.max() < 100 * TOL[dtype]


@pytest.mark.parametrize("N", [3, 4])
def test_adjoint_rhs_fp32_on_the_box(N):
    """FP32 A^T on the 648-element box (21 blocks of element slots, a ragged last one) against the
    FP64 library operator, element by element."""
    w = adjoint_box()
    mesh = ridg.Mesh(w.xyz, w.tets, default_bc=w.default_bc)
    lam = random_state(w.K, (N + 1) * (N + 2) * (N + 3) // 6, seed=43).astype(np.float32).astype(np.float64)
    outs = {}
    for dtype in ("f32", "f64"):
        sv = ridg.Solver(mesh, N, w.c, w.rho, dtype=dtype, cfl=w.cfl, n_levels_max=1)
        outs[dtype] = sv.eval_adjoint_rhs(lam)
    assert rel_l2(outs["f32"], outs["f64"]) < TOL["f32"]
    per = np.linalg.norm((outs["f32"] - outs["f64"]).reshape(w.K, -1), axis=1) / np.linalg.norm(
        outs["f64"].reshape(w.K, -1), axis=1)
    assert per.max() < 100 * TOL["f32"]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
def test_adjoint_dot_product(dtype, N):
    w = tiny_layered_rtm(N=N)
    s = _solver(w, dtype=dtype, face_bc=mixed_bc(w), n_levels_max=3)
    x = random_state(w.K, s.Np, seed=5)
    y = random_state(w.K, s.Np, seed=6)
    aty = s.eval_adjoint_rhs(x)
    ay = s.eval_rhs(y)
    lhs, rhs_ = float(np.sum(aty * y)), float(np.sum(x * ay))
    scale = np.linalg.norm(aty) * np.linalg.norm(y)
    assert abs(lhs - rhs_) < (1e-12 if dtype == "f64" else 1e-5) * scale


def test_misfit_and_gradient_match_the_oracle():
    w = adjoint_box_small()
    prob = make_problem(w.xyz, w.tets, w.c, w.rho, w.N, default_bc=w.default_bc, cfl=w.cfl, n_levels_max=1)
    s = _solver(w)
    s.set_velocity(w.c_observed)
    n_t = s.trace_len(w.t_final)
    _, obs = s.misfit_forward(w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final,
                              np.zeros((len(w.receivers), n_t)))
    c = w.c * (1.0 + 0.02 * np.random.default_rng(8).standard_normal(w.K))
    J_ref, g_ref = misfit_gradient(prob, c, w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final, obs)
    s.set_velocity(c)
    J, _ = s.misfit_forward(w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final, obs, n_checkpoints=4)
    g = s.misfit_backward()
    assert abs(J - J_ref) < 1e-10 * J_ref
    assert rel_l2(g, g_ref) < 1e-9


@pytest.fixture(scope="module")
def box():
    w = adjoint_box()
    s = _solver(w)
    n_t = s.trace_len(w.t_final)
    s.set_velocity(adjoint_observed_velocity(w))
    _, obs = s.misfit_forward(w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final,
                              np.zeros((len(w.receivers), n_t)))
    s.set_velocity(w.c)
    return w, s, obs


def test_gradient_matches_finite_differences(box):
    w, s, obs = box
    J, _ = s.misfit_forward(w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final, obs, n_checkpoints=16)
    g = s.misfit_backward()
    assert J > 0 and np.all(np.isfinite(g)) and np.abs(g).max() > 0
    for k in np.random.default_rng(2).choice(w.K, 20, replace=False):
        d = 1e-4 * w.c[k]
        Js = []
        for sign in (1.0, -1.0):
            c = w.c.copy()
            c[k] += sign * d
            s.set_velocity(c)
            Js.append(s.misfit_forward(w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final, obs)[0])
        fd = (Js[0] - Js[1]) / (2 * d)
        assert abs(fd - g[k]) < 1e-5 * abs(g[k]) + 1e-8 * np.abs(g).max(), (k, fd, g[k])
    s.set_velocity(w.c)


def test_gradient_does_not_depend_on_the_checkpoints(box):
    w, s, obs = box
    grads = []
    for nc in (1, 7, 16, 300):
        s.misfit_forward(w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final, obs, n_checkpoints=nc)
        grads.append(s.misfit_backward())
    for g in grads[1:]:
        assert np.array_equal(g, grads[0])


def test_autograd_function(box):
    torch = pytest.importorskip("torch")
    w, s, obs = box
    c = torch.tensor(w.c, dtype=torch.float64, requires_grad=True)
    J = ridg.misfit(c, s, w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final, obs)
    (3.0 * J).backward()
    J2, _ = s.misfit_forward(w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final, obs)
    g = s.misfit_backward()
    assert J.detach().item() == J2
    assert np.array_equal(c.grad.numpy(), 3.0 * g)


def test_gradient_errors():
    w = adjoint_box_small()
    s = _solver(w)
    with pytest.raises(ridg.RidgError) as e:
        s.misfit_backward()  # no forward run yet
    assert e.value.code == -1
    t = tiny_layered_rtm(N=2)
    s3 = _solver(t, n_levels_max=3)
    assert s3.info.n_levels == 3
    outside = np.array([[1e5, 0.0, 0.0]])
    with pytest.raises(ridg.RidgError):
        s3.misfit_forward(t.source_xyz, t.f0, t.t_peak, 1.0, outside, 0.002, np.zeros((1, s3.trace_len(0.002))))
    with pytest.raises(ridg.RidgError):
        s.set_velocity(-w.c)


def test_fp32_gradient_follows_fp64(box):
    """The adjoint kernels in FP32 (CUDA cores for A^T, tensor cores for the forward steps) give the
    FP64 gradient to FP32 accuracy, relative to the gradient's size."""
    w, s64, obs = box
    s64.misfit_forward(w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final, obs)
    g64 = s64.misfit_backward()
    s32 = _solver(w, dtype="f32")
    J32, _ = s32.misfit_forward(w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final, obs)
    g32 = s32.misfit_backward()
    assert J32 > 0
    assert rel_l2(g32, g64) < 1e-3


@functools.lru_cache(maxsize=None)
def _multirate_reference(n_levels, N):
    w = (adjoint_box_two_level if n_levels == 2 else adjoint_box_three_level)()
    prob = make_problem(w.xyz, w.tets, w.c, w.rho, N, default_bc=w.default_bc, cfl=w.cfl, n_levels_max=n_levels)
    assert prob.n_levels == n_levels
    args = (w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final)
    obs = shot_misfit(prob, w.c_observed, *args, 0.0).traces
    J_ref, g_ref = misfit_gradient_levels(prob, w.c, *args, obs)
    return w, args, obs, J_ref, g_ref


@pytest.mark.parametrize("n_levels,N", [(2, 1), (3, 1), (3, 2)])
def test_multirate_gradient_matches_the_oracle(n_levels, N):
    """Two and three rate levels (24 elements, FP64; three levels use the mod-3 reuse of the inbox
    slots with a coarsest stride of 4, N = 2 the face-node paths of several nodes per face): the
    library's reverse accumulation over its fine steps (pull of the pushed traces, the update and
    right-hand-side transposes) against the oracle's, which assembles each fine step's matrix from
    its own Algorithm 1; and the same gradient bit for bit with 1, 3 and 16 checkpoints."""
    w, args, obs, J_ref, g_ref = _multirate_reference(n_levels, N)
    s = _solver(w, N=N, n_levels_max=n_levels)
    assert s.info.n_levels == n_levels
    grads = []
    for n_ck in (16, 3, 1):
        J, _ = s.misfit_forward(*args, obs, n_checkpoints=n_ck)
        assert abs(J - J_ref) < 1e-10 * J_ref
        grads.append(s.misfit_backward())
    assert rel_l2(grads[0], g_ref) < 1e-9
    assert np.array_equal(grads[0], grads[1]) and np.array_equal(grads[0], grads[2])


def test_multirate_gradient_fp32_follows_the_oracle():
    """The same three-level reverse sweep in FP32 (the precision of the bench): misfit and gradient
    against the FP64 oracle within 1e-3 relative (FP32 rounding accumulated over the forward run
    and the reverse sweep, as for the single-rate FP32 gradient)."""
    w, args, obs, J_ref, g_ref = _multirate_reference(3, 2)
    s = _solver(w, dtype="f32", N=2, n_levels_max=3)
    J, _ = s.misfit_forward(*args, obs, n_checkpoints=4)
    g = s.misfit_backward()
    assert abs(J - J_ref) < 1e-3 * J_ref
    assert rel_l2(g, g_ref) < 1e-3
