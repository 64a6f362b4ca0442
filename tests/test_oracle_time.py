"""Pins of the oracle's time stepping (Sec. 3.2, Algorithm 1) and image integration
(Sec. 3.3): printed constants, the closed-form standing mode, convergence orders, LTS
reductions and the backward-in-time symmetry."""

from fractions import Fraction

import numpy as np
import pytest

from oracle.dg_rhs import attach_media, energy, rhs, traces
from oracle.imaging import C_MAT, C_VEC, characteristic, step_increment
from oracle.mesh_geometry import MeshGeometry
from oracle.mrab import AB_A, AB_B, MRAB, assign_levels
from oracle.reference_element import reference_element
from oracle.rtm import make_problem
from oracle.wavelet import cubic_weights, interpolate_trace, ricker
from synth import config1_cube, standing_mode, tiny_layered_rtm, unit_cube_mesh


def _golden():
    rows = {}
    for line in open("tests/golden/ab3_coefficients.txt"):
        if line.startswith("#") or not line.strip():
            continue
        key, *vals = line.split()
        rows.setdefault(key, []).append([Fraction(v) for v in vals])
    return rows


def test_printed_coefficients():
    """a = A(1), b = A(1/2) and C_ij = int_0^1 A_i A_j reproduce the printed values exactly."""
    g = _golden()
    assert tuple(g["a"][0]) == AB_A
    assert tuple(g["b"][0]) == AB_B
    assert tuple(tuple(r) for r in g["C"]) == C_MAT
    assert C_VEC == (Fraction(19, 24), Fraction(-5, 12), Fraction(1, 8))
    assert sum(C_VEC) == Fraction(1, 2) and sum(sum(r) for r in C_MAT) == Fraction(1, 3)


def test_step_increment_exact_against_quadrature():
    """Gauss-Legendre integration of the product of two AB3 interpolants."""
    rng = np.random.default_rng(0)
    xg, wg = np.polynomial.legendre.leggauss(8)
    for h in (0.37, -0.21):
        xS, xR = rng.standard_normal(2)
        rS, rR = rng.standard_normal(3), rng.standard_normal(3)
        tau = 0.5 * (xg + 1.0)
        # A_s(tau) from the exact a-type polynomials: integrate l_s from 0
        def A(s, t):
            nodes = [0.0, -1.0, -2.0]
            xx = np.linspace(0, 1, 1)
            # l_s via Lagrange; integrate numerically with a fine Gauss rule on [0, t]
            xs, ws = np.polynomial.legendre.leggauss(8)
            u = 0.5 * t * (xs + 1.0)
            ls = np.ones_like(u)
            for j, nj in enumerate(nodes):
                if j != s:
                    ls *= (u - nj) / (nodes[s] - nj)
            return 0.5 * t * np.sum(ws * ls)
        fS = [xS + h * sum(A(s, t) * rS[s] for s in range(3)) for t in tau]
        fR = [xR + h * sum(A(s, t) * rR[s] for s in range(3)) for t in tau]
        brute = h * 0.5 * np.sum(wg * np.array(fS) * np.array(fR))
        assert np.isclose(step_increment(h, xS, list(rS), xR, list(rR)), brute, rtol=1e-13)


def test_image_of_constant_fields():
    """p_S = p_R = 1 (zero right-hand sides): the negated backward increments sum to t_f - t_i."""
    h = -0.01
    total = 0.0
    for _ in range(37):
        total -= step_increment(h, 1.0, [0, 0, 0], 1.0, [0, 0, 0])
    assert np.isclose(total, 0.37)


def test_characteristic_plane_wave():
    """A purely up-going wave (p = Z e_up.v) has q^- = 0: it leaves no trace in I_Q from S."""
    Z = np.array([2.5e6])
    v = np.zeros((1, 3, 4))
    v[0, 2] = -np.linspace(1, 2, 4)  # e_up = (0,0,-1): e_up.v = -v_z
    p = Z[0] * np.einsum("d,dn->n", [0, 0, -1], v[0])[None]
    assert np.allclose(characteristic(p, v, Z, (0, 0, -1), -1.0), 0.0)
    assert np.allclose(characteristic(p, v, Z, (0, 0, -1), +1.0), 2 * p)


def test_ricker_and_cubic_interpolation():
    assert np.isclose(ricker(0.2, 10.0, 0.2), 1.0)
    assert abs(ricker(0.0, 10.0, 0.13524)) < 1e-6
    # cubic interpolation is exact on cubics and returns samples at sample times
    n_local = 4
    tr = np.array([(n - 3.0) ** 3 - n for n in range(12)], dtype=float)
    for tau in range(4, 32):
        u = tau / n_local
        assert np.isclose(interpolate_trace(tr, tau, n_local), (u - 3.0) ** 3 - u)
    n0, w = cubic_weights(8, 4)
    assert n0 == 1 and np.allclose(w, [0, 1, 0, 0])


def _standing_setup(n, N, cfl=0.15, levels=None):
    xyz, tets = unit_cube_mesh(n)
    K = len(tets)
    g = attach_media(MeshGeometry(xyz, tets, reference_element(N), default_bc=3), np.ones(K), np.ones(K))
    lev, nl, dtl = assign_levels(g, N, np.ones(K), cfl, 1)
    x = g.x
    sm = lambda t: np.stack(standing_mode(x[..., 0], x[..., 1], x[..., 2], t), axis=1)  # noqa: E731
    r_of = lambda q: rhs(np.arange(K), q, traces(q, g), g)  # noqa: E731
    return g, lev, nl, dtl, sm, r_of


def _single_rate(g, q0, r1, r2, dt, steps):
    """Plain single-rate AB3 (Eq. updateAB with one level), written out on its own."""
    K = g.K
    q = q0.copy()
    hist = [r1, r2]
    for _ in range(steps):
        r0 = rhs(np.arange(K), q, traces(q, g), g)
        q = q + dt * (23.0 / 12.0 * r0 - 16.0 / 12.0 * hist[0] + 5.0 / 12.0 * hist[1])
        hist = [r0, hist[0]]
    return q


def test_config1_closed_form_and_energy():
    """Unit cube, 384 tets, N=3, rigid walls, 200 steps: error vs the standing mode and a
    non-increasing discrete energy."""
    w = config1_cube()
    g, lev, nl, dtl, sm, r_of = _standing_setup(4, 3, w.cfl)
    assert nl == 1 and np.all(lev == 1)
    st = MRAB(g, lev, nl, dtl)
    st.set_state(sm(0.0))
    st.set_history(r_of(sm(-dtl)), r_of(sm(-2 * dtl)))
    e0 = energy(st.q, g)
    es = []
    for _ in range(w.n_steps):
        st.global_step()
        es.append(energy(st.q, g))
    # AB3 is a multistep method: its state energy is not monotone step by step (single steps
    # grow by ~1e-8), but it stays bounded by the initial energy and decays overall.
    assert max(es) <= e0 * (1 + 1e-6)
    assert es[-1] < e0
    qe = sm(st.time())
    err = np.linalg.norm(st.q[:, 0] - qe[:, 0]) / np.linalg.norm(qe[:, 0])
    assert 1e-4 < err < 2e-2


def test_mrab_one_level_equals_single_rate():
    g, lev, nl, dtl, sm, r_of = _standing_setup(2, 3)
    st = MRAB(g, lev, nl, dtl)
    st.set_state(sm(0.0))
    r1, r2 = r_of(sm(-dtl)), r_of(sm(-2 * dtl))
    st.set_history(r1, r2)
    for _ in range(25):
        st.global_step()
    q = _single_rate(g, sm(0.0), r1, r2, dtl, 25)
    assert np.allclose(st.q, q, rtol=0, atol=1e-13)


def test_mrab_all_finest_equals_single_rate_small_step():
    """All elements forced onto level 3 of 3: identical to single-rate AB3 at Delta t_local."""
    g, lev, nl, dtl, sm, r_of = _standing_setup(2, 2)
    lev3 = np.full(g.K, 3)
    st = MRAB(g, lev3, 3, dtl)
    st.set_state(sm(0.0))
    r1, r2 = r_of(sm(-dtl)), r_of(sm(-2 * dtl))
    st.set_history(r1, r2)
    for _ in range(6):
        st.global_step()
    q = _single_rate(g, sm(0.0), r1, r2, dtl, 24)
    assert np.allclose(st.q, q, rtol=0, atol=1e-13)


def test_two_level_third_order_in_time():
    """Half the elements on the coarse level: the difference to single-rate at the fine step
    shrinks like Delta t^3 (the half-step traces keep the multi-rate scheme third order)."""
    xyz, tets = unit_cube_mesh(2)
    K = len(tets)
    g = attach_media(MeshGeometry(xyz, tets, reference_element(2), default_bc=3), np.ones(K), np.ones(K))
    x = g.x
    sm = lambda t: np.stack(standing_mode(x[..., 0], x[..., 1], x[..., 2], t), axis=1)  # noqa: E731
    lev = np.where(g.P[:, :, 0].mean(axis=1) < 0.5, 1, 2)
    diffs = []
    T = 0.08
    for dt_fine in (T / 16, T / 32):
        st = MRAB(g, lev, 2, dt_fine)
        st.set_state(sm(0.0))
        r_of = lambda q: rhs(np.arange(K), q, traces(q, g), g)  # noqa: E731
        # exact-solution history per level
        for l, hl in ((1, 2 * dt_fine), (2, dt_fine)):
            E = lev == l
            st.hist[0][E] = r_of(sm(-hl))[E]
            st.hist[1][E] = r_of(sm(-2 * hl))[E]
        n = int(round(T / (2 * dt_fine)))
        for _ in range(n):
            st.global_step()
        ref = _single_rate(g, sm(0.0), r_of(sm(-dt_fine)), r_of(sm(-2 * dt_fine)), dt_fine, 2 * n)
        diffs.append(np.linalg.norm(st.q - ref))
    order = np.log2(diffs[0] / diffs[1])
    assert order > 2.5


@pytest.mark.slow
def test_spatial_convergence_order():
    """h^(N+1): standing mode at N=2 on 2, 4, 8 hexahedra per side (fixed small Delta t)."""
    errs = []
    T = 0.1
    for n in (2, 4, 8):
        g, lev, nl, dtl, sm, r_of = _standing_setup(n, 2)
        dt = T / 160
        q = _single_rate(g, sm(0.0), r_of(sm(-dt)), r_of(sm(-2 * dt)), dt, 160)
        qe = sm(T)
        errs.append(np.sqrt(np.sum(g.J[:, None] * (q[:, 0] - qe[:, 0]) ** 2)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders[-1] > 3.0 - 0.5


def test_backward_run_is_forward_run_of_reflected_state():
    """Sec. 3.2 backward stepping (Delta t < 0, tau < 0) equals the forward run of (p, -v) with
    source -f, to roundoff, on a 3-level mesh with half-steps."""
    w = tiny_layered_rtm(N=2)
    prob = make_problem(w.xyz, w.tets, w.c, w.rho, 2, default_bc=2, cfl=0.15)
    assert prob.n_levels == 3
    g = prob.geo
    rng = np.random.default_rng(7)
    q0 = rng.standard_normal((g.K, 4, g.ref.Np))
    ks, rs = g.locate(w.source_xyz)
    ws = g.source_weights(ks, rs)
    amp = lambda tau: float(ricker(tau * prob.dt_local, 60.0, 0.01))  # noqa: E731
    B = MRAB(g, prob.levels, 3, prob.dt_local, direction=-1, tau0=40)
    B.set_state(q0)
    B.injections = [(ks, ws, amp)]
    qm = q0.copy()
    qm[:, 1:] *= -1
    F = MRAB(g, prob.levels, 3, prob.dt_local, direction=+1, tau0=-40)
    F.set_state(qm)
    F.injections = [(ks, -ws, lambda tau: amp(-tau))]
    for _ in range(3):
        B.global_step()
        F.global_step()
    out = F.q.copy()
    out[:, 1:] *= -1
    assert np.allclose(B.q, out, rtol=1e-12, atol=1e-12 * np.abs(out).max())


def test_mrab_energy_non_increasing_three_levels():
    w = tiny_layered_rtm(N=2)
    prob = make_problem(w.xyz, w.tets, w.c, w.rho, 2, default_bc=2, cfl=0.15)
    g = prob.geo
    x = g.x
    q0 = np.zeros((g.K, 4, g.ref.Np))
    q0[:, 0] = np.exp(-((x - np.array([100.0, 100.0, 50.0])) ** 2).sum(-1) / (2 * 20.0 ** 2))
    st = MRAB(g, prob.levels, prob.n_levels, prob.dt_local)
    st.set_state(q0)
    e = [energy(st.q, g)]
    for _ in range(30):
        st.global_step()
        e.append(energy(st.q, g))
    assert max(e) <= e[0] * (1 + 1e-6) and e[-1] < e[0]


def test_serving_models_have_three_levels():
    """The shot-serving models use three rate levels (the smallest is checked here with the
    oracle's level rule; the larger ones use the same bands at a finer spacing)."""
    from oracle.dg_rhs import attach_media
    from oracle.mesh_geometry import MeshGeometry
    from oracle.mrab import assign_levels
    from oracle.reference_element import reference_element
    from synth import serving_model

    w = serving_model("50k")
    g = attach_media(MeshGeometry(w.xyz, w.tets, reference_element(1), default_bc=2), w.c, w.rho)
    lev, nl, _ = assign_levels(g, w.N, w.c, w.cfl, w.n_levels_max)
    assert nl == 3 and all(np.bincount(lev)[1:] > 0)
