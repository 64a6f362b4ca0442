"""Pins of the oracle's geometry (appendix) and right-hand side (Eqs. dgLocalSchemeP/U,
weakFormP/V) against chain-rule identities, the semi-discrete energy balance and the
backward-in-time symmetry."""

import numpy as np
import pytest

from oracle.dg_rhs import attach_media, energy, rhs, traces
from oracle.mesh_geometry import MeshGeometry
from oracle.reference_element import reference_element
from synth import unit_cube_mesh, tiny_layered_rtm
from synth.meshes import HexGrid


def _geo(xyz, tets, N=3, bc=3, c=None, rho=None, face_bc=None):
    K = len(tets)
    g = MeshGeometry(xyz, tets, reference_element(N), face_bc=face_bc, default_bc=bc)
    return attach_media(g, np.ones(K) if c is None else c, np.ones(K) if rho is None else rho)


def test_inverse_jacobian_on_sheared_tet():
    """d/dx_i of the coordinate functions: the chain rule with d r_j/d x_i gives delta_ij."""
    xyz = np.array([[0.1, 0.2, 0.0], [1.3, 0.1, 0.2], [0.4, 1.1, -0.1], [0.2, 0.5, 0.9]])
    g = _geo(xyz, np.array([[0, 1, 2, 3]]), N=2)
    x = g.x[0]
    for i in range(3):
        Dr = np.stack([g.ref.D[j] @ x[:, i] for j in range(3)])  # [j, n]
        for m in range(3):
            deriv = np.einsum("j,jn->n", g.rx[0, m], Dr)
            assert np.allclose(deriv, 1.0 if m == i else 0.0, atol=1e-12)


def test_normals_areas_volume():
    xyz, tets = unit_cube_mesh(2)
    g = _geo(xyz, tets)
    assert np.allclose(np.linalg.norm(g.normal, axis=2), 1.0)
    # closed surface: sum of area-weighted normals vanishes
    assert np.allclose(np.einsum("kf,kfd->kd", g.area, g.normal), 0.0, atol=1e-14)
    assert np.isclose(g.volume.sum(), 1.0)
    # outward: the normal points away from the opposite vertex
    cen = g.P.mean(axis=1)
    for f in range(4):
        fc = g.x[:, g.ref.Fmask[f]].mean(axis=1)
        assert np.all(np.einsum("kd,kd->k", g.normal[:, f], fc - cen) > 0)


def test_cube_connectivity():
    xyz, tets = unit_cube_mesh(4)
    g = _geo(xyz, tets)
    n_boundary = int(np.sum(g.nbr < 0))
    assert n_boundary == 6 * 16 * 2
    # matched face nodes coincide and the neighbour relation is symmetric
    for k in range(g.K):
        for f in range(4):
            k2 = g.nbr[k, f]
            if k2 < 0:
                continue
            f2 = g.nbr_face[k, f]
            assert g.nbr[k2, f2] == k and g.nbr_face[k2, f2] == f
            xa = g.x[k, g.ref.Fmask[f]]
            xb = g.x[k2, g.ref.Fmask[f2][g.nbr_node[k, f]]]
            assert np.allclose(xa, xb, atol=1e-13)
            assert np.allclose(g.normal[k, f], -g.normal[k2, f2], atol=1e-14)


def _dEdt(g, q, r):
    M = g.ref.M
    ep = np.einsum("kn,nm,km->k", q[:, 0], M, r[:, 0]) / (g.rho * g.c ** 2)
    ev = g.rho * np.einsum("kin,nm,kim->k", q[:, 1:], M, r[:, 1:])
    return float(np.sum(g.J * (ep + ev)))


def _face_dissipation(g, q, sign=1.0):
    """-1/2 sum over interior faces int (tau_p [p]^2 + tau_v [n.v]^2) plus the boundary terms:
    free -int tau_p p^2, transparent -1/2 int (tau_p p^2 + tau_v (n.v)^2), rigid -int tau_v (n.v)^2,
    each face integral computed with the face mass matrix times J_f."""
    qf = traces(q, g)
    total = 0.0
    for k in range(g.K):
        for f in range(4):
            Mf = g.ref.Mface[f] * g.Jf[k, f]
            p, v = qf[k, 0, f], qf[k, 1, f]
            k2 = g.nbr[k, f]
            Zk = g.rho[k] * g.c[k]
            if k2 >= 0:
                if k2 < k:
                    continue  # each interior face once
                f2 = g.nbr_face[k, f]
                j = g.nbr_node[k, f]
                jp = qf[k2, 0, f2, j] - p
                jv = -qf[k2, 1, f2, j] - v
                Zb = 0.5 * (Zk + g.rho[k2] * g.c[k2])
                total -= 0.5 * sign * (jp @ Mf @ jp / Zb + Zb * jv @ Mf @ jv)
            else:
                bc = g.bc[k, f]
                if bc == 1:
                    total -= sign * (p @ Mf @ p) / Zk
                elif bc == 2:
                    total -= 0.5 * sign * (p @ Mf @ p / Zk + Zk * v @ Mf @ v)
                else:
                    total -= sign * Zk * (v @ Mf @ v)
    return total


@pytest.mark.parametrize("bc", [1, 2, 3])
def test_semidiscrete_energy_balance(bc):
    """dE/dt from the right-hand side equals the penalty dissipation (exact with face-mass
    quadrature); holds only with the 1/2 of the weak form and the stated ghost states."""
    xyz, tets = unit_cube_mesh(2)
    g = _geo(xyz, tets, N=3, bc=bc)
    q = np.random.default_rng(1).standard_normal((g.K, 4, g.ref.Np))
    r = rhs(np.arange(g.K), q, traces(q, g), g)
    lhs, rhs_ = _dEdt(g, q, r), _face_dissipation(g, q)
    assert rhs_ < 0
    assert np.isclose(lhs, rhs_, rtol=1e-10)


def test_energy_balance_two_materials():
    """Heterogeneous interface: tau from the mean impedance keeps the balance exact."""
    xyz, tets = unit_cube_mesh(2)
    K = len(tets)
    rng = np.random.default_rng(3)
    c = rng.uniform(1.0, 3.0, K)
    rho = rng.uniform(0.5, 2.0, K)
    g = _geo(xyz, tets, N=2, bc=2, c=c, rho=rho)
    q = rng.standard_normal((g.K, 4, g.ref.Np))
    r = rhs(np.arange(g.K), q, traces(q, g), g)
    assert np.isclose(_dEdt(g, q, r), _face_dissipation(g, q), rtol=1e-10)


def test_linear_pressure_gradient_exact():
    """p = a.x, v = 0 is continuous across faces, so r_v = -a/rho and r_p = 0 in the interior."""
    xyz, tets = unit_cube_mesh(3)
    g = _geo(xyz, tets, N=2, bc=3, rho=np.full(len(tets), 2.0))
    a = np.array([0.3, -1.2, 0.7])
    q = np.zeros((g.K, 4, g.ref.Np))
    q[:, 0] = g.x @ a
    r = rhs(np.arange(g.K), q, traces(q, g), g)
    interior = np.all(g.nbr >= 0, axis=1)
    assert interior.sum() > 0
    for i in range(3):
        assert np.allclose(r[interior, 1 + i], -a[i] / 2.0, atol=1e-12)
    assert np.allclose(r[interior, 0], 0.0, atol=1e-12)


def test_backward_symmetry_of_rhs():
    """r_p(p, v; -tau) = -r_p(p, -v; tau) and r_v(p, v; -tau) = r_v(p, -v; tau) on every face type."""
    w = tiny_layered_rtm()
    K = len(w.tets)
    fb = np.zeros((K, 4), dtype=np.int64)
    g0 = _geo(w.xyz, w.tets, N=2, bc=2, c=w.c, rho=w.rho)
    bnd = np.nonzero(g0.nbr < 0)
    fb[bnd] = np.random.default_rng(0).integers(1, 4, len(bnd[0]))
    g = _geo(w.xyz, w.tets, N=2, bc=2, c=w.c, rho=w.rho, face_bc=fb)
    q = np.random.default_rng(5).standard_normal((g.K, 4, g.ref.Np))
    qm = q.copy()
    qm[:, 1:] *= -1
    E = np.arange(g.K)
    rb = rhs(E, q, traces(q, g), g, sign=-1.0)
    rf = rhs(E, qm, traces(qm, g), g, sign=1.0)
    assert np.allclose(rb[:, 0], -rf[:, 0], rtol=1e-12, atol=1e-9)
    assert np.allclose(rb[:, 1:], rf[:, 1:], rtol=1e-12, atol=1e-12)


def test_point_source_projection():
    """Eq. sourceTerm: the projected Dirac integrates to 1 and reproduces point values of
    every polynomial of degree <= N; dp/dt += f w therefore injects f per unit time."""
    xyz = np.array([[0.0, 0.0, 0.0], [2.0, 0.1, 0.0], [0.3, 1.7, 0.2], [0.1, 0.4, 1.5]])
    g = _geo(xyz, np.array([[0, 1, 2, 3]]), N=3)
    x0 = np.array([0.5, 0.5, 0.3])
    k, rst = g.locate(x0)
    assert k == 0
    w = g.source_weights(k, rst)
    Mk = g.J[0] * g.ref.M
    assert np.isclose(np.sum(Mk @ w), 1.0)
    xn = g.x[0]
    for poly in (lambda x: x[..., 0] ** 2 * x[..., 1], lambda x: 1 + x[..., 2] ** 3, lambda x: x[..., 0] * x[..., 1] * x[..., 2]):
        assert np.isclose(poly(xn) @ Mk @ w, poly(x0), rtol=1e-10)
    # interpolation row reproduces the same values
    row = g.interpolation_row(rst)
    assert np.isclose(row @ (xn[:, 0] ** 3), x0[0] ** 3)


def test_locate_ties_take_lowest_index():
    xyz, tets = unit_cube_mesh(2)
    g = _geo(xyz, tets)
    k, _ = g.locate([0.5, 0.5, 0.5])  # a shared vertex
    owners = [e for e in range(g.K) if np.any(np.all(np.isclose(g.P[e], [0.5, 0.5, 0.5]), axis=1))]
    assert k == min(owners)
    assert g.locate([2.0, 0.0, 0.0])[0] == -1


@pytest.mark.parametrize("bc", [1, 2, 3])
def test_energy_rate_is_linear_in_the_penalty_scale(bc):
    """Scaling tau_p and tau_v by s scales every face's energy loss by s: the central flux
    (s = 0) conserves the discrete energy exactly, s = 2.5 loses 2.5 times the upwind loss."""
    xyz, tets = unit_cube_mesh(2)
    g = _geo(xyz, tets, N=3, bc=bc)
    q = np.random.default_rng(5).standard_normal((g.K, 4, g.ref.Np))
    upwind = _face_dissipation(g, q)
    for s in (0.0, 2.5):
        g.tau_scale = s
        r = rhs(np.arange(g.K), q, traces(q, g), g)
        assert abs(_dEdt(g, q, r) - s * upwind) < 1e-10 * abs(upwind)
