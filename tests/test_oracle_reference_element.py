"""Pins of the oracle's reference element (Sec. 3.1 and the appendix) against closed forms,
exact integrals and identities that a wrong index, sign or scale would break."""

from fractions import Fraction
from itertools import permutations

import numpy as np
import pytest
from scipy import integrate

from oracle.reference_element import (FACE_VERTICES, OPPOSITE, ReferenceElement, barycentric, gauss_lobatto,
                                      n_face_nodes, n_nodes)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
def test_node_counts_and_faces(N):
    re = ReferenceElement(N)
    assert re.Np == (N + 1) * (N + 2) * (N + 3) // 6 == n_nodes(N)
    assert re.Nfp == (N + 1) * (N + 2) // 2 == n_face_nodes(N)
    lam = barycentric(re.rst)
    assert np.all(lam > -1e-12)
    for f in range(4):
        assert np.allclose(lam[re.Fmask[f], OPPOSITE[f]], 0.0, atol=1e-12)


def test_salt_dome_count_identity():
    """Sec. 5.2: 2,787,335 tetrahedra at N=3 give 222,986,800 unknowns with 4 fields."""
    vals = dict(line.split() for line in open("tests/golden/model_counts.txt") if line[0] != "#")
    assert int(vals["K"]) * n_nodes(int(vals["N"])) * 4 == int(vals["unknowns"])


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6])
def test_edge_nodes_are_gauss_lobatto(N):
    """Warp-and-blend places the Gauss-Lobatto-Legendre points on every edge."""
    re = ReferenceElement(N)
    lam = barycentric(re.rst)
    gll = gauss_lobatto(N)
    for a in range(4):
        for b in range(a + 1, 4):
            others = [i for i in range(4) if i not in (a, b)]
            on = np.all(np.abs(lam[:, others]) < 1e-12, axis=1)
            r = np.sort(lam[on, b] - lam[on, a])
            assert len(r) == N + 1
            assert np.allclose(r, gll, atol=1e-13)


def test_gauss_lobatto_small_cases():
    assert np.allclose(gauss_lobatto(2), [-1, 0, 1])
    assert np.allclose(gauss_lobatto(3), [-1, -1 / np.sqrt(5), 1 / np.sqrt(5), 1])
    assert np.allclose(gauss_lobatto(4), [-1, -np.sqrt(3 / 7), 0, np.sqrt(3 / 7), 1])


@pytest.mark.parametrize("N", [3, 4, 5])
def test_node_set_symmetric(N):
    """The node set is invariant under every permutation of the four vertices."""
    lam = barycentric(ReferenceElement(N).rst)
    key = lambda L: set(tuple(np.round(row, 10)) for row in L)  # noqa: E731
    base = key(lam)
    for perm in permutations(range(4)):
        assert key(lam[:, list(perm)]) == base


def _monomials(N):
    return [(a, b, c) for a in range(N + 1) for b in range(N + 1 - a) for c in range(N + 1 - a - b)]


@pytest.mark.parametrize("N", [1, 3, 4, 6])
def test_differentiation_exact(N):
    """D_r, D_s, D_t differentiate every polynomial of degree <= N exactly."""
    re = ReferenceElement(N)
    r, s, t = re.rst.T
    for a, b, c in _monomials(N):
        f = r ** a * s ** b * t ** c
        grads = [a * r ** max(a - 1, 0) * s ** b * t ** c, b * r ** a * s ** max(b - 1, 0) * t ** c,
                 c * r ** a * s ** b * t ** max(c - 1, 0)]
        for j in range(3):
            assert np.allclose(re.D[j] @ f, grads[j], atol=1e-9 * (1 + np.abs(grads[j]).max()))


def _tet_integral(fun):
    # reference tetrahedron: r, s, t >= -1, r + s + t <= -1
    val, _ = integrate.tplquad(lambda t, s, r: fun(r, s, t), -1, 1, lambda r: -1, lambda r: -r,
                               lambda r, s: -1, lambda r, s: -1 - r - s, epsabs=1e-13, epsrel=1e-13)
    return val


@pytest.mark.parametrize("N", [2, 3])
def test_mass_matrix_integrates_products(N):
    """f^T M g equals the exact integral of f g for polynomials f, g of degree <= N
    (checked against adaptive cubature, which shares nothing with the Dirichlet formula)."""
    re = ReferenceElement(N)
    r, s, t = re.rst.T
    assert np.isclose(np.sum(re.M), 4.0 / 3.0, atol=1e-14)
    cases = [((1, 0, 0), (0, 1, 1)), ((N, 0, 0), (0, 0, N)), ((0, 1, 0), (1, 0, 1))]
    for (a1, b1, c1), (a2, b2, c2) in cases:
        f = r ** a1 * s ** b1 * t ** c1
        g = r ** a2 * s ** b2 * t ** c2
        exact = _tet_integral(lambda x, y, z: x ** (a1 + a2) * y ** (b1 + b2) * z ** (c1 + c2))
        assert np.isclose(f @ re.M @ g, exact, atol=1e-12)
    w = np.linalg.eigvalsh(re.M)
    assert w.min() > 0


@pytest.mark.parametrize("N", [1, 3, 5])
def test_integration_by_parts(N):
    """M D_j + (M D_j)^T equals the boundary integral sum_f n_j,f |F_f|/2 E_f (face masses on
    a 2-D triangle of area 2; reference face areas 2, 2, 2 sqrt(3), 2)."""
    re = ReferenceElement(N)
    normals = np.array([[0, 0, -1], [0, -1, 0], [1, 1, 1] / np.sqrt(3), [-1, 0, 0]])
    areas = np.array([2.0, 2.0, 2.0 * np.sqrt(3.0), 2.0])
    for j in range(3):
        lhs = re.M @ re.D[j]
        lhs = lhs + lhs.T
        rhs = np.zeros_like(lhs)
        for f in range(4):
            Ef = np.zeros_like(lhs)
            Fm = re.Fmask[f]
            Ef[np.ix_(Fm, Fm)] = re.Mface[f]
            rhs += normals[f, j] * areas[f] / 2.0 * Ef
        assert np.allclose(lhs, rhs, atol=1e-11)


def test_face_mass_exact():
    """On a triangle of area A, int lambda_1^2 = A/6 and int lambda_1 lambda_2 = A/12."""
    re = ReferenceElement(3)
    lam = barycentric(re.rst)
    for f in range(4):
        P, Q, _ = FACE_VERTICES[f]
        mu = lam[re.Fmask[f]]
        one = np.ones(re.Nfp)
        assert np.isclose(one @ re.Mface[f] @ one, 2.0)
        assert np.isclose(mu[:, P] @ re.Mface[f] @ mu[:, P], 2.0 / 6.0)
        assert np.isclose(mu[:, P] @ re.Mface[f] @ mu[:, Q], 2.0 / 12.0)


def test_lift_is_inverse_mass_times_face_mass():
    re = ReferenceElement(4)
    assert np.allclose(re.M @ re.LIFT, re.E, atol=1e-12)
    # the lift of a constant face function is the same on every node set ordering
    for f in range(4):
        col = re.LIFT[:, f * re.Nfp:(f + 1) * re.Nfp] @ np.ones(re.Nfp)
        assert np.isclose(np.sum(re.M @ col), 2.0)


@pytest.mark.parametrize("N", [2, 4])
def test_lagrange_basis_interpolates(N):
    re = ReferenceElement(N)
    assert np.allclose(re.lagrange_at(re.rst), np.eye(re.Np), atol=1e-10)
    # partition of unity at an arbitrary point
    assert np.isclose(re.lagrange_at(np.array([[-0.3, -0.4, -0.5]])).sum(), 1.0)
