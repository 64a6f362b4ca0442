"""Reference tetrahedron of the nodal DG scheme (oracle, FP64, test infrastructure).

Follows Sec. 3.1 ("Nodal Discontinuous Galerkin Scheme") and the appendix of the paper:

* Nodes: Np = (N+1)(N+2)(N+3)/6 warp-and-blend nodes (Warburton 2006, cited in Sec. 3.1),
  pure warp-and-blend (no optimisation constant).
* Lagrange basis l_n on those nodes.  The oracle spans P_N with the homogeneous
  barycentric monomials lambda^alpha (|alpha| = N), whose exact integrals over a simplex
  are given by the Dirichlet formula  int_T lambda^a = |T| d! a! / (|a| + d)!.
* D_j = V_j V^{-1}  (derivative of the nodal interpolant, reference coordinate r_j).
* M   = V^{-T} G V^{-1} with the exact Gram matrix G of the monomials (the appendix's M_I).
* Face mass matrices on each face (2-D reference triangle of area 2) and
  LIFT = M^{-1} E, where E places each face mass matrix on that face's node rows
  (the appendix's M_k^{-1} M_{k,f} = (J_f/J_k) L_f).

Reference tetrahedron: v0 = (-1,-1,-1), v1 = (1,-1,-1), v2 = (-1,1,-1), v3 = (-1,-1,1);
barycentrics lambda_0 = -(1+r+s+t)/2, lambda_1 = (1+r)/2, lambda_2 = (1+s)/2,
lambda_3 = (1+t)/2.  Local face f spans the vertices FACE_VERTICES[f]; it is the set
lambda_{OPPOSITE[f]} = 0.
"""

from __future__ import annotations

from functools import lru_cache
from itertools import product
from math import factorial

import numpy as np
from numpy.polynomial import legendre as npleg

FACE_VERTICES = ((0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 2, 3))
OPPOSITE = (3, 2, 0, 1)
REF_VERTICES = np.array([[-1.0, -1.0, -1.0], [1.0, -1.0, -1.0], [-1.0, 1.0, -1.0], [-1.0, -1.0, 1.0]])
# d lambda_j / d r_i  (rows: r, s, t; columns: lambda_0..lambda_3)
DLAMBDA = np.array([[-0.5, 0.5, 0.0, 0.0], [-0.5, 0.0, 0.5, 0.0], [-0.5, 0.0, 0.0, 0.5]])
REF_VOLUME = 4.0 / 3.0
REF_FACE_AREA_2D = 2.0  # every face is integrated over a 2-D reference triangle of area 2


def n_nodes(N: int) -> int:
    return (N + 1) * (N + 2) * (N + 3) // 6


def n_face_nodes(N: int) -> int:
    return (N + 1) * (N + 2) // 2


def barycentric(rst: np.ndarray) -> np.ndarray:
    r, s, t = rst[..., 0], rst[..., 1], rst[..., 2]
    return np.stack([-(1 + r + s + t) / 2, (1 + r) / 2, (1 + s) / 2, (1 + t) / 2], axis=-1)


# ---------------------------------------------------------------- 1-D Gauss-Lobatto points
def gauss_lobatto(N: int) -> np.ndarray:
    """N+1 Gauss-Lobatto-Legendre points on [-1, 1], ascending: +-1 and the roots of P_N'."""
    if N == 0:
        return np.array([0.0])
    if N == 1:
        return np.array([-1.0, 1.0])
    c = np.zeros(N + 1)
    c[N] = 1.0
    inner = np.sort(np.real(npleg.legroots(npleg.legder(c))))
    return np.concatenate([[-1.0], inner, [1.0]])


def warp_factor(N: int, r: np.ndarray) -> np.ndarray:
    """Blend-divided 1-D warp (Warburton 2006): w(r) / (1 - r^2), where w is the degree-N
    interpolant through the equidistant nodes of the displacement to the GLL nodes.
    Zero at r = +-1."""
    req = np.linspace(-1.0, 1.0, N + 1)
    d = gauss_lobatto(N) - req
    w = np.zeros_like(r, dtype=np.float64)
    for i in range(N + 1):
        li = np.ones_like(r, dtype=np.float64)
        for j in range(N + 1):
            if j != i:
                li = li * (r - req[j]) / (req[i] - req[j])
        w = w + d[i] * li
    inside = np.abs(r) < 1.0 - 1e-10
    out = np.zeros_like(w)
    out[inside] = w[inside] / (1.0 - r[inside] ** 2)
    return out


# --------------------------------------------------------------------- nodes in 3-D
_EQUI = np.array(
    [[-1.0, -1.0 / np.sqrt(3.0), -1.0 / np.sqrt(6.0)], [1.0, -1.0 / np.sqrt(3.0), -1.0 / np.sqrt(6.0)],
     [0.0, 2.0 / np.sqrt(3.0), -1.0 / np.sqrt(6.0)], [0.0, 0.0, 3.0 / np.sqrt(6.0)]]
)


def equidistant_rst(N: int) -> np.ndarray:
    """Equidistant lattice of the reference tetrahedron; t slowest, then s, r fastest."""
    pts = []
    for k in range(N + 1):
        for j in range(N + 1 - k):
            for i in range(N + 1 - j - k):
                if N == 0:
                    pts.append([-0.5, -0.5, -0.5])
                else:
                    pts.append([-1 + 2.0 * i / N, -1 + 2.0 * j / N, -1 + 2.0 * k / N])
    return np.array(pts)


def nodes(N: int) -> np.ndarray:
    """Warp-and-blend nodes (Np, 3) in reference coordinates, equidistant lattice order.

    Each face contributes the 2-D warp of its three edges (edge A->B moves a point along
    unit(B-A) by 4 l_A l_B warp_factor(l_B - l_A)), blended into the volume with
    l_P l_Q l_R / ((l_P + l_O/2)(l_Q + l_O/2)(l_R + l_O/2)) (O = opposite vertex).
    Points on an edge take the unblended edge warp (the blend is 0/0 there).
    """
    eq = equidistant_rst(N)
    if N <= 1:
        return eq
    lam = barycentric(eq)
    X = lam @ _EQUI
    shift = np.zeros_like(X)
    tol = 1e-10
    on_edge = np.sum(lam > tol, axis=1) == 2
    edge_shift = np.zeros_like(X)
    for f in range(4):
        P, Q, R = FACE_VERTICES[f]
        O = OPPOSITE[f]
        warp = np.zeros_like(X)
        for A, B in ((P, Q), (Q, R), (R, P)):
            t = _EQUI[B] - _EQUI[A]
            t = t / np.linalg.norm(t)
            amount = 4.0 * lam[:, A] * lam[:, B] * warp_factor(N, lam[:, B] - lam[:, A])
            warp += amount[:, None] * t[None, :]
        num = lam[:, P] * lam[:, Q] * lam[:, R]
        den = (lam[:, P] + 0.5 * lam[:, O]) * (lam[:, Q] + 0.5 * lam[:, O]) * (lam[:, R] + 0.5 * lam[:, O])
        blend = np.where(den > tol, num / np.where(den > tol, den, 1.0), 0.0)
        shift += blend[:, None] * warp
        face_edge = on_edge & (lam[:, O] < tol)
        edge_shift[face_edge] = warp[face_edge]
    shift[on_edge] = edge_shift[on_edge]
    Xw = X + shift
    # back to reference coordinates: X = (v1+v2+v3-v0)/2 + (r v1' + s v2' + t v3')/2
    A = 0.5 * np.stack([_EQUI[1] - _EQUI[0], _EQUI[2] - _EQUI[0], _EQUI[3] - _EQUI[0]], axis=1)
    rhs = Xw - 0.5 * (_EQUI[1] + _EQUI[2] + _EQUI[3] - _EQUI[0])
    return np.linalg.solve(A, rhs.T).T


# ------------------------------------------------------------ barycentric monomials
def multi_indices(N: int, d: int):
    return [a for a in product(range(N + 1), repeat=d) if sum(a) == N]


def _mono(lam: np.ndarray, alphas) -> np.ndarray:
    return np.stack([np.prod(lam ** np.array(a)[None, :], axis=1) for a in alphas], axis=1)


def _mono_grad(lam: np.ndarray, alphas, dlam_row: np.ndarray) -> np.ndarray:
    cols = []
    for a in alphas:
        a = np.array(a)
        g = np.zeros(lam.shape[0])
        for j in range(lam.shape[1]):
            if a[j] == 0 or dlam_row[j] == 0.0:
                continue
            am = a.copy()
            am[j] -= 1
            g = g + a[j] * dlam_row[j] * np.prod(lam ** am[None, :], axis=1)
        cols.append(g)
    return np.stack(cols, axis=1)


def _gram(alphas, measure: float, d: int) -> np.ndarray:
    """Exact int over a d-simplex of measure `measure` of lambda^a lambda^b (Dirichlet)."""
    n = len(alphas)
    G = np.zeros((n, n))
    for i, a in enumerate(alphas):
        for j, b in enumerate(alphas):
            s = [x + y for x, y in zip(a, b)]
            num = factorial(d)
            for x in s:
                num *= factorial(x)
            G[i, j] = measure * num / factorial(sum(s) + d)
    return G


class ReferenceElement:
    """All reference operators for order N (FP64)."""

    def __init__(self, N: int):
        if N < 1:
            raise ValueError("N >= 1")
        self.N = N
        self.Np = n_nodes(N)
        self.Nfp = n_face_nodes(N)
        self.rst = nodes(N)
        lam = barycentric(self.rst)
        self.alphas = multi_indices(N, 4)
        V = _mono(lam, self.alphas)
        self.V = V
        Vinv = np.linalg.inv(V)
        # differentiation matrices D_r, D_s, D_t
        self.D = np.stack([_mono_grad(lam, self.alphas, DLAMBDA[i]) @ Vinv for i in range(3)])
        G = _gram(self.alphas, REF_VOLUME, 3)
        self.M = Vinv.T @ G @ Vinv
        self.Minv = np.linalg.inv(self.M)
        # face node masks
        self.Fmask = np.zeros((4, self.Nfp), dtype=np.int64)
        for f in range(4):
            idx = np.nonzero(np.abs(lam[:, OPPOSITE[f]]) < 1e-10)[0]
            if len(idx) != self.Nfp:
                raise RuntimeError("face node count mismatch")
            self.Fmask[f] = idx
        # face mass matrices on a 2-D reference triangle of area 2
        beta = multi_indices(N, 3)
        Gf = _gram(beta, REF_FACE_AREA_2D, 2)
        self.Mface = np.zeros((4, self.Nfp, self.Nfp))
        for f in range(4):
            mu = lam[self.Fmask[f]][:, list(FACE_VERTICES[f])]
            Vf = _mono(mu, beta)
            Vfi = np.linalg.inv(Vf)
            self.Mface[f] = Vfi.T @ Gf @ Vfi
        E = np.zeros((self.Np, 4 * self.Nfp))
        for f in range(4):
            for i in range(self.Nfp):
                E[self.Fmask[f][i], f * self.Nfp:(f + 1) * self.Nfp] = self.Mface[f][i]
        self.E = E
        self.LIFT = self.Minv @ E

    def lagrange_at(self, rst_pts: np.ndarray) -> np.ndarray:
        """Values of the Np Lagrange basis functions at reference points (n_pts, Np)."""
        lam = barycentric(np.atleast_2d(rst_pts))
        phi = _mono(lam, self.alphas)
        return np.linalg.solve(self.V.T, phi.T).T


@lru_cache(maxsize=None)
def reference_element(N: int) -> ReferenceElement:
    return ReferenceElement(N)
