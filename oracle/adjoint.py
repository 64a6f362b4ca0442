"""Least-squares misfit of one shot and its gradient with respect to the per-element velocity
(oracle, FP64, test infrastructure).

The paper migrates with the imaging condition alone; the gradient here extends its forward
scheme (Sec. 3.1 right-hand side, Sec. 3.2 Adams-Bashforth; ``misfit_gradient`` with one rate
level, ``misfit_gradient_levels`` with any number) with its exact discrete adjoint.  Readings (the
paper has no gradient, so each is a definition):

* Model parameter: the velocity c_k of each element where it enters the pressure equation,
  through rho_k c_k^2 (Eq. dgLocalSchemeP).  The time step, the rate level and the penalty
  parameters tau_p, tau_v (Sec. 3.1) stay those of the reference model the problem was built
  with: they are frozen, so the discrete scheme is a smooth function of c.  The recursion below
  is that of one rate level (single-rate AB3); several levels follow at the end.
* Misfit: J(c) = 1/2 Dt sum_{n=0}^{Nt} sum_r (y_r^n - d_r^n)^2 with the traces
  y_r^n = l(x_r) . p^n_{k_r} of the forward run at the global steps t_n = n Dt (Sec. 2) and the
  observed data d.
* Scheme: q^{n+1} = q^n + h sum_s a_s (A q^{n-s} + f(t_{n-s}) w), q^0 = 0 and zero history,
  with A the linear right-hand side operator, w the projected Dirac of the source.
* Lagrangian L = J + sum_n lambda^{n+1} . (q^{n+1} - q^n - h sum_s a_s (A q^{n-s} + f w)).
  Stationarity in q^m gives the adjoint recursion, run from m = Nt down to 1:
      lambda^m = lambda^{m+1} + h A^T sum_s a_s lambda^{m+1+s} - g^m,
  lambda^j = 0 for j > Nt, g^m = dJ/dq^m = Dt sum_r (y_r^m - d_r^m) P_r^T
  (P_r^T puts l(x_r) on the pressure nodes of element k_r).  The gradient is
      dJ/dc_k = -sum_n lambda^{n+1} . h sum_s a_s (dA/dc_k) q^{n-s},
  and with tau frozen dA/dc_k multiplies the pressure rows of element k of A by 2/c_k.

The operator A is assembled column by column from this package's own right-hand side
(``dg_rhs.rhs``) and A^T is its sparse transpose: no transposed operator is derived by hand.

Several rate levels (``misfit_gradient_levels``): the scheme is Algorithm 1 with the levels
frozen as well.  One fine step of it (right-hand sides of the active elements, Eq. updateAB for
the levels that finish, Eq. updateABcoarse traces for their coarse neighbours) is an affine map
Z' = F_tau Z + (source) of the full state Z = (fields q, stored face traces, three right-hand-side
histories); F_tau depends on tau only through tau mod 2^{L-1}.  Its matrix is assembled column
by column from ``MRAB.fine_step`` itself, and so is B_tau, the response of Z' to the pressure
right-hand side computed in the step.  Velocity enters a fine step only through the pressure rows
of that right-hand side, (A q)_p of element k scaling with c_k^2, so reverse accumulation gives
    mu_T = dJ/dZ_T,   mu_tau = F_tau^T mu_{tau+1} + dJ/dZ_tau,
    dJ/dc_k = sum_tau (2/c_k) (B_tau^T mu_{tau+1})_{p,k} . (A q_tau)_{p,k}   (k active at tau),
with dJ/dZ nonzero at the global steps only.  With one level this is the recursion above, written
over the state instead of q alone.
"""

from __future__ import annotations

import copy
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from .dg_rhs import rhs, traces
from .mesh_geometry import MeshGeometry
from .mrab import AB_A, MRAB
from .wavelet import ricker


def frozen_geometry(geo: MeshGeometry, c) -> MeshGeometry:
    """The geometry with velocity c in rho c^2; the impedance behind tau stays the reference one."""
    g = copy.copy(geo)
    g.c = np.asarray(c, dtype=np.float64)
    return g


def _distance2_colors(geo: MeshGeometry):
    """Greedy colouring in which two elements of one colour have no element in common among
    themselves and their face neighbours (their right-hand-side responses do not overlap)."""
    K = geo.K
    nb = [set(int(x) for x in geo.nbr[k] if x >= 0) for k in range(K)]
    color = -np.ones(K, dtype=np.int64)
    for k in range(K):
        near = set(nb[k])
        for j in nb[k]:
            near |= nb[j]
        used = {int(color[j]) for j in near if color[j] >= 0}
        c = 0
        while c in used:
            c += 1
        color[k] = c
    return color, nb


def assemble_operator(geo: MeshGeometry) -> sp.csr_matrix:
    """The matrix of q -> rhs(q) (all elements, no source) on unknowns ordered as q[K, 4, Np]."""
    K, Np = geo.K, geo.ref.Np
    nd = 4 * Np
    color, nb = _distance2_colors(geo)
    rows, cols, vals = [], [], []
    allk = np.arange(K)
    for col in range(int(color.max()) + 1):
        members = np.nonzero(color == col)[0]
        for i in range(nd):
            x = np.zeros((K, nd))
            x[members, i] = 1.0
            x = x.reshape(K, 4, Np)
            y = rhs(allk, x, traces(x, geo), geo).reshape(K, nd)
            for e in members:
                for r in [int(e)] + sorted(nb[e]):
                    nz = np.nonzero(y[r])[0]
                    rows.extend(r * nd + nz)
                    cols.extend([int(e) * nd + i] * len(nz))
                    vals.extend(y[r, nz])
    n = K * nd
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


@dataclass
class MisfitResult:
    misfit: float
    traces: np.ndarray
    states: list | None


def _receivers(geo, rec_xyz):
    out = []
    for x in np.atleast_2d(rec_xyz):
        k, r = geo.locate(x)
        if k < 0:
            raise ValueError("receiver outside the mesh")
        out.append((k, geo.interpolation_row(r)))
    return out


def shot_misfit(prob, c, source_xyz, f0, t_peak, amplitude, rec_xyz, t_final, observed, keep_states=False):
    """Forward run (Algorithm 1 with the problem's levels) with velocity c (frozen tau, levels and
    step) and its misfit; ``keep_states`` keeps q at the global steps."""
    geo = frozen_geometry(prob.geo, c)
    n_global = int(np.ceil(t_final / prob.dt_global - 1e-9))
    ks, rs = geo.locate(source_xyz)
    if ks < 0:
        raise ValueError("source outside the mesh")
    rec = _receivers(geo, rec_xyz)
    S = MRAB(geo, prob.levels, prob.n_levels, prob.dt_local, +1)
    S.injections = [(ks, geo.source_weights(ks, rs),
                     lambda tau: float(ricker(tau * prob.dt_local, f0, t_peak, amplitude)))]
    tr = np.zeros((len(rec), n_global + 1))
    states = [S.q.copy()] if keep_states else None
    for n in range(n_global + 1):
        if n > 0:
            S.global_step()
            if keep_states:
                states.append(S.q.copy())
        tr[:, n] = [row @ S.q[k, 0] for k, row in rec]
    J = 0.5 * prob.dt_global * float(np.sum((tr - observed) ** 2))
    return MisfitResult(J, tr, states)


def misfit_gradient(prob, c, source_xyz, f0, t_peak, amplitude, rec_xyz, t_final, observed):
    """(J, dJ/dc [K]) by the discrete adjoint above (one rate level)."""
    if prob.n_levels != 1:
        raise ValueError("misfit_gradient is the single-rate adjoint; use misfit_gradient_levels")
    fwd = shot_misfit(prob, c, source_xyz, f0, t_peak, amplitude, rec_xyz, t_final, observed, keep_states=True)
    geo = frozen_geometry(prob.geo, c)
    K, Np = geo.K, geo.ref.Np
    A = assemble_operator(geo)
    AT = A.T.tocsr()
    h = prob.dt_local
    a = [float(x) for x in AB_A]
    Nt = len(fwd.states) - 1
    rec = _receivers(geo, rec_xyz)
    res = fwd.traces - observed

    def g(m):
        out = np.zeros((K, 4, Np))
        for r, (k, row) in enumerate(rec):
            out[k, 0] += prob.dt_global * res[r, m] * row
        return out.reshape(-1)

    q = [s.reshape(-1) for s in fwd.states]
    Aq = [A @ x for x in q]
    lam = {}
    s_hist = {}
    zero = np.zeros(K * 4 * Np)
    for m in range(Nt, 0, -1):
        acc = zero.copy()
        for s in range(3):
            j = m + 1 + s
            if j <= Nt:
                if j not in s_hist:
                    s_hist[j] = AT @ lam[j]
                acc += a[s] * s_hist[j]
        lam[m] = (lam[m + 1] if m + 1 <= Nt else zero) + h * acc - g(m)
    grad = np.zeros(K)
    for n in range(Nt):
        dAq = zero.copy()
        for s in range(3):
            if n - s >= 0:
                dAq += h * a[s] * Aq[n - s]
        prod = (lam[n + 1] * dAq).reshape(K, 4, Np)[:, 0].sum(axis=1)
        grad -= (2.0 / geo.c) * prod
    return fwd.misfit, grad


# ---------------------------------------------------------------- several rate levels
def _get_state(S: MRAB) -> np.ndarray:
    return np.concatenate([S.q.ravel(), S.qf.ravel(), S.hist.ravel()])


def _set_state(S: MRAB, z: np.ndarray) -> None:
    nq, nf = S.q.size, S.qf.size
    S.q = z[:nq].reshape(S.q.shape).copy()
    S.qf = z[nq:nq + nf].reshape(S.qf.shape).copy()
    S.hist = z[nq + nf:].reshape(S.hist.shape).copy()


def _fine_step_matrices(geo, prob, tau):
    """F (state to state) and B (pressure right-hand side of the active elements to state) of the
    source-free fine step at tau, both assembled from MRAB.fine_step on unit vectors; ``cols``
    lists the (element, node) of each column of B."""
    S = MRAB(geo, prob.levels, prob.n_levels, prob.dt_local, +1)
    n = _get_state(S).size
    F = np.zeros((n, n))
    for i in range(n):
        z = np.zeros(n)
        z[i] = 1.0
        _set_state(S, z)
        S.tau = tau
        S.fine_step()
        F[:, i] = _get_state(S)
    active = S.active(tau)
    Np = geo.ref.Np
    cols = [(int(k), j) for k in active for j in range(Np)]
    B = np.zeros((n, len(cols)))
    for ci, (k, j) in enumerate(cols):
        _set_state(S, np.zeros(n))
        S.tau = tau
        w = np.zeros(Np)
        w[j] = 1.0
        S.injections = [(k, w, lambda t: 1.0)]
        S.fine_step()
        B[:, ci] = _get_state(S)
    S.injections = []
    return sp.csr_matrix(F), sp.csr_matrix(B), cols


def misfit_gradient_levels(prob, c, source_xyz, f0, t_peak, amplitude, rec_xyz, t_final, observed):
    """(J, dJ/dc [K]) for any number of rate levels, by reverse accumulation over the fine steps
    of Algorithm 1 (module docstring).  The state matrices are dense during assembly: for small
    meshes only."""
    geo = frozen_geometry(prob.geo, c)
    K, Np = geo.K, geo.ref.Np
    nl = 2 ** (prob.n_levels - 1)
    n_global = int(np.ceil(t_final / prob.dt_global - 1e-9))
    T = n_global * nl
    ks, rs = geo.locate(source_xyz)
    if ks < 0:
        raise ValueError("source outside the mesh")
    rec = _receivers(geo, rec_xyz)
    # forward run, keeping each fine step's state and the source-free pressure right-hand side
    S = MRAB(geo, prob.levels, prob.n_levels, prob.dt_local, +1)
    S.injections = [(ks, geo.source_weights(ks, rs),
                     lambda tau: float(ricker(tau * prob.dt_local, f0, t_peak, amplitude)))]
    Z, R = [], []
    tr = np.zeros((len(rec), n_global + 1))
    tr[:, 0] = [row @ S.q[k, 0] for k, row in rec]
    for tau in range(T):
        Z.append(_get_state(S))
        act = S.active(tau)
        R.append((act, rhs(act, S.q, S.qf, geo)[:, 0].copy() if len(act) else None))
        S.fine_step()
        if (tau + 1) % nl == 0:
            tr[:, (tau + 1) // nl] = [row @ S.q[k, 0] for k, row in rec]
    J = 0.5 * prob.dt_global * float(np.sum((tr - observed) ** 2))
    res = tr - observed
    n = Z[0].size

    def dJdZ(tau):
        out = np.zeros(n)
        if tau % nl == 0:
            q = out[:K * 4 * Np].reshape(K, 4, Np)
            for r, (k, row) in enumerate(rec):
                q[k, 0] += prob.dt_global * res[r, tau // nl] * row
        return out

    mats = {p: _fine_step_matrices(geo, prob, p) for p in range(nl)}
    grad = np.zeros(K)
    mu = dJdZ(T)
    for tau in range(T - 1, -1, -1):
        F, B, cols = mats[tau % nl]
        act, r = R[tau]
        if r is not None:
            v = B.T @ mu
            pos = {int(k): i for i, k in enumerate(act)}
            for ci, (k, j) in enumerate(cols):
                grad[k] += (2.0 / geo.c[k]) * v[ci] * r[pos[k], j]
        mu = F.T @ mu + dJdZ(tau)
    return J, grad
