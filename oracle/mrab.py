"""Multi-rate Adams-Bashforth time stepping (oracle, FP64, test infrastructure).

Sec. 3.2 of the paper and Algorithm 1 ("Forward time-stepping procedure"):

* Levels: Delta t_l = 2^(Nlev - l) Delta t_local, level 1 the coarsest; each element
  gets the coarsest level its local bound Delta t_k = C l_k/((N+1)^2 c_k) allows, then
  elements are moved to finer levels until neighbours differ by at most one level.
  Reading of the level rule (the paper gives it in words only):
  L_k = floor(log2(Delta t_k / Delta t_local) (1 + 1e-12)), Nlev = min(Nlev_max, 1 + max L_k),
  level_k = Nlev - min(L_k, Nlev - 1), then repeat lev_a = max(lev_a, lev_b - 1) over
  neighbours until nothing changes.
* Eq. updateAB: q^{new} = q + Delta t_l sum_s a_s r^{m-s}, a = (23/12, -16/12, 5/12).
* Eq. updateABcoarse (coefficients read b_s; the paper prints b_f): traces of a coarse
  element at the midpoint of its step, b = (17/24, -7/24, 2/24), for the fine neighbours.
* Algorithm 1, per step of the finest level: right-hand sides of every element whose
  unknowns sit at t_start; then levels Nlev..1 are updated if they must be evaluated at
  t_new; then the traces of every element not updated at this step but coarse neighbour
  of an updated element are set with the half-step formula.
* Backward in time: the same formulas with Delta t_l < 0 and tau < 0 (Sec. 3.2).

Time is counted in integer units of Delta t_local (``tau``); t = tau * Delta t_local.
"""

from __future__ import annotations

from fractions import Fraction

import numpy as np

from .dg_rhs import rhs, traces_of
from .imaging import A_POLY
from .mesh_geometry import BC_INTERIOR, MeshGeometry


def _eval_at(poly, x: Fraction) -> Fraction:
    return sum((c * x ** i for i, c in enumerate(poly)), Fraction(0))


# Eq. updateAB / Eq. updateABcoarse: a_s = A_s(1), b_s = A_s(1/2), with A_s the integral
# from 0 of the Lagrange polynomial on the nodes 0, -1, -2 (see oracle.imaging).
AB_A = tuple(_eval_at(A, Fraction(1)) for A in A_POLY)
AB_B = tuple(_eval_at(A, Fraction(1, 2)) for A in A_POLY)


def assign_levels(geo: MeshGeometry, N: int, c, cfl: float, n_levels_max: int):
    """Levels (1 = coarsest) per element, the number of levels and Delta t_local."""
    dtk = geo.dt_bound(N, c, cfl)
    dt_local = float(dtk.min())
    L = np.floor(np.log2(dtk / dt_local) * (1.0 + 1e-12)).astype(np.int64)
    n_levels = int(min(n_levels_max, 1 + L.max()))
    lev = n_levels - np.minimum(L, n_levels - 1)
    inter = geo.nbr >= 0
    while True:
        nb_lev = np.where(inter, lev[np.maximum(geo.nbr, 0)], 0)
        new = np.maximum(lev, nb_lev.max(axis=1) - 1)
        if np.array_equal(new, lev):
            break
        lev = new
    return lev, n_levels, dt_local


class MRAB:
    """State and Algorithm 1 for one wavefield.

    ``injections``: list of (element, weights[Np], amplitude(tau) -> float) added to the
    pressure right-hand side at each evaluation time (Eq. sourceTerm).
    ``replay``: optional dict tau -> {(element, face): traces[2, Nfp]} (backward source run).
    ``record``: optional dict filled with tau -> {(element, face): traces[2, Nfp]} for every
    boundary face of every element whose right-hand side is evaluated at tau.
    """

    def __init__(self, geo: MeshGeometry, levels, n_levels, dt_local, direction=1, tau0=0):
        self.geo = geo
        self.lev = np.asarray(levels, dtype=np.int64)
        self.n_levels = int(n_levels)
        self.dt_local = float(dt_local)
        self.sign = 1 if direction > 0 else -1
        self.n_local = 2 ** (self.n_levels - 1)
        self.stride = {l: 2 ** (self.n_levels - l) for l in range(1, self.n_levels + 1)}
        self.h = {l: self.sign * self.stride[l] * self.dt_local for l in self.stride}
        K, Np = geo.K, geo.ref.Np
        self.q = np.zeros((K, 4, Np))
        self.qf = traces_of(self.q, geo.normal, geo.ref.Fmask)
        self.hist = np.zeros((3, K, 4, Np))
        self.tau = int(tau0)
        self.injections = []
        self.replay = None
        self.record = None
        self.level_elems = {l: np.nonzero(self.lev == l)[0] for l in self.stride}
        self.boundary_faces = [(k, f) for k, f in zip(*np.nonzero(geo.bc != BC_INTERIOR))]
        self.dof_updates = 0
        self.a = tuple(float(x) for x in AB_A)
        self.b = tuple(float(x) for x in AB_B)

    # ------------------------------------------------------------------ state
    def set_state(self, q):
        self.q = np.array(q, dtype=np.float64)
        self.qf = traces_of(self.q, self.geo.normal, self.geo.ref.Fmask)

    def set_history(self, r_prev1, r_prev2):
        """History before the first step: r at one and two level steps back (per element)."""
        self.hist[0] = r_prev1
        self.hist[1] = r_prev2

    def time(self, tau=None):
        return (self.tau if tau is None else tau) * self.dt_local

    # ------------------------------------------------------------------ phases of one fine step
    def active(self, tau):
        return np.nonzero(np.array([tau % self.stride[l] == 0 for l in range(1, self.n_levels + 1)])[self.lev - 1])[0]

    def phase_rhs(self):
        """Right-hand sides of all elements whose unknowns sit at t_start (Algorithm 1)."""
        tau = self.tau
        A = self.active(tau)
        if len(A) == 0:
            self._A = A
            return A
        rep = None if self.replay is None else self.replay.get(tau, {})
        r = rhs(A, self.q, self.qf, self.geo, sign=float(self.sign), replay=rep)
        pos = {int(k): i for i, k in enumerate(A)}
        for elem, w, amp in self.injections:
            if elem in pos:
                r[pos[elem], 0] += amp(tau) * w
        self.hist[2][A] = self.hist[1][A]
        self.hist[1][A] = self.hist[0][A]
        self.hist[0][A] = r
        if self.record is not None:
            act = set(int(k) for k in A)
            rec = {}
            for k, f in self.boundary_faces:
                if int(k) in act:
                    rec[(int(k), int(f))] = self.qf[k, :, f].copy()
            self.record[tau] = rec
        self._A = A
        return A

    def levels_to_update(self):
        tn = self.tau + self.sign
        return [l for l in range(self.n_levels, 0, -1) if tn % self.stride[l] == 0]

    def phase_update(self, l):
        """Eq. updateAB for every element of level l."""
        E = self.level_elems[l]
        if len(E) == 0:
            return E
        h = self.h[l]
        a = self.a
        self.q[E] = self.q[E] + h * (a[0] * self.hist[0][E] + a[1] * self.hist[1][E] + a[2] * self.hist[2][E])
        self.qf[E] = traces_of(self.q[E], self.geo.normal[E], self.geo.ref.Fmask)
        self.dof_updates += len(E) * 4 * self.geo.ref.Np
        return E

    def halfstep_elements(self, updated_mask):
        """Elements not updated at this step that are coarse neighbours of updated elements."""
        geo = self.geo
        inter = geo.nbr >= 0
        nb = np.maximum(geo.nbr, 0)
        coarse_nbr = np.any(inter & updated_mask[nb] & (self.lev[nb] > self.lev[:, None]), axis=1)
        return np.nonzero(coarse_nbr & ~updated_mask)[0]

    def phase_halfstep(self, updated_mask):
        """Eq. updateABcoarse for elements not updated at this step that are coarse
        neighbours of updated elements."""
        return self.apply_halfstep(self.halfstep_elements(updated_mask))

    def apply_halfstep(self, H):
        """Traces of the elements H set to their fields at the middle of their own step."""
        geo = self.geo
        if len(H) == 0:
            return H
        b = self.b
        hl = np.array([self.h[int(l)] for l in self.lev[H]])[:, None, None]
        qh = self.q[H] + hl * (b[0] * self.hist[0][H] + b[1] * self.hist[1][H] + b[2] * self.hist[2][H])
        self.qf[H] = traces_of(qh, geo.normal[H], geo.ref.Fmask)
        return H

    def fine_step(self, before_update=None):
        self.phase_rhs()
        updated = np.zeros(self.geo.K, dtype=bool)
        for l in self.levels_to_update():
            if before_update is not None:
                before_update(l)
            E = self.phase_update(l)
            updated[E] = True
        self.phase_halfstep(updated)
        self.tau += self.sign

    def global_step(self, before_update=None):
        for _ in range(self.n_local):
            self.fine_step(before_update)
