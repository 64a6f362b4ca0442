"""Domain decomposition of the multi-rate scheme (oracle, FP64, test infrastructure).

Sec. 4.2 of the paper: each device advances one part of the mesh; at each local time step the
traces of the fields on faces between parts are transferred when necessary; the source and
receiver runs of the backward phase use the same partition, so the images need no transfer.

* Weights: an element of level l (1 = coarsest) weighs N_l = 2^(l-1), the number of its
  right-hand-side evaluations per global step, so that equal weights mean equal work.
* Lumping: every element of the finest level, or connected group of them, is lumped with its face
  neighbours before partitioning and the lump stays in one part.  No finest element then lies at an
  interface, and at the fine steps that update the finest level only nothing has to cross (the
  paper's "half of all potential" transfers).  Reading: the paper finds its finest elements
  isolated; a lump heavier than half of one part's share of the weight would spoil the balance, so
  such a lump is not kept whole (its elements are partitioned one by one), and then the steps that
  update the finest level only transfer traces like the others whenever a finest element ends up at
  an interface (every part checks this on the partition).
* Partitioner (reading): the paper uses METIS with these weights; here weighted recursive
  coordinate bisection of the lumps (their weighted centroids, split across the longest extent at
  the weighted median), which balances the same weights without the external library.
* Transfer: at the end of every fine step, each part sends the traces (p, n.v) of its elements
  whose traces changed at that step (updated by Eq. updateAB, or set to the half-step value of
  Eq. updateABcoarse) and that have a face neighbour in another part, to that part, which writes
  them into its copy of the trace array; nothing is sent at steps that update the finest level
  only.  A part evaluates right-hand sides, updates and half-steps only its own elements; which
  elements are updated or half-stepped at a step is known to every part from the levels.

``PartMRAB`` is a drop-in stepper for ``oracle.rtm.rtm_shot`` (its ``stepper`` argument): the
shot of a part accumulates the images of its own elements and samples the receivers that lie in
them; the union over the parts is the unpartitioned shot.
"""

from __future__ import annotations

import numpy as np

from .mrab import MRAB


def element_weights(levels):
    """N_l = 2^(l-1) per element (Sec. 4.2)."""
    return 2.0 ** (np.asarray(levels, dtype=np.int64) - 1)


def lump_units(levels, nbr, n_levels):
    """Unit (lump) index per element: each finest element is joined with its face neighbours
    (union-find over those pairs); every other element is its own unit unless a lump took it."""
    K = len(levels)
    parent = np.arange(K)

    def find(a):
        root = a
        while parent[root] != root:
            root = parent[root]
        while parent[a] != root:
            parent[a], a = root, parent[a]
        return root

    if n_levels >= 2:
        for k in np.nonzero(np.asarray(levels) == n_levels)[0]:
            for k2 in nbr[k]:
                if k2 >= 0:
                    ra, rb = find(int(k)), find(int(k2))
                    if ra != rb:
                        parent[max(ra, rb)] = min(ra, rb)
    roots = np.array([find(k) for k in range(K)])
    _, unit = np.unique(roots, return_inverse=True)
    return unit


def rcb(points, weights, n_parts):
    """Weighted recursive coordinate bisection: part index per point.  Each split cuts across the
    longest extent of its points at the weighted median, in proportion to the parts on each side."""
    out = np.zeros(len(points), dtype=np.int64)

    def split(idx, first, n):
        if n == 1 or len(idx) == 0:
            out[idx] = first
            return
        p = points[idx]
        axis = int(np.argmax(p.max(axis=0) - p.min(axis=0)))
        order = idx[np.lexsort((idx, p[:, axis]))]
        n_left = n // 2
        cw = np.cumsum(weights[order])
        cut = int(np.searchsorted(cw, cw[-1] * n_left / n))
        cut = min(max(cut, 1), len(order) - 1) if len(order) > 1 else len(order)
        split(order[:cut], first, n_left)
        split(order[cut:], first + n_left, n - n_left)

    split(np.arange(len(points)), 0, n_parts)
    return out


def partition(geo, levels, n_levels, n_parts):
    """Part index per element: lumps of the finest level kept whole, weights 2^(l-1), weighted
    recursive coordinate bisection of the lumps."""
    w = element_weights(levels)
    unit = lump_units(levels, geo.nbr, n_levels)
    uw = np.bincount(unit, weights=w)
    big = uw[unit] > 0.5 * w.sum() / n_parts  # lumps too heavy to keep whole
    unit = np.where(big, int(unit.max()) + 1 + np.arange(len(unit)), unit)
    _, unit = np.unique(unit, return_inverse=True)
    n_units = int(unit.max()) + 1
    uw = np.bincount(unit, weights=w, minlength=n_units)
    cen = geo.xyz[geo.tets].mean(axis=1)
    uc = np.stack([np.bincount(unit, weights=w * cen[:, d], minlength=n_units) for d in range(3)], axis=1) / uw[:, None]
    return rcb(uc, uw, n_parts)[unit]


def interface_lists(nbr, part, rank):
    """For each other part r: the elements of this part with a face neighbour in r (``send[r]``) and
    the elements of r with a face neighbour in this part (``recv[r]``), in increasing order."""
    K = len(part)
    own = part == rank
    send, recv = {}, {}
    for k in range(K):
        for k2 in nbr[k]:
            if k2 < 0 or part[k2] == part[k]:
                continue
            if own[k]:
                send.setdefault(int(part[k2]), set()).add(k)
            elif part[k2] == rank:
                recv.setdefault(int(part[k]), set()).add(k)
    return ({r: np.array(sorted(v)) for r, v in send.items()}, {r: np.array(sorted(v)) for r, v in recv.items()})


class PartMRAB(MRAB):
    """Algorithm 1 for the elements of one part (``part == rank``), with the trace transfer above.

    ``comm.exchange(sends, recv_shapes)`` moves arrays between parts: ``sends`` maps a part to the
    array sent to it, ``recv_shapes`` a part to the shape of the array it sends here; it returns the
    received arrays.  Every part calls it at the same points of the same program."""

    def __init__(self, geo, levels, n_levels, dt_local, direction=1, tau0=0, *, part, rank, comm):
        super().__init__(geo, levels, n_levels, dt_local, direction, tau0)
        self.part = np.asarray(part)
        self.rank = int(rank)
        self.comm = comm
        self.owned = self.part == self.rank
        self.level_elems = {l: E[self.owned[E]] for l, E in self.level_elems.items()}
        self.boundary_faces = [(k, f) for k, f in self.boundary_faces if self.owned[k]]
        self.send, self.recv = interface_lists(geo.nbr, self.part, self.rank)
        # finest elements all inside their parts (lumping held): finest-only steps transfer nothing
        fin = np.nonzero(self.lev == self.n_levels)[0]
        nb = geo.nbr[fin]
        self.finest_inside = self.n_levels >= 2 and bool(
            np.all((nb < 0) | (self.part[np.maximum(nb, 0)] == self.part[fin][:, None])))
        self.messages = 0  # arrays sent (a count for tests)
        self.silent_steps = 0  # fine steps that needed no transfer

    def active(self, tau):
        A = super().active(tau)
        return A[self.owned[A]]

    def _exchange(self, changed):
        sends = {r: self.qf[E[changed[E]]] for r, E in self.send.items()}
        rsel = {r: E[changed[E]] for r, E in self.recv.items()}
        shapes = {r: (len(E),) + self.qf.shape[1:] for r, E in rsel.items()}
        sends = {r: a for r, a in sends.items() if len(a)}
        shapes = {r: s for r, s in shapes.items() if s[0]}
        got = self.comm.exchange(sends, shapes)
        self.messages += len(sends)
        for r, arr in got.items():
            self.qf[rsel[r]] = arr

    def set_state(self, q):
        super().set_state(q)
        # the fields of other parts' elements are not this part's to know: take their traces
        everything = np.ones(self.geo.K, dtype=bool)
        self._exchange(everything)

    def phase_halfstep(self, updated_mask):
        upd = np.isin(self.lev, self.levels_to_update())  # every part knows who is updated
        H = self.halfstep_elements(upd)
        Ho = H[self.owned[H]]
        self.apply_halfstep(Ho)
        if self.finest_inside and self.levels_to_update() == [self.n_levels]:
            self.silent_steps += 1  # finest level only: lumping keeps every changed trace inside
            return Ho
        changed = upd.copy()
        changed[H] = True
        self._exchange(changed)
        return Ho
