"""Semi-discrete right-hand side of the nodal DG scheme (oracle, FP64, test infrastructure).

Eqs. dgLocalSchemeP / dgLocalSchemeU (Sec. 3.1) with the penalty terms of the weak
form, Eqs. weakFormP / weakFormV:

    dp/dt   = -rho c^2 div v - sum_f (J_f/J) L_f P^p_f
    dv_i/dt = -(1/rho) d p / d x_i - sum_f (J_f/J) L_f P^{v_i}_f
    P^p     = rho c^2 * 1/2 ( n.[v] - tau_p [p] )
    P^{v_i} = (n_i / rho) * 1/2 ( [p] - tau_v n.[v] )

with [u] = u^+ - u^- (exterior minus interior) and n the outward unit normal of the
element.  Readings (where the paper is silent or differs from itself):

* The factor 1/2 of the weak form is kept (the appendix drops it); only with 1/2 do
  the central parts of the interface terms cancel in the energy balance.
* tau_p = 1/Zbar, tau_v = Zbar with Zbar = (rho^- c^- + rho^+ c^+)/2 on interior faces
  (the upwind values of Sec. 3.1 when the medium is homogeneous), Zbar = rho c on
  boundary faces; tau is multiplied by -1 in backward-in-time runs (Sec. 3.2).  A
  penalty scale s (``geo.tau_scale``, 1 by default) multiplies both: s = 1 is the upwind
  flux of Sec. 3.1, s = 0 the central flux, and every face's energy loss is linear in s.
* Boundary conditions through an exterior ("ghost") state: free surface p^+ = -p^-,
  n.v^+ = n.v^-; transparent (Eq. ABC) p^+ = 0, v^+ = 0; rigid wall p^+ = p^-,
  n.v^+ = -n.v^-.  Only p and n.v enter the fluxes, so traces (p, n.v) suffice, as in
  the paper's qf array.
* The point source follows Eq. waveSyst1: dp/dt += f(t) w with w the L2-projected Dirac.

The surface term reads its traces from a trace array ``qf[K, 2, 4, Nfp]`` holding p and
n.v (with the owner's outward normal) on each face node, as the paper's qf does.
"""

from __future__ import annotations

import numpy as np

from .mesh_geometry import BC_FREE, BC_INTERIOR, BC_RIGID, BC_TRANSPARENT, MeshGeometry


def traces_of(q: np.ndarray, normal: np.ndarray, Fmask: np.ndarray) -> np.ndarray:
    """Traces (p, n.v) on the face nodes of each element of ``q`` [E, 4, Np]: [E, 2, 4, Nfp].
    ``normal`` [E, 4, 3] holds the outward unit normals of those elements."""
    E = q.shape[0]
    qf = np.zeros((E, 2, 4, Fmask.shape[1]))
    for f in range(4):
        qf[:, 0, f] = q[:, 0, Fmask[f]]
        qf[:, 1, f] = np.einsum("kd,kdn->kn", normal[:, f], q[:, 1:4, Fmask[f]])
    return qf


def traces(q: np.ndarray, geo: MeshGeometry) -> np.ndarray:
    return traces_of(q, geo.normal, geo.ref.Fmask)


def face_jumps(elems, qf, geo: MeshGeometry, sign=1.0, replay=None):
    """Jumps ([p], n.[v]) and penalty parameters on every face node of ``elems``.

    Returns jp, jv [E, 4, Nfp] and tau_p, tau_v [E, 4].  ``replay`` (optional) maps
    (element, face) -> traces (p, n.v) [2, Nfp] recorded on that boundary face by the
    forward run at the same time; such faces take the recorded traces as their exterior
    state (in place of the boundary condition's ghost state) with this run's tau.
    """
    elems = np.asarray(elems)
    E = len(elems)
    Nfp = geo.ref.Nfp
    pm = qf[elems, 0]  # [E, 4, Nfp]
    vm = qf[elems, 1]
    Z = geo.Z
    sign = sign * geo.tau_scale
    jp = np.zeros((E, 4, Nfp))
    jv = np.zeros((E, 4, Nfp))
    taup = np.zeros((E, 4))
    tauv = np.zeros((E, 4))
    for f in range(4):
        nb = geo.nbr[elems, f]
        bc = geo.bc[elems, f]
        inter = bc == BC_INTERIOR
        # interior faces: neighbour traces, its n.v taken with the opposite normal
        if np.any(inter):
            ei = np.nonzero(inter)[0]
            k2 = nb[ei]
            f2 = geo.nbr_face[elems[ei], f]
            j2 = geo.nbr_node[elems[ei], f]  # [Ei, Nfp]
            pp = qf[k2[:, None], 0, f2[:, None], j2]
            vp = -qf[k2[:, None], 1, f2[:, None], j2]
            jp[ei, f] = pp - pm[ei, f]
            jv[ei, f] = vp - vm[ei, f]
            Zb = 0.5 * (Z[elems[ei]] + Z[k2])
            taup[ei, f] = sign / Zb
            tauv[ei, f] = sign * Zb
        for code in (BC_FREE, BC_TRANSPARENT, BC_RIGID):
            sel = np.nonzero(bc == code)[0]
            if len(sel) == 0:
                continue
            p_in, v_in = pm[sel, f], vm[sel, f]
            if code == BC_FREE:
                jp[sel, f], jv[sel, f] = -2.0 * p_in, 0.0
            elif code == BC_TRANSPARENT:
                jp[sel, f], jv[sel, f] = -p_in, -v_in
            else:
                jp[sel, f], jv[sel, f] = 0.0, -2.0 * v_in
            if replay is not None:
                # backward source run: the exterior state is the recorded forward trace
                for a, e in enumerate(sel):
                    rec = replay.get((int(elems[e]), f))
                    if rec is not None:
                        jp[sel[a], f] = rec[0] - p_in[a]
                        jv[sel[a], f] = rec[1] - v_in[a]
            Zk = Z[elems[sel]]
            taup[sel, f] = sign / Zk
            tauv[sel, f] = sign * Zk
    return jp, jv, taup, tauv


def rhs(elems, q, qf, geo: MeshGeometry, sign=1.0, replay=None):
    """Right-hand side [E, 4, Np] for the elements ``elems`` (Eqs. dgLocalSchemeP/U)."""
    ref = geo.ref
    elems = np.asarray(elems)
    qe = q[elems]
    p, v = qe[:, 0], qe[:, 1:4]
    rho = geo.rho[elems]
    rc2 = rho * geo.c[elems] ** 2
    rx = geo.rx[elems]  # [E, i, j] = d r_j / d x_i
    # reference derivatives D_j applied to p and to each v_i
    Dp = np.einsum("jnm,em->ejn", ref.D, p)  # [E, j, Np]
    Dv = np.einsum("jnm,eim->eijn", ref.D, v)  # [E, i, j, Np]
    grad_p = np.einsum("eij,ejn->ein", rx, Dp)  # d p / d x_i
    div_v = np.einsum("eij,eijn->en", rx, Dv)
    out = np.zeros_like(qe)
    out[:, 0] = -rc2[:, None] * div_v
    out[:, 1:4] = -grad_p / rho[:, None, None]
    # surface term
    jp, jv, taup, tauv = face_jumps(elems, qf, geo, sign, replay)
    Pp = rc2[:, None, None] * 0.5 * (jv - taup[:, :, None] * jp)  # [E, 4, Nfp]
    Pv = (0.5 * (jp - tauv[:, :, None] * jv)) / rho[:, None, None]  # times n_i
    n = geo.normal[elems]  # [E, 4, 3]
    Fs = geo.Fscale[elems]  # [E, 4]
    Nfp = ref.Nfp
    for f in range(4):
        Lf = ref.LIFT[:, f * Nfp:(f + 1) * Nfp]
        out[:, 0] -= Fs[:, f, None] * (Pp[:, f] @ Lf.T)
        for i in range(3):
            out[:, 1 + i] -= Fs[:, f, None] * ((n[:, f, i, None] * Pv[:, f]) @ Lf.T)
    return out


def energy(q, geo: MeshGeometry) -> float:
    """Discrete energy sum_k J_k/2 (p^T M p / (rho c^2) + rho v^T M v)."""
    M = geo.ref.M
    p, v = q[:, 0], q[:, 1:4]
    ep = np.einsum("kn,nm,km->k", p, M, p) / (geo.rho * geo.c ** 2)
    ev = geo.rho * np.einsum("kin,nm,kim->k", v, M, v)
    return float(np.sum(0.5 * geo.J * (ep + ev)))


def attach_media(geo: MeshGeometry, c, rho, tau_scale=1.0):
    geo.c = np.asarray(c, dtype=np.float64)
    geo.rho = np.asarray(rho, dtype=np.float64)
    geo.Z = geo.rho * geo.c
    geo.tau_scale = float(tau_scale)
    return geo
