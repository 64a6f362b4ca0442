"""One reverse-time-migration shot (oracle, FP64, test infrastructure).

Sec. 2 and Sec. 4.3 of the paper:

1. Forward source run from rest with the point source f(t) (Eq. waveSyst1), receiver
   pressures sampled at every global step, and the traces (p, n.v) of every domain-boundary
   face recorded at every evaluation time of its element.
2. The run continues two global steps past t_f so that, for each level l, the
   right-hand sides at t_f + Delta t_l and t_f + 2 Delta t_l exist; together with q(t_f)
   they start the backward Adams-Bashforth run of the source wavefield (reading of
   "the final solution saved").
3. Backward in time (Delta t_l < 0, tau < 0): the source wavefield re-simulated from
   q(t_f) with the source re-injected and, on boundary faces, the forward boundary flux
   rebuilt from the recorded traces (forward boundary condition and tau); the receiver
   wavefield from rest with every receiver re-injecting its (observed) trace.  Both run in
   lockstep over [t_i, t_f] and, right before each update, the AB3-exact increments of the
   classical (Eq. imageP) and characteristic (Eq. imageQ) images are accumulated.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .dg_rhs import attach_media, rhs, traces
from .imaging import characteristic, step_increment
from .mesh_geometry import MeshGeometry
from .mrab import MRAB, assign_levels
from .reference_element import reference_element
from .wavelet import interpolate_trace, ricker, sampled


@dataclass
class Problem:
    geo: MeshGeometry
    N: int
    levels: np.ndarray
    n_levels: int
    dt_local: float

    @property
    def n_local(self):
        return 2 ** (self.n_levels - 1)

    @property
    def dt_global(self):
        return self.dt_local * self.n_local


def make_problem(xyz, tets, c, rho, N, face_bc=None, default_bc=2, cfl=0.15, n_levels_max=3,
                 tau_scale=1.0) -> Problem:
    ref = reference_element(N)
    geo = attach_media(MeshGeometry(xyz, tets, ref, face_bc=face_bc, default_bc=default_bc), c, rho, tau_scale)
    lev, nl, dtl = assign_levels(geo, N, c, cfl, n_levels_max)
    return Problem(geo, N, lev, nl, dtl)


def full_rhs(prob: Problem, q, sign=1.0):
    geo = prob.geo
    return rhs(np.arange(geo.K), q, traces(q, geo), geo, sign=sign)


@dataclass
class ShotResult:
    traces: np.ndarray
    image_p: np.ndarray
    image_q: np.ndarray
    q_final: np.ndarray
    q_source_back: np.ndarray  # source wavefield reconstructed at t_i by the backward run
    q_source_fwd_ti: np.ndarray  # forward source wavefield at t_i
    dof_updates: int
    n_global: int


def _source_signal(f0, t_peak, amplitude, dtl, wavelet=None, wavelet_dt=None):
    """Source amplitude at integer fine time tau: the Ricker pulse, or the sampled signal."""
    if wavelet is None:
        return lambda tau: float(ricker(tau * dtl, f0, t_peak, amplitude))
    samples = np.asarray(wavelet, dtype=np.float64).reshape(-1)
    return lambda tau: sampled(tau * dtl, samples, wavelet_dt, amplitude)


def _receivers(geo, rec_xyz):
    rec = []
    for x in np.atleast_2d(rec_xyz):
        if x.size == 0:
            continue
        kr, rr = geo.locate(x)
        if kr < 0:
            raise ValueError("receiver outside the mesh")
        rec.append((kr, geo.interpolation_row(rr), geo.source_weights(kr, rr)))
    return rec


def forward(prob: Problem, source_xyz, f0, t_peak, amplitude, rec_xyz, t_final, wavelet=None,
            wavelet_dt=None) -> np.ndarray:
    """Forward modelling alone (Eq. waveSyst1 from a medium at rest): the receiver traces
    [nrec, n_global + 1] sampled at every global step t_n = n Delta t_global."""
    geo = prob.geo
    n_global = int(np.ceil(t_final / prob.dt_global - 1e-9))
    ks, rs = geo.locate(source_xyz)
    if ks < 0:
        raise ValueError("source outside the mesh")
    rec = _receivers(geo, rec_xyz)
    S = MRAB(geo, prob.levels, prob.n_levels, prob.dt_local, direction=+1, tau0=0)
    S.injections = [(ks, geo.source_weights(ks, rs),
                     _source_signal(f0, t_peak, amplitude, prob.dt_local, wavelet, wavelet_dt))]
    tr = np.zeros((len(rec), n_global + 1))
    for n in range(n_global + 1):
        if n > 0:
            S.global_step()
        tr[:, n] = [row @ S.q[k, 0] for k, row, _ in rec]
    return tr


def rtm_shot(prob: Problem, source_xyz, f0, t_peak, amplitude, rec_xyz, t_final, t_image_start=0.0,
             observed=None, e_up=(0.0, 0.0, -1.0), wavelet=None, wavelet_dt=None, observe=None,
             stepper=MRAB) -> ShotResult:
    """``observe`` (tests only): called as observe(tau, q_S, q_R) with the backward source and
    receiver fields at t = tau Delta t_local, once at tau_f and after every fine step of the
    backward sweep down to tau_i; it lets a test integrate the imaging conditions on its own.
    ``stepper``: the class that advances each wavefield (Algorithm 1); ``oracle.partition`` gives one
    that advances a single part of a partitioned mesh and exchanges interface traces (Sec. 4.2)."""
    geo = prob.geo
    K, Np = geo.K, geo.ref.Np
    nl = prob.n_local
    dtl = prob.dt_local
    n_global = int(np.ceil(t_final / prob.dt_global - 1e-9))
    n_i = int(np.floor(t_image_start / prob.dt_global + 1e-9))
    tau_f, tau_i = n_global * nl, n_i * nl
    ks, rs = geo.locate(source_xyz)
    if ks < 0:
        raise ValueError("source outside the mesh")
    w_src = geo.source_weights(ks, rs)
    rec = _receivers(geo, rec_xyz)
    src_amp = _source_signal(f0, t_peak, amplitude, dtl, wavelet, wavelet_dt)

    def sample(q):
        return np.array([row @ q[k, 0] for k, row, _ in rec])

    # ---------------------------------------------------------------- forward
    S = stepper(geo, prob.levels, prob.n_levels, dtl, direction=+1, tau0=0)
    S.injections = [(ks, w_src, src_amp)]
    S.record = {}
    tr = np.zeros((len(rec), n_global + 1))
    tr[:, 0] = sample(S.q)
    q_ti = S.q.copy() if tau_i == 0 else None
    for n in range(n_global):
        S.global_step()
        tr[:, n + 1] = sample(S.q)
        if S.tau == tau_i:
            q_ti = S.q.copy()
    q_tf = S.q.copy()
    record = S.record
    saved = {}
    stride = S.stride
    for _ in range(2 * nl):
        tau = S.tau
        S.fine_step()
        for l in stride:
            if tau == tau_f + 2 * stride[l]:
                E = S.level_elems[l]
                saved[l] = (S.hist[1][E].copy(), S.hist[0][E].copy())
    # the coarsest level evaluates its right-hand side at t_f + 2 Delta t_global
    S.record = None
    S.phase_rhs()
    E = S.level_elems[1]
    saved[1] = (S.hist[1][E].copy(), S.hist[0][E].copy())

    # ---------------------------------------------------------------- backward
    Sb = stepper(geo, prob.levels, prob.n_levels, dtl, direction=-1, tau0=tau_f)
    Sb.set_state(q_tf)
    for l, (r1, r2) in saved.items():
        E = Sb.level_elems[l]
        Sb.hist[0][E] = r1
        Sb.hist[1][E] = r2
    Sb.injections = [(ks, w_src, src_amp)]
    Sb.replay = record
    data = tr if observed is None else np.asarray(observed, dtype=np.float64)
    R = stepper(geo, prob.levels, prob.n_levels, dtl, direction=-1, tau0=tau_f)
    R.injections = [(kr, wr, (lambda tau, d=data[i]: interpolate_trace(d, tau, nl))) for i, (kr, _, wr) in enumerate(rec)]
    I_p = np.zeros((K, Np))
    I_q = np.zeros((K, Np))
    Z = geo.Z

    def image(l):
        E = Sb.level_elems[l]
        if len(E) == 0:
            return
        h = Sb.h[l]
        xS, xR = Sb.q[E, 0], R.q[E, 0]
        rS = [Sb.hist[s][E, 0] for s in range(3)]
        rR = [R.hist[s][E, 0] for s in range(3)]
        I_p[E] -= step_increment(h, xS, rS, xR, rR)
        ZE = Z[E]
        qS = characteristic(Sb.q[E, 0], Sb.q[E, 1:4], ZE, e_up, -1.0)
        qR = characteristic(R.q[E, 0], R.q[E, 1:4], ZE, e_up, +1.0)
        rqS = [characteristic(Sb.hist[s][E, 0], Sb.hist[s][E, 1:4], ZE, e_up, -1.0) for s in range(3)]
        rqR = [characteristic(R.hist[s][E, 0], R.hist[s][E, 1:4], ZE, e_up, +1.0) for s in range(3)]
        I_q[E] -= step_increment(h, qS, rqS, qR, rqR)

    if observe is not None:
        observe(Sb.tau, Sb.q.copy(), R.q.copy())
    while Sb.tau > tau_i:
        Sb.phase_rhs()
        R.phase_rhs()
        updated = np.zeros(K, dtype=bool)
        for l in Sb.levels_to_update():
            image(l)
            E = Sb.phase_update(l)
            R.phase_update(l)
            updated[E] = True
        Sb.phase_halfstep(updated)
        R.phase_halfstep(updated)
        Sb.tau -= 1
        R.tau -= 1
        if observe is not None:
            observe(Sb.tau, Sb.q.copy(), R.q.copy())
    return ShotResult(tr, I_p, I_q, q_tf, Sb.q.copy(), q_ti, S.dof_updates + Sb.dof_updates + R.dof_updates, n_global)
