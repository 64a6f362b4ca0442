"""ctypes binding of the C ABI in ``include/ridg.h`` (argument marshalling only).

Every computation runs in ``libridg.so``: the mesh setup on the host, everything in the time loop
in CUDA kernels.  Host arrays are numpy float64/int64 arrays; device buffers may be given as
torch CUDA tensors (their ``data_ptr()`` is passed through).  There is no fallback: if the
library is missing or was built for another machine, importing this module raises.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libridg.so")

RIDG_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "BAD_MESH", -3: "OOM", -4: "CUDA", -5: "UNSTABLE", -6: "TIMEOUT", -7: "NOT_FOUND",
          -8: "BUSY"}
BC_AUTO, BC_FREE, BC_TRANSPARENT, BC_RIGID = 0, 1, 2, 3
F32, F64 = 0, 1

EXPORTED = [
    "ridg_last_error", "ridg_version", "ridg_mesh_create", "ridg_mesh_destroy", "ridg_mesh_counts",
    "ridg_reference_operators", "ridg_solver_create", "ridg_solver_destroy", "ridg_solver_info",
    "ridg_solver_levels", "ridg_solver_nodes", "ridg_set_state", "ridg_set_history", "ridg_eval_rhs", "ridg_step",
    "ridg_rtm_shots", "ridg_rtm_shots_device", "ridg_server_set_batch", "ridg_set_graph_replay",
    "ridg_get_state", "ridg_energy", "ridg_trace_len", "ridg_rtm_shot", "ridg_rtm_shot_device",
    "ridg_last_shot_stats", "ridg_set_profiling", "ridg_energy_noalloc", "ridg_server_create", "ridg_server_create_slots", "ridg_server_submit",
    "ridg_server_wait", "ridg_server_destroy", "ridg_forward", "ridg_set_state_device", "ridg_get_state_device",
    "ridg_set_velocity", "ridg_eval_adjoint_rhs", "ridg_misfit_forward", "ridg_misfit_backward", "ridg_mesh_locate",
    "ridg_partition", "ridg_group_create", "ridg_group_rtm_shot", "ridg_group_info_get", "ridg_group_trace_len",
    "ridg_group_destroy", "ridg_inject_fault", "ridg_fault_armed", "ridg_set_trace_budget",
]
MAX_PARTS = 64


class RidgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ridg error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


class Options(C.Structure):
    _fields_ = [("dtype", C.c_int32), ("cfl", C.c_double), ("n_levels_max", C.c_int32), ("image_mask", C.c_int32),
                ("tau_scale", C.c_double), ("contraction", C.c_int32), ("reserved", C.c_int32 * 3)]


IMAGE_P, IMAGE_Q = 1, 2
CONTRACT_TENSOR, CONTRACT_CUDA_CORES, CONTRACT_TENSOR_BF16, CONTRACT_TENSOR_FP16, CONTRACT_TENSOR_TF32 = 0, 1, 2, 3, 4
SRC_RICKER, SRC_SAMPLED = 0, 1


class Info(C.Structure):
    _fields_ = [("N", C.c_int32), ("Np", C.c_int32), ("Nfp", C.c_int32), ("n_levels", C.c_int32), ("K", C.c_int64),
                ("dt_local", C.c_double), ("dt_global", C.c_double), ("level_count", C.c_int64 * 8),
                ("n_boundary_faces", C.c_int64), ("device_bytes", C.c_int64), ("n_half_step", C.c_int64)]


class Source(C.Structure):
    _fields_ = [("xyz", C.c_double * 3), ("f0", C.c_double), ("t_peak", C.c_double), ("amplitude", C.c_double),
                ("kind", C.c_int32), ("reserved", C.c_int32), ("sample_dt", C.c_double), ("n_samples", C.c_int64),
                ("samples", C.c_void_p)]


def _source(source_xyz, f0, t_peak, amplitude, wavelet=None, wavelet_dt=None):
    """Source struct and the array it points to (kept alive by the caller): a Ricker pulse, or with
    ``wavelet`` (samples at t = n * wavelet_dt) a sampled wavelet scaled by ``amplitude``."""
    if wavelet is None:
        return Source((C.c_double * 3)(*source_xyz), f0, t_peak, amplitude, SRC_RICKER, 0, 0.0, 0, None), None
    w = _f64(wavelet).reshape(-1)
    return Source((C.c_double * 3)(*source_xyz), 0.0, 0.0, amplitude, SRC_SAMPLED, 0, float(wavelet_dt), w.size,
                  _ptr(w)), w


class ShotIO(C.Structure):
    _fields_ = [("source", Source), ("rec_xyz", C.c_void_p), ("nrec", C.c_int64), ("observed", C.c_void_p),
                ("traces_out", C.c_void_p), ("image_p", C.c_void_p), ("image_q", C.c_void_p)]


MAX_BATCH = 4  # RIDG_MAX_BATCH: shots of one lockstep batch


class ShotStats(C.Structure):
    _fields_ = [("dof_updates_forward", C.c_int64), ("dof_updates_backward", C.c_int64),
                ("fused_launches", C.c_int64), ("kernel_launches", C.c_int64), ("n_global", C.c_int64),
                ("boundary_trace_bytes", C.c_int64), ("prof_forward_ms", C.c_double),
                ("prof_backward_ms", C.c_double), ("prof_forward_launches", C.c_int64),
                ("prof_backward_launches", C.c_int64), ("trace_chunks", C.c_int64),
                ("host_trace_bytes", C.c_int64), ("graph_replay", C.c_int64)]


class ShotRequest(C.Structure):
    _fields_ = [("source", Source), ("rec_xyz", C.c_void_p), ("nrec", C.c_int64), ("t_final", C.c_double),
                ("t_image_start", C.c_double), ("observed", C.c_void_p), ("traces_out", C.c_void_p),
                ("image_p", C.c_void_p), ("image_q", C.c_void_p), ("e_up", C.c_void_p), ("model", C.c_int32),
                ("reserved", C.c_int32)]


class GroupInfo(C.Structure):
    _fields_ = [("n_parts", C.c_int32), ("reserved", C.c_int32), ("elements", C.c_int64 * 64),
                ("ghosts", C.c_int64 * 64), ("interface_faces", C.c_int64 * 64), ("dof_updates", C.c_int64),
                ("transfer_steps", C.c_int64), ("silent_steps", C.c_int64), ("transfer_bytes", C.c_int64)]


class RequestTiming(C.Structure):
    _fields_ = [("queued_s", C.c_double), ("run_s", C.c_double), ("total_s", C.c_double), ("start_s", C.c_double),
                ("end_s", C.c_double), ("slot", C.c_int64)]


def load_library(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_1506_00907_gb300.build.build()")
    lib = C.CDLL(path)
    P = C.c_void_p
    sig = {
        "ridg_last_error": (C.c_char_p, []),
        "ridg_version": (C.c_char_p, []),
        "ridg_mesh_create": (C.c_int, [P, C.c_int64, P, C.c_int64, P, C.c_int8, C.POINTER(P)]),
        "ridg_mesh_destroy": (None, [P]),
        "ridg_mesh_counts": (C.c_int, [P, P, P]),
        "ridg_reference_operators": (C.c_int, [C.c_int, P, P, P, P, P]),
        "ridg_solver_create": (C.c_int, [P, C.c_int, P, P, P, C.c_size_t, C.POINTER(P)]),
        "ridg_solver_destroy": (None, [P]),
        "ridg_solver_info": (C.c_int, [P, P]),
        "ridg_solver_levels": (C.c_int, [P, P]),
        "ridg_solver_nodes": (C.c_int, [P, P]),
        "ridg_set_state": (C.c_int, [P, P]),
        "ridg_set_history": (C.c_int, [P, P, P]),
        "ridg_eval_rhs": (C.c_int, [P, P, P]),
        "ridg_step": (C.c_int, [P, C.c_int64]),
        "ridg_get_state": (C.c_int, [P, P]),
        "ridg_energy": (C.c_int, [P, P]),
        "ridg_trace_len": (C.c_int64, [P, C.c_double]),
        "ridg_rtm_shot": (C.c_int, [P, P, P, C.c_int64, C.c_double, C.c_double, P, P, P, P, P]),
        "ridg_rtm_shot_device": (C.c_int, [P, P, P, C.c_int64, C.c_double, C.c_double, P, P, P, P, P]),
        "ridg_rtm_shots": (C.c_int, [P, C.c_int32, P, C.c_double, C.c_double, P]),
        "ridg_rtm_shots_device": (C.c_int, [P, C.c_int32, P, C.c_double, C.c_double, P]),
        "ridg_last_shot_stats": (C.c_int, [P, P]),
        "ridg_set_profiling": (C.c_int, [P, C.c_int32]),
        "ridg_set_graph_replay": (C.c_int, [P, C.c_int32]),
        "ridg_set_trace_budget": (C.c_int, [P, C.c_int64]),
        "ridg_energy_noalloc": (C.c_int, [P, P]),
        "ridg_forward": (C.c_int, [P, P, P, C.c_int64, C.c_double, P]),
        "ridg_set_state_device": (C.c_int, [P, P]),
        "ridg_get_state_device": (C.c_int, [P, P]),
        "ridg_set_velocity": (C.c_int, [P, P]),
        "ridg_mesh_locate": (C.c_int, [P, P, C.c_int64, P, P]),
        "ridg_eval_adjoint_rhs": (C.c_int, [P, P, P]),
        "ridg_misfit_forward": (C.c_int, [P, P, P, C.c_int64, C.c_double, P, C.c_int32, P, P]),
        "ridg_misfit_backward": (C.c_int, [P, P]),
        "ridg_server_create": (C.c_int, [P, C.c_int64, C.POINTER(P)]),
        "ridg_server_create_slots": (C.c_int, [P, P, C.c_int64, C.c_int64, C.POINTER(P)]),
        "ridg_server_submit": (C.c_int, [P, P, C.POINTER(C.c_int64)]),
        "ridg_server_wait": (C.c_int, [P, C.c_int64, C.c_double, P]),
        "ridg_server_destroy": (C.c_int, [P]),
        "ridg_server_set_batch": (C.c_int, [P, C.c_int32]),
        "ridg_partition": (C.c_int, [P, C.c_int, P, P, C.c_int32, P]),
        "ridg_group_create": (C.c_int, [P, C.c_int, P, P, P, P, C.c_int32, P, C.POINTER(P)]),
        "ridg_group_rtm_shot": (C.c_int, [P, P, P, C.c_int64, C.c_double, C.c_double, P, P, P, P, P]),
        "ridg_group_info_get": (C.c_int, [P, P]),
        "ridg_group_trace_len": (C.c_int64, [P, C.c_double, P]),
        "ridg_group_destroy": (None, [P]),
        "ridg_inject_fault": (C.c_int, [C.c_char_p, C.c_int64]),
        "ridg_fault_armed": (C.c_int, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


def _check(code):
    if code != RIDG_OK:
        raise RidgError(code, lib().ridg_last_error().decode())


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()  # torch tensor


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != tuple(shape):
        a = a.reshape(shape)
    return a


def reference_operators(N: int):
    Np = (N + 1) * (N + 2) * (N + 3) // 6
    Nfp = (N + 1) * (N + 2) // 2
    rst = np.zeros((Np, 3))
    D = np.zeros((3, Np, Np))
    M = np.zeros((Np, Np))
    LIFT = np.zeros((Np, 4 * Nfp))
    fm = np.zeros((4, Nfp), dtype=np.int32)
    _check(lib().ridg_reference_operators(N, _ptr(rst), _ptr(D), _ptr(M), _ptr(LIFT), _ptr(fm)))
    return dict(rst=rst, D=D, M=M, LIFT=LIFT, fmask=fm)


class Mesh:
    def __init__(self, xyz, tets, face_bc=None, default_bc=BC_TRANSPARENT):
        self.xyz = _f64(xyz)
        self.tets = np.ascontiguousarray(tets, dtype=np.int64)
        fb = None if face_bc is None else np.ascontiguousarray(face_bc, dtype=np.int8)
        h = C.c_void_p()
        _check(lib().ridg_mesh_create(_ptr(self.xyz), self.xyz.shape[0], _ptr(self.tets), self.tets.shape[0],
                                      _ptr(fb), int(default_bc), C.byref(h)))
        self._h = h
        self.K = self.tets.shape[0]

    def counts(self):
        nb, ni = C.c_int64(), C.c_int64()
        _check(lib().ridg_mesh_counts(self._h, C.byref(nb), C.byref(ni)))
        return nb.value, ni.value

    def locate(self, xyz):
        """(element [n], reference coordinates [n, 3]) of the points xyz [n, 3]; element -1 outside."""
        x = _f64(np.atleast_2d(xyz))
        elem = np.zeros(x.shape[0], dtype=np.int64)
        rst = np.zeros((x.shape[0], 3))
        _check(lib().ridg_mesh_locate(self._h, _ptr(x), x.shape[0], _ptr(elem), _ptr(rst)))
        return elem, rst

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.ridg_mesh_destroy(self._h)
            self._h = None


class Solver:
    def __init__(self, mesh: Mesh, N: int, c, rho, dtype="f32", cfl=0.15, n_levels_max=3, stream=0, tau_scale=1.0,
                 image_mask=IMAGE_P | IMAGE_Q, contraction=CONTRACT_TENSOR):
        self.mesh = mesh
        c = _f64(c)
        rho = _f64(rho)
        opt = Options(F64 if dtype == "f64" else F32, float(cfl), int(n_levels_max), int(image_mask),
                      float(tau_scale), int(contraction))
        h = C.c_void_p()
        _check(lib().ridg_solver_create(mesh._h, int(N), _ptr(c), _ptr(rho), C.byref(opt), int(stream), C.byref(h)))
        self._h = h
        self.info = self.get_info()
        self.N, self.Np, self.K = self.info.N, self.info.Np, self.info.K

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.ridg_solver_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def get_info(self) -> Info:
        inf = Info()
        _check(lib().ridg_solver_info(self._h, C.byref(inf)))
        return inf

    def levels(self):
        out = np.zeros(self.K, dtype=np.int32)
        _check(lib().ridg_solver_levels(self._h, _ptr(out)))
        return out

    def nodes(self):
        out = np.zeros((self.K, self.Np, 3))
        _check(lib().ridg_solver_nodes(self._h, _ptr(out)))
        return out

    def set_state(self, q):
        q = _f64(q, (self.K, 4, self.Np))
        _check(lib().ridg_set_state(self._h, _ptr(q)))

    def set_history(self, r1=None, r2=None):
        a = None if r1 is None else _f64(r1, (self.K, 4, self.Np))
        b = None if r2 is None else _f64(r2, (self.K, 4, self.Np))
        _check(lib().ridg_set_history(self._h, _ptr(a), _ptr(b)))

    def eval_rhs(self, q):
        q = _f64(q, (self.K, 4, self.Np))
        out = np.zeros_like(q)
        _check(lib().ridg_eval_rhs(self._h, _ptr(q), _ptr(out)))
        return out

    def step(self, n_global=1):
        _check(lib().ridg_step(self._h, int(n_global)))

    def get_state(self):
        out = np.zeros((self.K, 4, self.Np))
        _check(lib().ridg_get_state(self._h, _ptr(out)))
        return out

    def energy(self):
        e = C.c_double()
        _check(lib().ridg_energy(self._h, C.byref(e)))
        return e.value

    def energy_noalloc(self, out):
        """Energy into a caller-owned device buffer (torch CUDA float64 tensor with >= 1 element),
        without any device allocation; asynchronous on the solver's stream."""
        _check(lib().ridg_energy_noalloc(self._h, _ptr(out)))

    def trace_len(self, t_final):
        return int(lib().ridg_trace_len(self._h, float(t_final)))

    def set_state_device(self, q):
        """Fields from a torch CUDA float64 tensor [K, 4, Np] (asynchronous on the solver's stream)."""
        _check(lib().ridg_set_state_device(self._h, _ptr(q)))

    def get_state_device(self, q):
        """Fields into a torch CUDA float64 tensor [K, 4, Np] (asynchronous on the solver's stream)."""
        _check(lib().ridg_get_state_device(self._h, _ptr(q)))

    def set_velocity(self, c):
        """Velocity per element in rho c^2 (time step, level and penalty parameters stay frozen)."""
        c = _f64(c, (self.K,))
        _check(lib().ridg_set_velocity(self._h, _ptr(c)))

    def eval_adjoint_rhs(self, lam):
        """A^T lam for the transposed right-hand-side operator ([K, 4, Np] host arrays)."""
        lam = _f64(lam, (self.K, 4, self.Np))
        out = np.zeros_like(lam)
        _check(lib().ridg_eval_adjoint_rhs(self._h, _ptr(lam), _ptr(out)))
        return out

    def misfit_forward(self, source_xyz, f0, t_peak, amplitude, rec_xyz, t_final, observed, n_checkpoints=16,
                       wavelet=None, wavelet_dt=None):
        """(J, traces) of a forward run against observed traces [nrec, n_t]; keeps checkpoints for
        ``misfit_backward`` (any number of rate levels)."""
        src, _keep = _source(source_xyz, f0, t_peak, amplitude, wavelet, wavelet_dt)
        rec = _f64(np.atleast_2d(rec_xyz))
        n_t = self.trace_len(t_final)
        obs = _f64(observed, (rec.shape[0], n_t))
        traces = np.zeros((rec.shape[0], n_t))
        J = C.c_double()
        _check(lib().ridg_misfit_forward(self._h, C.byref(src), _ptr(rec), rec.shape[0], float(t_final), _ptr(obs),
                                         int(n_checkpoints), C.byref(J), _ptr(traces)))
        return J.value, traces

    def misfit_backward(self):
        """dJ/dc [K] of the last ``misfit_forward`` (discrete adjoint, checkpointed recomputation)."""
        g = np.zeros(self.K)
        _check(lib().ridg_misfit_backward(self._h, _ptr(g)))
        return g

    def forward(self, source_xyz, f0, t_peak, amplitude, rec_xyz, t_final, wavelet=None, wavelet_dt=None):
        """Forward modelling: receiver traces [nrec, n_t] of the forward run alone."""
        src, _keep = _source(source_xyz, f0, t_peak, amplitude, wavelet, wavelet_dt)
        rec = _f64(np.atleast_2d(rec_xyz)) if len(rec_xyz) else np.zeros((0, 3))
        traces = np.zeros((rec.shape[0], self.trace_len(t_final)))
        _check(lib().ridg_forward(self._h, C.byref(src), _ptr(rec), rec.shape[0], float(t_final), _ptr(traces)))
        return traces

    def rtm_shot(self, source_xyz, f0, t_peak, amplitude, rec_xyz, t_final, t_image_start=0.0, observed=None,
                 e_up=(0.0, 0.0, -1.0), want_images=True, wavelet=None, wavelet_dt=None):
        """Host-buffer shot: returns (traces [nrec, n_t], image_p [K, Np], image_q [K, Np])."""
        src, _keep = _source(source_xyz, f0, t_peak, amplitude, wavelet, wavelet_dt)
        rec = _f64(np.atleast_2d(rec_xyz)) if len(rec_xyz) else np.zeros((0, 3))
        n_t = self.trace_len(t_final)
        traces = np.zeros((rec.shape[0], n_t))
        ip = np.zeros((self.K, self.Np)) if want_images else None
        iq = np.zeros((self.K, self.Np)) if want_images else None
        obs = None if observed is None else _f64(observed, (rec.shape[0], n_t))
        eu = _f64(e_up)
        _check(lib().ridg_rtm_shot(self._h, C.byref(src), _ptr(rec), rec.shape[0], float(t_final),
                                   float(t_image_start), _ptr(obs), _ptr(traces), _ptr(ip), _ptr(iq), _ptr(eu)))
        return traces, ip, iq

    def rtm_shot_device(self, source_xyz, f0, t_peak, amplitude, rec_xyz, t_final, t_image_start=0.0,
                        observed=None, traces=None, image_p=None, image_q=None, e_up=(0.0, 0.0, -1.0),
                        wavelet=None, wavelet_dt=None):
        """Device-buffer shot (torch CUDA float64 tensors or None); returns after enqueueing."""
        src, _keep = _source(source_xyz, f0, t_peak, amplitude, wavelet, wavelet_dt)
        rec = _f64(np.atleast_2d(rec_xyz)) if len(rec_xyz) else np.zeros((0, 3))
        eu = _f64(e_up)
        _check(lib().ridg_rtm_shot_device(self._h, C.byref(src), _ptr(rec), rec.shape[0], float(t_final),
                                          float(t_image_start), _ptr(observed), _ptr(traces), _ptr(image_p),
                                          _ptr(image_q), _ptr(eu)))

    def _shot_ios(self, shots, host, t_final, want_images=True):
        """ShotIO array (and the arrays it points to) of a lockstep batch; host: numpy outputs."""
        n = len(shots)
        ios = (ShotIO * max(n, 1))()  # the library rejects n outside 1 .. MAX_BATCH
        keep, outs = [], []
        n_t = self.trace_len(t_final)
        for i, sh in enumerate(shots):
            src, w = _source(sh["source_xyz"], sh.get("f0", 10.0), sh.get("t_peak", 0.0), sh.get("amplitude", 1.0),
                             sh.get("wavelet"), sh.get("wavelet_dt"))
            rx = sh.get("rec_xyz", ())
            rec = _f64(np.atleast_2d(rx)) if len(rx) else np.zeros((0, 3))
            keep += [w, rec]
            if host:
                obs = None if sh.get("observed") is None else _f64(sh["observed"], (rec.shape[0], n_t))
                tr = np.zeros((rec.shape[0], n_t))
                ip = np.zeros((self.K, self.Np)) if want_images else None
                iq = np.zeros((self.K, self.Np)) if want_images else None
                keep.append(obs)
                outs.append((tr, ip, iq))
            else:
                obs, tr, ip, iq = sh.get("observed"), sh.get("traces"), sh.get("image_p"), sh.get("image_q")
            ios[i] = ShotIO(src, _ptr(rec), rec.shape[0], _ptr(obs), _ptr(tr), _ptr(ip), _ptr(iq))
        return ios, keep, outs

    def rtm_shots(self, shots, t_final, t_image_start=0.0, e_up=(0.0, 0.0, -1.0), want_images=True):
        """Several shots of this model in lockstep, one merged launch per fine step (ridg_rtm_shots).
        ``shots``: dicts with the arguments of rtm_shot (source_xyz, f0, t_peak, amplitude, rec_xyz,
        observed, wavelet, wavelet_dt); returns [(traces, image_p, image_q)] in their order."""
        ios, _keep, outs = self._shot_ios(shots, True, t_final, want_images)
        eu = _f64(e_up)
        _check(lib().ridg_rtm_shots(self._h, len(shots), ios, float(t_final), float(t_image_start), _ptr(eu)))
        return outs

    def rtm_shots_device(self, shots, t_final, t_image_start=0.0, e_up=(0.0, 0.0, -1.0)):
        """Device-buffer batch (ridg_rtm_shots_device): each dict may hold torch CUDA float64 tensors
        observed, traces, image_p, image_q; returns after enqueueing."""
        ios, _keep, _ = self._shot_ios(shots, False, t_final)
        eu = _f64(e_up)
        _check(lib().ridg_rtm_shots_device(self._h, len(shots), ios, float(t_final), float(t_image_start), _ptr(eu)))

    def set_profiling(self, every: int):
        _check(lib().ridg_set_profiling(self._h, int(every)))

    def set_graph_replay(self, on: bool = True):
        """Repeated shots with the same launch arguments run their time stepping as one CUDA-graph launch
        (ridg_set_graph_replay)."""
        _check(lib().ridg_set_graph_replay(self._h, 1 if on else 0))

    def set_trace_budget(self, device_bytes: int):
        """Device bytes for a shot's boundary-trace records; beyond them the records live in pinned
        host memory (ridg_set_trace_budget).  0: all on the device."""
        _check(lib().ridg_set_trace_budget(self._h, int(device_bytes)))

    def shot_stats(self) -> ShotStats:
        st = ShotStats()
        _check(lib().ridg_last_shot_stats(self._h, C.byref(st)))
        return st


def inject_fault(point: str, after: int = 0):
    """Arms a host-side failure point ("alloc", "arena", "admission", "exchange"; "none" disarms) that
    fires once after `after` passes (ridg_inject_fault)."""
    _check(lib().ridg_inject_fault(point.encode(), int(after)))


def fault_armed() -> int:
    return int(lib().ridg_fault_armed())


def partition(mesh: Mesh, N: int, c, n_parts: int, cfl=0.15, n_levels_max=3):
    """Part of each element (int32 [K]) for n_parts parts: weights 2^(l-1), finest-level lumping,
    weighted recursive coordinate bisection (ridg_partition; host only)."""
    c = _f64(c)
    opt = Options(F32, float(cfl), int(n_levels_max), IMAGE_P | IMAGE_Q, 1.0, CONTRACT_TENSOR)
    out = np.zeros(mesh.K, dtype=np.int32)
    _check(lib().ridg_partition(mesh._h, int(N), _ptr(c), C.byref(opt), int(n_parts), _ptr(out)))
    return out


class Group:
    """One shot over a partitioned mesh, one solver per part (ridg_group_*); part i on CUDA device
    devices[i] (default: all on the current device)."""

    def __init__(self, mesh: Mesh, N: int, c, rho, part, dtype="f32", cfl=0.15, n_levels_max=3, devices=None,
                 tau_scale=1.0, image_mask=IMAGE_P | IMAGE_Q, contraction=CONTRACT_TENSOR):
        self.mesh = mesh
        c, rho = _f64(c), _f64(rho)
        self.part = np.ascontiguousarray(part, dtype=np.int32)
        self.n_parts = int(self.part.max()) + 1 if self.part.size else 0
        dev = None if devices is None else np.ascontiguousarray(devices, dtype=np.int32)
        opt = Options(F64 if dtype == "f64" else F32, float(cfl), int(n_levels_max), int(image_mask),
                      float(tau_scale), int(contraction))
        h = C.c_void_p()
        _check(lib().ridg_group_create(mesh._h, int(N), _ptr(c), _ptr(rho), C.byref(opt), _ptr(self.part),
                                       self.n_parts, _ptr(dev), C.byref(h)))
        self._h = h
        self.K = mesh.K

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.ridg_group_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def trace_len(self, t_final):
        return int(lib().ridg_group_trace_len(self._h, float(t_final), None))

    def info(self) -> GroupInfo:
        out = GroupInfo()
        _check(lib().ridg_group_info_get(self._h, C.byref(out)))
        return out

    def rtm_shot(self, source_xyz, f0, t_peak, amplitude, rec_xyz, t_final, t_image_start=0.0, observed=None,
                 e_up=(0.0, 0.0, -1.0), wavelet=None, wavelet_dt=None):
        """Host-buffer shot over all parts: (traces [nrec, n_t], image_p [K, Np], image_q [K, Np])."""
        src, _keep = _source(source_xyz, f0, t_peak, amplitude, wavelet, wavelet_dt)
        rec = _f64(np.atleast_2d(rec_xyz)) if len(rec_xyz) else np.zeros((0, 3))
        np_ = C.c_int32()
        n_t = int(lib().ridg_group_trace_len(self._h, float(t_final), C.byref(np_)))
        traces = np.zeros((rec.shape[0], n_t))
        ip = np.zeros((self.K, np_.value))
        iq = np.zeros((self.K, np_.value))
        obs = None if observed is None else _f64(observed, (rec.shape[0], n_t))
        eu = _f64(e_up)
        _check(lib().ridg_group_rtm_shot(self._h, C.byref(src), _ptr(rec), rec.shape[0], float(t_final),
                                         float(t_image_start), _ptr(obs), _ptr(traces), _ptr(ip), _ptr(iq), _ptr(eu)))
        return traces, ip, iq


class Server:
    """Shot server (``ridg_server_*``) over one solver or several slots.  ``solvers`` is a Solver or a
    list of them; ``models[i]`` is the model number of ``solvers[i]`` (default: all 0).  An idle slot
    takes the oldest waiting request of its model, so shots on different slots run concurrently
    (give those solvers different CUDA streams).  With ``max_batch`` > 1 a slot starts up to that many
    waiting requests of its model with the same time span together, as one lockstep batch (one merged
    launch per fine step).  The solvers must not be used directly while the server exists."""

    def __init__(self, solvers, max_queued: int = 8, models=None, max_batch: int = 1):
        solvers = list(solvers) if isinstance(solvers, (list, tuple)) else [solvers]
        models = [0] * len(solvers) if models is None else [int(m) for m in models]
        if len(models) != len(solvers):
            raise ValueError("one model number per solver")
        self.solvers = solvers
        self.models = models
        hs = (C.c_void_p * len(solvers))(*[s._h.value for s in solvers])
        ms = (C.c_int32 * len(models))(*models)
        h = C.c_void_p()
        _check(lib().ridg_server_create_slots(hs, ms, len(solvers), int(max_queued), C.byref(h)))
        self._h = h
        self._pending = {}
        if max_batch != 1:
            self.set_batch(max_batch)

    def set_batch(self, max_batch: int):
        _check(lib().ridg_server_set_batch(self._h, int(max_batch)))

    @property
    def solver(self):
        return self.solvers[0]

    def _model_solver(self, model):
        for s, m in zip(self.solvers, self.models):
            if m == model:
                return s
        raise ValueError(f"no slot serves model {model}")

    def submit(self, source_xyz, f0, t_peak, amplitude, rec_xyz, t_final, t_image_start=0.0, observed=None,
               e_up=(0.0, 0.0, -1.0), want_images=True, wavelet=None, wavelet_dt=None, model=0) -> int:
        """Queues a shot for ``model``; its host output buffers are kept here until ``wait`` returns them."""
        ms = self._model_solver(model)
        rec = _f64(np.atleast_2d(rec_xyz)) if len(rec_xyz) else np.zeros((0, 3))
        n_t = ms.trace_len(t_final)
        traces = np.zeros((rec.shape[0], n_t))
        ip = np.zeros((ms.K, ms.Np)) if want_images else None
        iq = np.zeros((ms.K, ms.Np)) if want_images else None
        obs = None if observed is None else _f64(observed, (rec.shape[0], n_t))
        eu = _f64(e_up)
        src, _keep = _source(source_xyz, f0, t_peak, amplitude, wavelet, wavelet_dt)
        req = ShotRequest(src, _ptr(rec), rec.shape[0], float(t_final), float(t_image_start), _ptr(obs),
                          _ptr(traces), _ptr(ip), _ptr(iq), _ptr(eu), int(model), 0)
        t = C.c_int64()
        _check(lib().ridg_server_submit(self._h, C.byref(req), C.byref(t)))
        self._pending[t.value] = (traces, ip, iq)
        return t.value

    def wait(self, ticket: int, timeout=None):
        """(traces, image_p, image_q, timing) of a completed request; RidgError (TIMEOUT) if it has not
        completed within ``timeout`` seconds (None: no limit), or the request's own error."""
        tm = RequestTiming()
        code = lib().ridg_server_wait(self._h, int(ticket), -1.0 if timeout is None else float(timeout), C.byref(tm))
        if code == -6:
            _check(code)
        out = self._pending.pop(ticket, None)
        _check(code)
        traces, ip, iq = out
        return traces, ip, iq, {"queued_s": tm.queued_s, "run_s": tm.run_s, "total_s": tm.total_s,
                                "start_s": tm.start_s, "end_s": tm.end_s, "slot": tm.slot}

    def close(self):
        if self._h:
            _check(lib().ridg_server_destroy(self._h))
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def misfit(c, solver: Solver, source_xyz, f0, t_peak, amplitude, rec_xyz, t_final, observed, n_checkpoints=16):
    """Least-squares trace misfit as a differentiable function of the per-element velocity ``c``
    (a torch float64 tensor [K]): forward run in ``forward``, gradient by the library's adjoint
    kernels with checkpointed recomputation in ``backward``."""
    import torch

    class _Misfit(torch.autograd.Function):
        @staticmethod
        def forward(ctx, cv):
            solver.set_velocity(cv.detach().cpu().numpy())
            J, _ = solver.misfit_forward(source_xyz, f0, t_peak, amplitude, rec_xyz, t_final, observed, n_checkpoints)
            ctx.device = cv.device
            return torch.tensor(J, dtype=torch.float64, device=cv.device)

        @staticmethod
        def backward(ctx, gJ):
            g = torch.from_numpy(solver.misfit_backward()).to(ctx.device)
            return gJ * g

    return _Misfit.apply(c)
