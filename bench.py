"""Benchmark: RTM shots of the layered 2 km x 2 km x 1 km model on GB300.

Workload (one "step" = one complete RTM shot): ~1.9e5 tetrahedra, N = 4, FP32, three multi-rate
levels, 10 Hz Ricker source at (1000, 1000, 8) m, 201 receivers, 1.5 s record, transparent
boundaries; forward source run with boundary-trace recording, then the backward source and
receiver runs in lockstep with both images (FP64 accumulation).  Metric: DOF updates per second
(elements updated x 4 fields x Np per local step, both wavefields counted in the backward phase).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ridg|reference]

Prints one JSON line.  With --gpus N > 1 (launched by torch.distributed.run) each rank migrates
its own shot (shots are independent: weak scaling) and the images are summed over ranks.
"""

from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "DOF-updates/s & RTM shots/s at stated error vs FP64; p50/p99 shot latency"
UNIT = "DOF-updates/s"
FALLBACK_HBM_GBS = 6800.0


def _workload():
    from synth import config2_layered_rtm

    return config2_layered_rtm()


def _config(w, extra=None):
    cfg = {
        "workload": "layered 2x2x1 km RTM shot: 190608 tets, N=4, FP32, 3 LTS levels, 201 receivers, 1.5 s record",
        "elements": int(w.K),
        "order": w.N,
        "record_s": w.t_final,
        "receivers": int(len(w.receivers)),
        "l2_policy": "inputs larger than L2 (fields+history+traces of two wavefields are ~GBs)",
    }
    if extra:
        cfg.update(extra)
    return cfg


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = os.path.join("/tmp", f"ridg_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def _rejected(clocks):
    bad = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}
    if any(r in bad for r in clocks.get("reasons", [])):
        return True
    sm, smax = clocks.get("sm_mhz"), clocks.get("sm_max_mhz")
    if sm and smax and sm < 0.6 * smax and not clocks.get("reasons"):
        return True
    return False


# --------------------------------------------------------------------------- roofline helpers
def step_bytes_per_element(Np, Nfp, W, real_bytes=4):
    """Algorithmic bytes one element moves in one fused step with W wavefields.

    Per wavefield: q read + write (8 Np), two older right-hand sides read and the new one written
    (12 Np), the face inbox read and the traces pushed to the neighbours (2 x 8 Nfp), injection
    range (8 B).  Per element: the FP32 coefficient table (56 floats: geometric factors, impedance,
    normals and penalty coefficients in 16-byte groups), connectivity and flags (4 neighbour slots +
    4 face bytes + boundary index + flags = 28 B); with W = 2 the two FP64 images are read and
    written (32 Np B)."""
    per_wave = (20 * Np + 16 * Nfp) * real_bytes + 8
    per_elem = 56 * 4 + 28
    img = 32 * Np if W == 2 else 0
    return W * per_wave + per_elem + img


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def _traffic():
    path = os.path.join(ROOT, "profiles", "dg_step_traffic.json")
    try:
        d = json.load(open(path))
        return d
    except (OSError, ValueError):
        return None


# --------------------------------------------------------------------------- CPU oracle leg
ORACLE_BYTES_PER_PROCESS = 3.5e9  # peak resident memory of one oracle instance of the bench mesh (measured 3.1 GB)


def _oracle_replica(root, warm, timed, barrier, queue):
    """One oracle instance (FP64 numpy, one thread): builds the bench problem, waits at the barrier so
    that every replica steps at the same time, then runs warm + timed global MRAB steps of the forward
    source run; reports (DOF updates of the timed steps, wall start and end of the timed steps)."""
    sys.path.insert(0, root)
    from oracle.mrab import MRAB
    from oracle.rtm import make_problem
    from oracle.wavelet import ricker
    from synth import config2_layered_rtm

    w = config2_layered_rtm()
    prob = make_problem(w.xyz, w.tets, w.c, w.rho, w.N, default_bc=w.default_bc, cfl=w.cfl,
                        n_levels_max=w.n_levels_max)
    g = prob.geo
    ks, rs = g.locate(w.source_xyz)
    S = MRAB(g, prob.levels, prob.n_levels, prob.dt_local, +1)
    S.injections = [(ks, g.source_weights(ks, rs), lambda tau: float(ricker(tau * prob.dt_local, w.f0, w.t_peak)))]
    barrier.wait(timeout=1200)
    for _ in range(warm):
        S.global_step()
    d0 = S.dof_updates
    t0 = time.time()
    for _ in range(timed):
        S.global_step()
    queue.put((S.dof_updates - d0, t0, time.time()))


def _replica_count():
    """Host cores, bounded so that the replicas take at most half of the available memory."""
    n = os.cpu_count() or 1
    try:
        avail = [int(l.split()[1]) * 1024 for l in open("/proc/meminfo") if l.startswith("MemAvailable:")][0]
        n = min(n, max(1, int(0.5 * avail // ORACLE_BYTES_PER_PROCESS)))
    except (OSError, IndexError, ValueError):
        n = 1
    return max(1, n)


def run_oracle_replicas(n_proc, warm, timed, timeout=3600):
    """n_proc independent oracle instances (spawned processes, one thread each: independent shots, the
    data-parallel form of the method) stepping at the same time.  Returns (DOF updates of the timed
    steps over all replicas, seconds from the first start to the last end of the timed steps)."""
    import multiprocessing as mp

    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    ctx = mp.get_context("spawn")
    barrier, queue = ctx.Barrier(n_proc), ctx.Queue()
    procs = [ctx.Process(target=_oracle_replica, args=(ROOT, warm, timed, barrier, queue)) for _ in range(n_proc)]
    for p in procs:
        p.start()
    try:
        res = [queue.get(timeout=timeout) for _ in range(n_proc)]
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    dof = sum(r[0] for r in res)
    return dof, max(r[2] for r in res) - min(r[1] for r in res)


def cpu_baseline_line():
    """The oracle on the host cores, after the GPU work: one global MRAB step of the bench mesh on one
    thread, then one step in each of P replicas stepping together (P = host cores, memory allowing)."""
    dof1, sec1 = run_oracle_replicas(1, 0, 1)
    n = _replica_count()
    dofn, secn = run_oracle_replicas(n, 0, 1) if n > 1 else (dof1, sec1)
    return {"value": dofn / secn, "unit": UNIT, "cores": n, "kind": "oracle",
            "one_thread": {"value": dof1 / sec1, "cores": 1, "seconds": sec1},
            "sample": f"1 global MRAB step (4 steps of the finest level, source on) of the same 190608-tet N=4 mesh "
                      f"in the FP64 numpy oracle: {n} independent single-threaded instances stepping together "
                      f"({dofn} DOF updates in {secn:.2f} s; value = all of them / wall time) and one instance alone "
                      f"({dof1} in {sec1:.2f} s)"}


# --------------------------------------------------------------------------- reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = _workload()
    n = _replica_count()
    dof, sec = run_oracle_replicas(n, args.warmup, args.steps)
    value = dof / sec
    sample = (f"{n} independent oracle instances (FP64 numpy, one thread each) stepping together: {args.steps} global "
              f"MRAB steps each after {args.warmup} warm-up steps")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(w, {"reference_step": "one global MRAB step of the forward source run per instance"}),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": n, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _poisson_stream(ridg, sv, w, src_x, rate, n_req, t_rec, seed=5):
    """Submits n_req short shots at Poisson arrival times of the given rate (sources along a line);
    returns (latencies, span from the first arrival to the last completion)."""
    gaps = np.random.default_rng(seed).exponential(1.0 / rate, n_req)
    t0 = time.perf_counter()
    arrive, tickets = 0.0, []
    for i in range(n_req):
        arrive += gaps[i]
        time.sleep(max(0.0, arrive - (time.perf_counter() - t0)))
        xs = (src_x[0] + 25.0 * (i % 5 - 2), src_x[1], src_x[2])
        tickets.append(sv.submit(xs, w.f0, w.t_peak, 1.0, w.receivers, t_rec))
    lat = [sv.wait(t)[3]["total_s"] for t in tickets]
    return lat, time.perf_counter() - t0 - gaps[0]


def _serving(ridg, torch, mesh, w, src_x):
    """Shot serving on the bench model: short shots through the shot server with one slot and with
    two slots (two solvers of the model on their own streams, whose shots overlap on the device),
    Poisson arrivals (seed 5) at 0.8x and 1.5x the measured sequential single-shot rate; p50/p99
    latency (submission to completion, host copies included) and shots/s."""
    n_req, t_rec = 16, 0.05
    streams = [torch.cuda.Stream() for _ in range(2)]
    slots = [ridg.Solver(mesh, w.N, w.c, w.rho, dtype="f32", cfl=w.cfl, n_levels_max=w.n_levels_max,
                         stream=st.cuda_stream) for st in streams]
    out = {"requests": n_req, "record_s": t_rec,
           "arrivals": "Poisson (seed 5) at 0.8x and 1.5x the sequential single-shot rate, sources along a line"}
    with ridg.Server(slots[:1], max_queued=n_req) as sv:
        sv.wait(sv.submit(src_x, w.f0, w.t_peak, 1.0, w.receivers, t_rec))  # buffers and arena in place
        t0 = time.perf_counter()
        for t in [sv.submit(src_x, w.f0, w.t_peak, 1.0, w.receivers, t_rec) for _ in range(3)]:
            sv.wait(t)
        service = (time.perf_counter() - t0) / 3
    out["sequential_service_s"] = service
    out["sequential_shots_per_s"] = 1.0 / service
    with ridg.Server(slots, max_queued=n_req) as sv:
        for t in [sv.submit(src_x, w.f0, w.t_peak, 1.0, w.receivers, t_rec) for _ in range(2)]:
            sv.wait(t)  # both slots' buffers in place
    for factor in (0.8, 1.5):
        for n_slots in (1, 2):
            with ridg.Server(slots[:n_slots], max_queued=n_req) as sv:
                lat, span = _poisson_stream(ridg, sv, w, src_x, factor / service, n_req, t_rec)
            out[f"rate{factor}x_slots{n_slots}"] = {
                "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "shots_per_s": n_req / span}
    base = out["rate0.8x_slots1"]
    out.update({"p50_s": base["p50_s"], "p99_s": base["p99_s"], "shots_per_s": base["shots_per_s"],
                "overload_two_slots_vs_sequential": out["rate1.5x_slots2"]["shots_per_s"] * service})
    for sl in slots:
        sl.close()
    return out


# --------------------------------------------------------------------------- GPU arm
def run_ridg(args):
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1506_00907_gb300 import ridg

    w = _workload()
    dev = torch.device("cuda", local)
    torch.cuda.synchronize()
    mesh = ridg.Mesh(w.xyz, w.tets, default_bc=w.default_bc)
    s = ridg.Solver(mesh, w.N, w.c, w.rho, dtype="f32", cfl=w.cfl, n_levels_max=w.n_levels_max,
                    stream=torch.cuda.current_stream(dev).cuda_stream)
    info = s.info
    nrec = len(w.receivers)
    n_t = s.trace_len(w.t_final)
    src_x = tuple(float(v) for v in w.source_xyz)
    # shots differ per rank by a lateral source shift (independent shots of a survey line)
    src_x = (src_x[0] + 50.0 * rank, src_x[1], src_x[2])
    traces = torch.zeros((nrec, n_t), dtype=torch.float64, device=dev)
    observed = torch.zeros_like(traces)
    img_p = torch.zeros((w.K, info.Np), dtype=torch.float64, device=dev)
    img_q = torch.zeros_like(img_p)

    from paper_1506_00907_gb300.shots import reduce_images

    def shot(obs):
        s.rtm_shot_device(src_x, w.f0, w.t_peak, 1.0, w.receivers, w.t_final, w.t_image_start, observed=obs,
                          traces=traces, image_p=img_p, image_q=img_q)
        if dist is not None:
            reduce_images([img_p, img_q])

    # warm-up: the first shot models the data that later shots migrate
    s.set_profiling(16)
    for i in range(args.warmup):
        shot(None if i == 0 else observed)
        if i == 0:
            torch.cuda.synchronize()
            observed.copy_(traces)
    torch.cuda.synchronize()

    def timed_region():
        clock = ClockSampler(local)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        clock.start()
        st = torch.cuda.current_stream(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        wall0 = time.perf_counter()
        e0.record(st)
        launches = 0
        for _ in range(args.steps):
            shot(observed)
            launches += s.shot_stats().kernel_launches
        e1.record(st)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        if dist is not None:
            dist.barrier()
        clocks = clock.stop()
        return e0.elapsed_time(e1) / 1e3, wall, launches, clocks

    sec, wall, launches, clocks = timed_region()
    redo = _rejected(clocks)
    if dist is not None:  # every rank takes the same decision (the timed region holds a barrier)
        flag = torch.tensor([1.0 if redo else 0.0], dtype=torch.float64, device=dev)
        dist.all_reduce(flag, op=dist.ReduceOp.MAX)
        redo = bool(flag.item() > 0)
    if redo:
        sec, wall, launches, clocks = timed_region()
    stats = s.shot_stats()
    dof_shot = stats.dof_updates_forward + stats.dof_updates_backward
    if dist is not None:
        t = torch.tensor([sec], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        sec = float(t.item())
    value = world * dof_shot * args.steps / sec

    # roofline of the dominant kernel: the fused backward step over every element (two wavefields)
    Np, Nfp = info.Np, info.Nfp
    bw_ms = stats.prof_backward_ms / max(stats.prof_backward_launches, 1)
    fw_ms = stats.prof_forward_ms / max(stats.prof_forward_launches, 1)
    bytes_bw = w.K * step_bytes_per_element(Np, Nfp, 2) + info.n_half_step * 2 * 8 * Nfp * 4
    bytes_fw = w.K * step_bytes_per_element(Np, Nfp, 1) + info.n_half_step * 8 * Nfp * 4
    peak, peak_kind = _peaks()
    ach_bw = bytes_bw / (bw_ms * 1e-3) / 1e9
    ach_fw = bytes_fw / (fw_ms * 1e-3) / 1e9
    tr = _traffic()
    traffic = None
    if tr and tr.get("kernel") == "dg_step_kernel_tc<4,2>" and tr.get("source_hash") == _kernel_hash():
        traffic = tr.get("bytes_per_launch_full_mesh")
    roofline = {"bound": "hbm", "achieved": ach_bw, "peak": peak, "unit": "GB/s", "frac": ach_bw / peak,
                "traffic": traffic, "kernel": "dg_step_kernel_tc<4,2> (backward S+R+images, all levels)",
                "peak_kind": peak_kind, "algorithmic_bytes_per_launch": bytes_bw, "avg_launch_ms": bw_ms,
                "forward_kernel": {"achieved": ach_fw, "frac": ach_fw / peak, "avg_launch_ms": fw_ms,
                                   "algorithmic_bytes_per_launch": bytes_fw}}

    # end to end through the host-buffer call: H2D of the observed traces, D2H of traces and images
    obs_host = observed.cpu().numpy()
    t0 = time.perf_counter()
    tr_h, ip_h, iq_h = s.rtm_shot(src_x, w.f0, w.t_peak, 1.0, w.receivers, w.t_final, w.t_image_start,
                                  observed=obs_host)
    e2e_sec = time.perf_counter() - t0
    if dist is not None:
        t = torch.tensor([e2e_sec], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_sec = float(t.item())
    e2e = {"value": world * dof_shot / e2e_sec, "unit": UNIT, "h2d_bytes_per_step": int(obs_host.nbytes),
           "d2h_bytes_per_step": int(tr_h.nbytes + ip_h.nbytes + iq_h.nbytes), "shots_per_s": world / e2e_sec}

    # the stated error of the FP32 shot: the same model, source and receivers over a short record in
    # the library's FP64 mode (itself held to the FP64 oracle at 1e-10 by the parity tests)
    error = None
    if rank == 0 and not args.no_error:
        t_err = 0.01
        try:
            s64 = ridg.Solver(mesh, w.N, w.c, w.rho, dtype="f64", cfl=w.cfl, n_levels_max=w.n_levels_max)
            a = s.rtm_shot(src_x, w.f0, w.t_peak, 1.0, w.receivers, t_err)
            b = s64.rtm_shot(src_x, w.f0, w.t_peak, 1.0, w.receivers, t_err)
            del s64

            def rl2(x, y):
                return float(np.linalg.norm(x - y) / max(np.linalg.norm(y), 1e-300))

            error = {"record_s": t_err, "traces_rel_l2": rl2(a[0], b[0]), "image_p_rel_l2": rl2(a[1], b[1]),
                     "image_q_rel_l2": rl2(a[2], b[2]),
                     "reference": "same shot over a 0.01 s record in the library's FP64 mode"}
        except ridg.RidgError as exc:  # reported in the line; the throughput stands on its own
            error = {"record_s": t_err, "failed": str(exc)}

    # serving: short shots through the shot server with Poisson arrivals below its capacity, for the
    # p50/p99 latency the metric quotes (a different, shorter record than the throughput shot)
    serving = None
    if rank == 0 and not args.no_serving:
        try:
            serving = _serving(ridg, torch, mesh, w, src_x)
        except ridg.RidgError as exc:  # reported in the line; the throughput stands on its own
            serving = {"failed": str(exc)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": _config(w, {"levels": [int(x) for x in info.level_count[:info.n_levels]],
                                  "dt_local_s": info.dt_local, "global_steps": int(stats.n_global),
                                  "boundary_trace_bytes": int(stats.boundary_trace_bytes),
                                  "parallelism": f"shots x{world} (replicas, image all-reduce)"}),
            "shots_per_s": world * args.steps / sec,
            "dof_updates_per_shot": int(dof_shot),
            "wall_s": wall,
            "roofline": roofline,
            "e2e": e2e,
            "error_vs_fp64": error,
            "serving": serving,
            "gpu_launches": int(launches),
            "clocks": clocks,
        }
        # the oracle CPU baseline (rank 0, N = 1) runs after every GPU leg, so it shares no host cores
        # with the GPU measurement
        if world == 1 and not args.no_cpu_baseline:
            torch.cuda.synchronize()
            try:
                line["cpu_baseline"] = cpu_baseline_line()
            except Exception as exc:  # noqa: BLE001
                line["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 0, "kind": "oracle",
                                        "sample": f"failed: {exc}"}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def profile_shot(t_final):
    """One short shot of the bench workload (same mesh, order, precision and launch configuration),
    for ncu captures: the first fused launch covers every element forward, the first backward
    launch every element with two wavefields."""
    from paper_1506_00907_gb300 import ridg

    w = _workload()
    mesh = ridg.Mesh(w.xyz, w.tets, default_bc=w.default_bc)
    s = ridg.Solver(mesh, w.N, w.c, w.rho, dtype="f32", cfl=w.cfl, n_levels_max=w.n_levels_max)
    tr, ip, iq = s.rtm_shot(w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, t_final)
    st = s.shot_stats()
    print(json.dumps({"n_global": st.n_global, "fused_launches": st.fused_launches,
                      "first_backward_fused_launch": st.fused_launches - st.n_global * (2 ** (s.info.n_levels - 1)),
                      "kernel_launches": st.kernel_launches, "finite": bool(np.isfinite(ip).all())}))
    return 0


def precision_sweep(orders, t_final=0.01):
    """Per order: the bench model's shot over a short record in FP64, in FP32 with the element
    products on tensor cores (three-term TF32 split, or BF16 hi + lo split) and in FP32 with them on
    CUDA cores; throughput,
    fused-kernel times and the relative L2 error of traces and images against the FP64 shot.  One
    JSON line per order."""
    from paper_1506_00907_gb300 import ridg

    w = _workload()
    mesh = ridg.Mesh(w.xyz, w.tets, default_bc=w.default_bc)

    def rel(a, b):
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

    for N in orders:
        out = {"order": N, "elements": int(w.K), "record_s": t_final}
        res = {}
        for name, dtype, contraction in (("f64", "f64", ridg.CONTRACT_TENSOR),
                                         ("f32_tensor_tf32x3", "f32", ridg.CONTRACT_TENSOR_TF32),
                                         ("f32_tensor_bf16x3", "f32", ridg.CONTRACT_TENSOR_BF16),
                                         ("f32_tensor_fp16x3", "f32", ridg.CONTRACT_TENSOR_FP16),
                                         ("f32_cuda_cores", "f32", ridg.CONTRACT_CUDA_CORES)):
            try:
                s = ridg.Solver(mesh, N, w.c, w.rho, dtype=dtype, cfl=w.cfl, n_levels_max=w.n_levels_max,
                                contraction=contraction)
            except ridg.RidgError as exc:
                out[name] = {"unavailable": str(exc)}
                continue
            s.set_profiling(1)
            s.rtm_shot(w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, 0.002)  # warm-up
            t0 = time.perf_counter()
            tr, ip, iq = s.rtm_shot(w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, t_final)
            wall = time.perf_counter() - t0
            st = s.shot_stats()
            res[name] = (tr, ip, iq)
            out[name] = {"dof_updates_per_s": (st.dof_updates_forward + st.dof_updates_backward) / wall,
                         "forward_full_launch_ms": st.prof_forward_ms / max(1, st.prof_forward_launches),
                         "backward_full_launch_ms": st.prof_backward_ms / max(1, st.prof_backward_launches)}
            s.close()
        if "f64" in res:
            for name in ("f32_tensor_tf32x3", "f32_tensor_bf16x3", "f32_tensor_fp16x3", "f32_cuda_cores"):
                if name in res:
                    out[name].update({k: rel(a, b) for k, a, b in zip(("traces_rel_l2", "image_p_rel_l2",
                                                                      "image_q_rel_l2"), res[name], res["f64"])})
        elif "f32_tensor_tf32x3" in res and "f32_cuda_cores" in res:
            out["tensor_vs_cuda_cores"] = {k: rel(a, b) for k, a, b in zip(
                ("traces_rel_l2", "image_p_rel_l2", "image_q_rel_l2"), res["f32_tensor_tf32x3"], res["f32_cuda_cores"])}
        print(json.dumps(out), flush=True)
    return 0


def serving_stream(n_req, t_rec=0.01, sizes=("50k", "200k", "800k"), slot_counts=(1, 2), contraction="tf32",
                   batch_sizes=(1,)):
    """Shot-serving stream over the serving models (about 5e4 / 2e5 / 8e5 elements at N = 3 / 4 / 5,
    three layers, three rate levels; ``sizes`` picks a subset): n_req requests (model, surface
    source, 101-401 receivers; seed 5) with Poisson arrivals (seed 5) at 0.8x and 1.5x the measured
    sequential rate, served with each number of slots per model in ``slot_counts`` and, for each
    size in ``batch_sizes``, slots that start up to that many waiting requests of their model as one
    lockstep batch (the same arrival times for every setting; the sequential rate is that of one shot
    at a time); FP32 with the TF32 or BF16 split.  Prints one JSON line."""
    import torch

    from paper_1506_00907_gb300 import ridg
    from synth import serving_model, serving_requests

    nm = len(sizes)
    kmax = max(slot_counts)
    models = [serving_model(sz) for sz in sizes]
    meshes = [ridg.Mesh(w.xyz, w.tets, default_bc=w.default_bc) for w in models]
    ctr = ridg.CONTRACT_TENSOR_BF16 if contraction == "bf16" else ridg.CONTRACT_TENSOR
    streams, slots = [], {}
    for m, (w, mesh) in enumerate(zip(models, meshes)):
        slots[m] = []
        for _ in range(kmax):
            st = torch.cuda.Stream()
            streams.append(st)
            slots[m].append(ridg.Solver(mesh, w.N, w.c, w.rho, dtype="f32", cfl=w.cfl, n_levels_max=w.n_levels_max,
                                        stream=st.cuda_stream, contraction=ctr))
    reqs = [(m % nm, src, rec) for m, src, rec in serving_requests(n_req)]
    out = {"requests": n_req, "record_s": t_rec, "contraction": contraction, "batch_sizes": list(batch_sizes),
           "models": [{"elements": int(w.K), "order": w.N, "levels": s[0].info.n_levels} for w, s in
                      zip(models, slots.values())],
           "arrivals": "Poisson (seed 5) at 0.8x and 1.5x the sequential rate; model, source and receiver count "
                       "drawn per request (seed 5)"}

    def submit(sv, r):
        m, src, rec = r
        w = models[m]
        return sv.submit(src, w.f0, w.t_peak, 1.0, rec, t_rec, model=m)

    def server(k, batch=1):
        sl = [slots[m][i] for m in range(nm) for i in range(k)]
        return ridg.Server(sl, max_queued=n_req, models=[m for m in range(nm) for _ in range(k)], max_batch=batch)

    with server(kmax) as sv:  # buffers of every slot in place
        for t in [submit(sv, (m, (1000.0, 1000.0, 8.0), reqs[0][2])) for m in range(nm) for _ in range(kmax)]:
            sv.wait(t)
    n_seq = min(n_req, 48)
    with server(1) as sv:
        t0 = time.perf_counter()
        for r in reqs[:n_seq]:
            sv.wait(submit(sv, r))
        seq = n_seq / (time.perf_counter() - t0)
    out["sequential_shots_per_s"] = seq
    for k, bsz, factor in [(k, b, f) for k in slot_counts for b in batch_sizes for f in (0.8, 1.5)]:
        gaps = np.random.default_rng(5).exponential(1.0 / (factor * seq), n_req)
        with server(k, bsz) as sv:
            t0 = time.perf_counter()
            arrive, tickets = 0.0, []
            for i, r in enumerate(reqs):
                arrive += gaps[i]
                time.sleep(max(0.0, arrive - (time.perf_counter() - t0)))
                tickets.append(submit(sv, r))
            lat = [sv.wait(t)[3]["total_s"] for t in tickets]
            span = time.perf_counter() - t0 - gaps[0]
        key = f"rate{factor}x_slots{k}" + ("" if bsz == 1 else f"_batch{bsz}")
        out[key] = {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                    "shots_per_s": n_req / span, "vs_sequential": n_req / span / seq}
    for ss in slots.values():
        for x in ss:
            x.close()
    print(json.dumps(out), flush=True)
    return 0


def batch_bench(sizes=("50k", "200k"), t_rec=0.01, batches=(1, 2, 4), reps=3, contraction="tf32"):
    """Lockstep shot batches (ridg_rtm_shots_device: one merged launch per fine step over every shot of
    the batch) against the same shots one after another, on the serving models (surface sources and
    receiver lines of the serving stream, seed 5), FP32 with the TF32 or BF16 split: shots/s and
    DOF-updates/s, CUDA events around ``reps`` back-to-back batches of each size (device buffers, so
    the host copies are left out), launched kernel by kernel and replayed as CUDA graphs.  Prints one
    JSON line."""
    import torch

    from paper_1506_00907_gb300 import ridg
    from synth import serving_model, serving_requests

    ctr = ridg.CONTRACT_TENSOR_BF16 if contraction == "bf16" else ridg.CONTRACT_TENSOR
    reqs = serving_requests(4 * max(batches))
    out = {"record_s": t_rec, "contraction": contraction, "reps": reps, "models": []}
    for sz in sizes:
        w = serving_model(sz)
        mesh = ridg.Mesh(w.xyz, w.tets, default_bc=w.default_bc)
        st = torch.cuda.Stream()
        s = ridg.Solver(mesh, w.N, w.c, w.rho, dtype="f32", cfl=w.cfl, n_levels_max=w.n_levels_max,
                        stream=st.cuda_stream, contraction=ctr)
        n_t = s.trace_len(t_rec)
        shots = []
        for _, src, rec in reqs[:max(batches)]:
            shots.append(dict(source_xyz=src, f0=w.f0, t_peak=w.t_peak, amplitude=1.0, rec_xyz=rec,
                              traces=torch.zeros((len(rec), n_t), dtype=torch.float64, device="cuda"),
                              image_p=torch.zeros((w.K, s.Np), dtype=torch.float64, device="cuda"),
                              image_q=torch.zeros((w.K, s.Np), dtype=torch.float64, device="cuda")))
        row = {"elements": int(w.K), "order": w.N, "levels": s.info.n_levels}
        s.rtm_shots_device(shots, t_rec)  # every shot's buffers in place
        torch.cuda.synchronize()
        for graph in (False, True):
            s.set_graph_replay(graph)
            for b in batches:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                for _ in range(2 if graph else 1):  # with graphs: the direct run and the capture
                    s.rtm_shots_device(shots[:b], t_rec)
                e0.record(st)
                for _ in range(reps):
                    s.rtm_shots_device(shots[:b], t_rec)
                e1.record(st)
                torch.cuda.synchronize()
                sec = e0.elapsed_time(e1) / 1e3
                stt = s.shot_stats()
                dof = (stt.dof_updates_forward + stt.dof_updates_backward) * reps
                row[f"batch{b}" + ("_graph" if graph else "")] = {
                    "shots_per_s": reps * b / sec, "dof_updates_per_s": dof / sec, "ms_per_batch": 1e3 * sec / reps,
                    "graph_replay": int(stt.graph_replay)}
        s.set_graph_replay(False)
        base = row[f"batch{batches[0]}"]["shots_per_s"]
        for key in [k for k in row if k.startswith("batch")]:
            row[key][f"vs_batch{batches[0]}"] = row[key]["shots_per_s"] / base
        out["models"].append(row)
        s.close()
    print(json.dumps(out), flush=True)
    return 0


def gradient_bench(dtype="f64", n_checkpoints=16, model="box"):
    """Misfit gradient: on the 648-element adjoint box (N = 3, one rate level, 0.5 s record, 25
    receivers, observed data from a model with a 5 % Gaussian velocity bump), or with ``model ==
    "bench"`` on the bench mesh (190,608 elements, N = 4, FP32, one rate level, 0.005 s record, 201
    receivers, observed data zero), or with ``model == "bench3"`` on the bench mesh with its three
    rate levels: time of the forward run with checkpoints and of the adjoint sweep.  One JSON line."""
    from paper_1506_00907_gb300 import ridg
    from synth import adjoint_box, adjoint_observed_velocity

    levels = 3 if model == "bench3" else 1
    if model in ("bench", "bench3"):
        w = _workload()
        dtype, t_final = "f32", 0.005
    else:
        w = adjoint_box()
        t_final = w.t_final
    w.t_final = t_final
    mesh = ridg.Mesh(w.xyz, w.tets, default_bc=w.default_bc)
    s = ridg.Solver(mesh, w.N, w.c, w.rho, dtype=dtype, cfl=w.cfl, n_levels_max=levels)
    n_t = s.trace_len(w.t_final)
    nrec = len(w.receivers)
    if model in ("bench", "bench3"):
        obs = np.zeros((nrec, n_t))
    else:
        s.set_velocity(adjoint_observed_velocity(w))
        _, obs = s.misfit_forward(w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final, np.zeros((nrec, n_t)))
        s.set_velocity(w.c)
    times = []
    for _ in range(3):
        t0 = time.perf_counter()
        J, _ = s.misfit_forward(w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final, obs, n_checkpoints)
        t1 = time.perf_counter()
        g = s.misfit_backward()
        t2 = time.perf_counter()
        times.append((t1 - t0, t2 - t1))
    fw, bw = min(t[0] for t in times), min(t[1] for t in times)
    label = {"bench": "bench mesh: 190608 tets, N=4, FP32, one level, 0.005 s record, 201 receivers",
             "bench3": "bench mesh: 190608 tets, N=4, FP32, three levels, 0.005 s record, 201 receivers"}.get(
                 model, "adjoint box: 648 tets, N=3, one level, 0.5 s record, 25 receivers")
    print(json.dumps({"workload": label, "elements": int(w.K),
                      "dtype": dtype, "steps": n_t - 1, "checkpoints": n_checkpoints, "misfit": J,
                      "grad_norm": float(np.linalg.norm(g)), "forward_s": fw, "backward_s": bw,
                      "gradient_s": fw + bw, "forward_us_per_step": 1e6 * fw / (n_t - 1),
                      "backward_us_per_step": 1e6 * bw / (n_t - 1)}), flush=True)
    return 0


def group_bench(n_parts, t_final=0.01):
    """Domain decomposition on one device: the bench model's shot over a short record with the mesh
    split into n_parts (the library's partition; each part its own solver and stream, interface traces
    copied after every fine step) against the single solver; wall times, the transfer counts and bytes,
    and whether the results are bit for bit the single solver's.  One JSON line."""
    from paper_1506_00907_gb300 import ridg

    w = _workload()
    mesh = ridg.Mesh(w.xyz, w.tets, default_bc=w.default_bc)
    args = (w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, t_final)
    s = ridg.Solver(mesh, w.N, w.c, w.rho, dtype="f32", cfl=w.cfl, n_levels_max=w.n_levels_max)
    s.rtm_shot(*args)  # buffers in place
    t0 = time.perf_counter()
    ref = s.rtm_shot(*args)
    t_single = time.perf_counter() - t0
    s.close()
    part = ridg.partition(mesh, w.N, w.c, n_parts, cfl=w.cfl, n_levels_max=w.n_levels_max)
    g = ridg.Group(mesh, w.N, w.c, w.rho, part, cfl=w.cfl, n_levels_max=w.n_levels_max)
    g.rtm_shot(*args)
    t0 = time.perf_counter()
    out = g.rtm_shot(*args)
    t_group = time.perf_counter() - t0
    info = g.info()
    print(json.dumps({"workload": f"bench mesh {w.K} tets N={w.N} FP32, {t_final} s record, {n_parts} parts on one device",
                      "single_s": t_single, "group_s": t_group, "group_vs_single": t_single / t_group,
                      "elements": list(info.elements[:n_parts]), "ghosts": list(info.ghosts[:n_parts]),
                      "interface_faces": list(info.interface_faces[:n_parts]), "transfer_steps": info.transfer_steps,
                      "silent_steps": info.silent_steps, "transfer_bytes": info.transfer_bytes,
                      "bitwise_equal": bool(all(np.array_equal(a, b) for a, b in zip(out, ref)))}), flush=True)
    g.close()
    return 0


def tier_bench(budget_gb, t_final=0.2):
    """Boundary-trace records beyond a device budget on the bench model: the same shot (FP32, a
    shorter record) with every record on the device and with budget_gb of device memory for them
    (the rest in pinned host memory, moved in chunks on a second stream); wall times, chunks, bytes
    and whether the results are bit for bit the same.  One JSON line."""
    from paper_1506_00907_gb300 import ridg

    w = _workload()
    mesh = ridg.Mesh(w.xyz, w.tets, default_bc=w.default_bc)
    args = (w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, t_final)
    s = ridg.Solver(mesh, w.N, w.c, w.rho, dtype="f32", cfl=w.cfl, n_levels_max=w.n_levels_max)
    s.rtm_shot(*args)  # buffers in place
    t0 = time.perf_counter()
    ref = s.rtm_shot(*args)
    t_dev = time.perf_counter() - t0
    full = s.shot_stats().boundary_trace_bytes
    s.set_trace_budget(int(budget_gb * 1e9))
    s.rtm_shot(*args)  # host memory in place
    t0 = time.perf_counter()
    out = s.rtm_shot(*args)
    t_tier = time.perf_counter() - t0
    st = s.shot_stats()
    print(json.dumps({"workload": f"bench mesh {w.K} tets N={w.N} FP32, {t_final} s record",
                      "record_bytes": full, "device_budget_bytes": int(budget_gb * 1e9),
                      "chunks": st.trace_chunks, "host_bytes_each_way": st.host_trace_bytes,
                      "all_device_s": t_dev, "tiered_s": t_tier, "tiered_vs_all_device": t_tier / t_dev,
                      "bitwise_equal": bool(all(np.array_equal(a, b) for a, b in zip(out, ref)))}), flush=True)
    s.close()
    return 0


def _kernel_hash():
    import hashlib

    h = hashlib.sha1()
    for f in ("step_kernel.cuh", "step_kernel_tc.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1506_00907_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:12]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ridg", choices=["ridg", "reference"])
    ap.add_argument("--no-error", action="store_true", help="skip the FP32-vs-FP64 error leg")
    ap.add_argument("--no-serving", action="store_true", help="skip the shot-server latency leg")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-shot", type=float, default=0.0,
                    help="run one shot of the bench workload with this record length (s) and exit (profiling case)")
    ap.add_argument("--precision-sweep", default="",
                    help="comma-separated orders: FP64 / FP32 tensor-core / FP32 CUDA-core shots of the bench model")
    ap.add_argument("--serving-stream", type=int, default=0,
                    help="run the three-model shot-serving stream with this many requests and exit")
    ap.add_argument("--serving-sizes", default="50k,200k,800k", help="serving models (subset of 50k,200k,800k)")
    ap.add_argument("--serving-slots", default="1,2", help="slots per model to compare")
    ap.add_argument("--serving-contraction", default="tf32", choices=["tf32", "bf16"])
    ap.add_argument("--serving-batch", default="1",
                    help="batch sizes to compare: waiting requests of a model a slot starts together (1..4)")
    ap.add_argument("--batch-bench", default="", help="lockstep batch throughput on these serving models (e.g. 50k,200k)")
    ap.add_argument("--serving-record", type=float, default=0.01, help="record length (s) of each served shot")
    ap.add_argument("--gradient", default="", nargs="?", const="box", choices=["", "box", "bench", "bench3"],
                    help="time the misfit gradient (on the adjoint box, or on the bench mesh with one or three levels) and exit")
    ap.add_argument("--trace-budget", type=float, default=0.0,
                    help="time the bench shot (0.2 s record) with this many GB of device memory for its boundary-trace records and exit")
    ap.add_argument("--group-parts", type=int, default=0,
                    help="time the bench shot with the mesh split into this many parts on one device and exit")
    args = ap.parse_args()
    if args.trace_budget > 0:
        from paper_1506_00907_gb300.build import build

        build()
        return tier_bench(args.trace_budget)
    if args.group_parts > 0:
        from paper_1506_00907_gb300.build import build

        build()
        return group_bench(args.group_parts)
    if args.gradient:
        from paper_1506_00907_gb300.build import build

        build()
        return gradient_bench(model=args.gradient)
    if args.serving_stream > 0:
        from paper_1506_00907_gb300.build import build

        build()
        return serving_stream(args.serving_stream, t_rec=args.serving_record, sizes=tuple(args.serving_sizes.split(",")),
                              slot_counts=tuple(int(x) for x in args.serving_slots.split(",")),
                              contraction=args.serving_contraction,
                              batch_sizes=tuple(int(x) for x in args.serving_batch.split(",")))
    if args.batch_bench:
        from paper_1506_00907_gb300.build import build

        build()
        return batch_bench(tuple(args.batch_bench.split(",")), t_rec=args.serving_record,
                           contraction=args.serving_contraction)
    if args.precision_sweep:
        from paper_1506_00907_gb300.build import build

        build()
        return precision_sweep([int(x) for x in args.precision_sweep.split(",")])
    if args.profile_shot > 0:
        from paper_1506_00907_gb300.build import build

        build()
        return profile_shot(args.profile_shot)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    from paper_1506_00907_gb300.build import build

    build()
    return run_ridg(args)


if __name__ == "__main__":
    sys.exit(main())
