"""Several shots of one model in lockstep (ridg_rtm_shots): one merged launch of the fused step kernel
per fine step over the active elements of every shot.  Each shot of a batch must give exactly (bit for
bit) what the same shot gives alone, whatever its neighbours in the batch (sources, wavelets, receiver
counts, observed data), in every contraction mode; one batched shot is also held to the FP64 oracle
at the stated tolerances."""

import time

import numpy as np
import pytest

from oracle.rtm import make_problem, rtm_shot
from paper_1506_00907_gb300 import ridg
from synth import tiny_layered_rtm
from tests.parity_cases import TOL, rel_l2

pytestmark = pytest.mark.gpu


def _shots(w, n_t):
    """Three different shots of the tiny three-level model: a Ricker pulse at the source with the
    standard receivers, a shifted lower-frequency pulse with fewer receivers and observed data that
    are not the modelled traces, and a sampled wavelet with more receivers."""
    rng = np.random.default_rng(23)
    rec2 = w.receivers[::2].copy()
    rec3 = np.stack([np.linspace(20.0, 180.0, 11), np.full(11, 90.0), np.full(11, 6.0)], axis=1)
    dt_s = 1e-4
    t = np.arange(80) * dt_s
    samples = np.sin(2 * np.pi * 300.0 * t) * np.exp(-((t - 0.003) / 0.001) ** 2)
    return [
        dict(source_xyz=w.source_xyz, f0=w.f0, t_peak=w.t_peak, amplitude=1.0, rec_xyz=w.receivers),
        dict(source_xyz=(120.0, 90.0, 6.0), f0=0.8 * w.f0, t_peak=w.t_peak / 0.8, amplitude=-2.0, rec_xyz=rec2,
             observed=rng.standard_normal((len(rec2), n_t))),
        dict(source_xyz=(85.0, 110.0, 3.0), amplitude=0.5, rec_xyz=rec3, wavelet=samples, wavelet_dt=dt_s),
    ]


def _alone(s, sh, t_final, t_i):
    return s.rtm_shot(sh["source_xyz"], sh.get("f0", 10.0), sh.get("t_peak", 0.0), sh.get("amplitude", 1.0),
                      sh["rec_xyz"], t_final, t_i, observed=sh.get("observed"), wavelet=sh.get("wavelet"),
                      wavelet_dt=sh.get("wavelet_dt"))


def _solver(w, dtype, contraction=ridg.CONTRACT_TENSOR):
    mesh = ridg.Mesh(w.xyz, w.tets, default_bc=w.default_bc)
    return ridg.Solver(mesh, w.N, w.c, w.rho, dtype=dtype, cfl=w.cfl, n_levels_max=w.n_levels_max,
                       contraction=contraction)


@pytest.mark.parametrize("dtype,contraction", [("f32", ridg.CONTRACT_TENSOR), ("f32", ridg.CONTRACT_TENSOR_BF16),
                                               ("f32", ridg.CONTRACT_TENSOR_FP16), ("f32", ridg.CONTRACT_CUDA_CORES),
                                               ("f64", ridg.CONTRACT_TENSOR)])
def test_batch_equals_each_shot_alone(dtype, contraction):
    w = tiny_layered_rtm(N=3, t_final=0.004)
    t_i = 0.25 * w.t_final
    s = _solver(w, dtype, contraction)
    n_t = s.trace_len(w.t_final)
    shots = _shots(w, n_t)
    alone = [_alone(s, sh, w.t_final, t_i) for sh in shots]
    batch = s.rtm_shots(shots, w.t_final, t_i)
    st = s.shot_stats()
    for (tr, ip, iq), (tr0, ip0, iq0) in zip(batch, alone):
        assert tr.shape == tr0.shape
        assert np.array_equal(tr, tr0) and np.array_equal(ip, ip0) and np.array_equal(iq, iq0)
        assert np.abs(ip).max() > 0 and np.abs(tr).max() > 0
    # a smaller batch right after (buffers reused), in another order
    again = s.rtm_shots([shots[2], shots[0]], w.t_final, t_i)
    for (tr, ip, iq), k in zip(again, (2, 0)):
        assert np.array_equal(tr, alone[k][0]) and np.array_equal(ip, alone[k][1]) and np.array_equal(iq, alone[k][2])
    # the batch counts the DOF updates of all its shots; FP32 tensor-core batches take one launch
    # per fine step, the other kernels one per shot
    s.rtm_shot(shots[0]["source_xyz"], shots[0]["f0"], shots[0]["t_peak"], 1.0, shots[0]["rec_xyz"], w.t_final, t_i)
    one = s.shot_stats()
    assert st.dof_updates_forward == 3 * one.dof_updates_forward
    assert st.dof_updates_backward == 3 * one.dof_updates_backward
    merged = dtype == "f32" and contraction != ridg.CONTRACT_CUDA_CORES
    assert st.fused_launches == (1 if merged else 3) * one.fused_launches


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batched_shot_matches_oracle(dtype):
    """The second shot of a batch (shifted source, observed data) against the FP64 oracle."""
    w = tiny_layered_rtm(N=3, t_final=0.004)
    s = _solver(w, dtype)
    n_t = s.trace_len(w.t_final)
    shots = _shots(w, n_t)[:2]
    out = s.rtm_shots(shots, w.t_final, 0.0)
    prob = make_problem(w.xyz, w.tets, w.c, w.rho, w.N, default_bc=w.default_bc, cfl=w.cfl,
                        n_levels_max=w.n_levels_max)
    sh = shots[1]
    ref = rtm_shot(prob, sh["source_xyz"], sh["f0"], sh["t_peak"], sh["amplitude"], sh["rec_xyz"], w.t_final, 0.0,
                   observed=sh["observed"])
    tr, ip, iq = out[1]
    assert rel_l2(tr, ref.traces) < TOL[dtype]
    assert rel_l2(ip, ref.image_p) < TOL[dtype]
    assert rel_l2(iq, ref.image_q) < TOL[dtype]


def test_batch_device_buffers_and_limits():
    import torch

    w = tiny_layered_rtm(N=3, t_final=0.003)
    s = _solver(w, "f32")
    n_t = s.trace_len(w.t_final)
    shots = _shots(w, n_t)
    host = s.rtm_shots(shots, w.t_final)
    dev = []
    for sh in shots:
        d = dict(sh)
        if sh.get("observed") is not None:
            d["observed"] = torch.tensor(sh["observed"], device="cuda")
        d["traces"] = torch.zeros((len(sh["rec_xyz"]), n_t), dtype=torch.float64, device="cuda")
        d["image_p"] = torch.zeros((w.K, s.Np), dtype=torch.float64, device="cuda")
        d["image_q"] = torch.zeros_like(d["image_p"])
        dev.append(d)
    s.rtm_shots_device(dev, w.t_final)
    torch.cuda.synchronize()
    for d, (tr, ip, iq) in zip(dev, host):
        assert np.array_equal(d["traces"].cpu().numpy(), tr)
        assert np.array_equal(d["image_p"].cpu().numpy(), ip) and np.array_equal(d["image_q"].cpu().numpy(), iq)
    with pytest.raises(ridg.RidgError):
        s.rtm_shots(shots + shots[:2], w.t_final)  # five shots: more than a batch holds
    s.set_trace_budget(1 << 20)
    with pytest.raises(ridg.RidgError):
        s.rtm_shots(shots[:2], w.t_final)  # a trace budget: one shot at a time
    s.set_trace_budget(0)
    out = s.rtm_shots(shots[:1], w.t_final)
    assert np.array_equal(out[0][0], host[0][0]) and np.array_equal(out[0][1], host[0][1])
    # a shot without receivers (no receiver run data) beside one with them
    silent = dict(shots[0], rec_xyz=np.zeros((0, 3)))
    mixed = s.rtm_shots([silent, shots[2]], w.t_final)
    alone = _alone(s, silent, w.t_final, 0.0)
    assert mixed[0][0].shape == (0, n_t)
    assert np.array_equal(mixed[0][1], alone[1]) and np.array_equal(mixed[0][2], alone[2])
    assert np.array_equal(mixed[1][0], host[2][0]) and np.array_equal(mixed[1][1], host[2][1])


def test_server_batches_waiting_requests():
    """A server with max_batch 3: requests that wait while the slot is busy start together (same start
    time) when they share the time span, at most three at a time; one with another record length is
    not batched with them; every result equals the same shot alone."""
    w = tiny_layered_rtm(N=3, t_final=0.004)
    s = _solver(w, "f32")
    shots = _shots(w, s.trace_len(w.t_final))
    specs = [(shots[0], w.t_final), (shots[1], w.t_final), (shots[2], 0.003), (shots[2], w.t_final),
             (shots[0], w.t_final)]
    alone = [_alone(s, sh, tf, 0.0) for sh, tf in specs]
    with ridg.Server(s, max_queued=8, max_batch=3) as sv:
        first = sv.submit(w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, 0.3, want_images=False)  # keeps it busy
        time.sleep(0.2)
        tickets = [sv.submit(sh["source_xyz"], sh.get("f0", 10.0), sh.get("t_peak", 0.0), sh.get("amplitude", 1.0),
                             sh["rec_xyz"], tf, observed=sh.get("observed"), wavelet=sh.get("wavelet"),
                             wavelet_dt=sh.get("wavelet_dt")) for sh, tf in specs]
        sv.wait(first, timeout=300)
        served = [sv.wait(t, timeout=300) for t in tickets]
    for (tr, ip, iq), (tr2, ip2, iq2, tm) in zip(alone, served):
        assert np.array_equal(tr, tr2) and np.array_equal(ip, ip2) and np.array_equal(iq, iq2)
    start = [x[3]["start_s"] for x in served]
    # requests 0, 1, 3 (same record) form the first batch; 2 (shorter record) and 4 follow
    assert start[0] == start[1] == start[3]
    assert start[2] != start[0] and start[4] != start[0]


def test_server_batch_with_a_failing_request():
    """A request whose source lies outside the mesh, batched with good ones: it completes with its own
    error (RIDG_E_NOT_FOUND) and the others with the results they give alone."""
    w = tiny_layered_rtm(N=3, t_final=0.004)
    s = _solver(w, "f32")
    shots = _shots(w, s.trace_len(w.t_final))
    alone = [_alone(s, sh, w.t_final, 0.0) for sh in shots[:2]]
    with ridg.Server(s, max_queued=8, max_batch=4) as sv:
        first = sv.submit(w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, 0.3, want_images=False)  # keeps it busy
        time.sleep(0.2)
        good0 = sv.submit(shots[0]["source_xyz"], shots[0]["f0"], shots[0]["t_peak"], 1.0, shots[0]["rec_xyz"],
                          w.t_final)
        bad = sv.submit((1e6, 0.0, 0.0), w.f0, w.t_peak, 1.0, w.receivers, w.t_final)
        good1 = sv.submit(shots[1]["source_xyz"], shots[1]["f0"], shots[1]["t_peak"], shots[1]["amplitude"],
                          shots[1]["rec_xyz"], w.t_final, observed=shots[1]["observed"])
        sv.wait(first, timeout=300)
        r0 = sv.wait(good0, timeout=300)
        with pytest.raises(ridg.RidgError) as e:
            sv.wait(bad, timeout=300)
        assert e.value.code == -7  # RIDG_E_NOT_FOUND
        r1 = sv.wait(good1, timeout=300)
    for (tr, ip, iq), got in zip(alone, (r0, r1)):
        assert np.array_equal(tr, got[0]) and np.array_equal(ip, got[1]) and np.array_equal(iq, got[2])
