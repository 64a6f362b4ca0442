"""CUDA-graph replay of repeated shots (ridg_set_graph_replay): the second shot with the same launch
arguments captures its time stepping into a graph and later ones launch the graph.  Every result must
equal, bit for bit, the same shot launched kernel by kernel, also when the source and receiver
positions and the observed data change between replays (they are read from device tables); a change
of wavelet or receiver count runs directly again."""

import numpy as np
import pytest

from paper_1506_00907_gb300 import ridg
from synth import tiny_layered_rtm

pytestmark = pytest.mark.gpu


def _solvers(w, dtype):
    import torch

    mesh = ridg.Mesh(w.xyz, w.tets, default_bc=w.default_bc)
    out = []
    for graph in (False, True):
        st = torch.cuda.Stream()
        s = ridg.Solver(mesh, w.N, w.c, w.rho, dtype=dtype, cfl=w.cfl, n_levels_max=w.n_levels_max,
                        stream=st.cuda_stream)
        s.set_graph_replay(graph)
        out.append((s, st))
    return out


def _buffers(s, w, nrec, n_t):
    import torch

    z = dict(dtype=torch.float64, device="cuda")
    return dict(traces=torch.zeros((nrec, n_t), **z), image_p=torch.zeros((w.K, s.Np), **z),
                image_q=torch.zeros((w.K, s.Np), **z))


def _run(s, bufs, shots, w):
    import torch

    torch.cuda.synchronize()
    s.rtm_shots_device([dict(sh, **b) for sh, b in zip(shots, bufs)], w.t_final)
    torch.cuda.synchronize()
    return [tuple(b[k].cpu().numpy().copy() for k in ("traces", "image_p", "image_q")) for b in bufs], \
        s.shot_stats().graph_replay


@pytest.mark.parametrize("dtype,n", [("f32", 1), ("f32", 2), ("f64", 1)])
def test_graph_replay_equals_direct_launches(dtype, n):
    import torch

    w = tiny_layered_rtm(N=3, t_final=0.003)
    (direct, _), (graphed, _) = _solvers(w, dtype)
    n_t = direct.trace_len(w.t_final)
    rng = np.random.default_rng(31)
    nrec = len(w.receivers)

    def shots(k):  # k-th set: the sources and receivers move, the wavelet and receiver count stay
        out = []
        for b in range(n):
            src = (90.0 + 7.0 * k + 15.0 * b, 100.0 - 5.0 * b, 4.0)
            rec = w.receivers + np.array([3.0 * k, 2.0 * b, 0.0])
            sh = dict(source_xyz=src, f0=w.f0, t_peak=w.t_peak, amplitude=1.0, rec_xyz=rec)
            out.append(sh)
        return out

    bd = [_buffers(direct, w, nrec, n_t) for _ in range(n)]
    bg = [_buffers(graphed, w, nrec, n_t) for _ in range(n)]
    modes = []
    for k in range(4):
        ref, r0 = _run(direct, bd, shots(k), w)
        got, rg = _run(graphed, bg, shots(k), w)
        assert r0 == 0
        modes.append(rg)
        for a, c in zip(ref, got):
            for x, y in zip(a, c):
                assert np.array_equal(x, y)
    assert modes == [0, 1, 1, 1]  # direct, captured, replayed, replayed
    # observed data instead of the modelled traces: other device buffers, a new key, then replays
    obs = [torch.tensor(rng.standard_normal((nrec, n_t)), device="cuda") for _ in range(n)]
    for k in range(3):
        sh = [dict(x, observed=o) for x, o in zip(shots(k), obs)]
        ref, _ = _run(direct, bd, sh, w)
        got, rg = _run(graphed, bg, sh, w)
        assert rg == (0 if k == 0 else 1)
        for a, c in zip(ref, got):
            for x, y in zip(a, c):
                assert np.array_equal(x, y)
        for o in obs:  # new data values in place: the graph reads them
            o.copy_(torch.tensor(rng.standard_normal((nrec, n_t)), device="cuda"))
    # another wavelet amplitude: its values are launch arguments, so the shot runs directly
    sh = [dict(x, amplitude=2.0) for x in shots(0)]
    ref, _ = _run(direct, bd, sh, w)
    got, rg = _run(graphed, bg, sh, w)
    assert rg == 0
    for a, c in zip(ref, got):
        for x, y in zip(a, c):
            assert np.array_equal(x, y)


def test_server_slot_with_graph_replay():
    """A server slot whose solver replays graphs: its repeated requests (new sources, same receiver
    count and wavelet) give the results of the same shots alone."""
    import torch

    w = tiny_layered_rtm(N=3, t_final=0.003)
    (direct, _), (graphed, _) = _solvers(w, "f32")
    sources = [(95.0 + 5.0 * k, 100.0, 4.0) for k in range(5)]
    alone = [direct.rtm_shot(x, w.f0, w.t_peak, 1.0, w.receivers, w.t_final) for x in sources]
    with ridg.Server(graphed, max_queued=8) as sv:
        served = [sv.wait(sv.submit(x, w.f0, w.t_peak, 1.0, w.receivers, w.t_final), timeout=120) for x in sources]
    replays = graphed.shot_stats().graph_replay  # the last request's
    for (tr, ip, iq), (tr2, ip2, iq2, _) in zip(alone, served):
        assert np.array_equal(tr, tr2) and np.array_equal(ip, ip2) and np.array_equal(iq, iq2)
    assert replays == 1
    torch.cuda.synchronize()


def test_graph_replay_stays_off_with_profiling_or_a_trace_budget():
    """Profiling events and the host-memory record tier need the shot launched step by step: with
    either, repeated shots with fixed device buffers run directly (and give the same results)."""
    w = tiny_layered_rtm(N=3, t_final=0.003)
    (direct, _), (graphed, _) = _solvers(w, "f32")
    n_t = direct.trace_len(w.t_final)
    sh = [dict(source_xyz=w.source_xyz, f0=w.f0, t_peak=w.t_peak, amplitude=1.0, rec_xyz=w.receivers)]
    bd = [_buffers(direct, w, len(w.receivers), n_t)]
    bg = [_buffers(graphed, w, len(w.receivers), n_t)]
    ref, _ = _run(direct, bd, sh, w)
    total = direct.shot_stats().boundary_trace_bytes
    graphed.set_profiling(1)
    for _ in range(3):
        got, rg = _run(graphed, bg, sh, w)
        assert rg == 0
        assert all(np.array_equal(a, b) for a, b in zip(ref[0], got[0]))
    graphed.set_profiling(0)
    graphed.set_trace_budget(max(total // 4, 1 << 16))
    for _ in range(3):
        got, rg = _run(graphed, bg, sh, w)
        assert rg == 0 and graphed.shot_stats().trace_chunks > 1
        assert all(np.array_equal(a, b) for a, b in zip(ref[0], got[0]))
    graphed.set_trace_budget(0)  # all records on the device again: the graphs come back
    modes = [_run(graphed, bg, sh, w)[1] for _ in range(3)]
    assert modes == [0, 1, 1]
