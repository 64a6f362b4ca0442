"""Shot server (``ridg_server_*``): requests run one after another on the solver's resident
buffers and give the same results as the same shots run alone; a full queue, a wait that runs
out, a failing request and an unknown ticket are reported without disturbing the other requests."""

import time

import numpy as np
import pytest

from paper_1506_00907_gb300 import ridg
from synth import tiny_layered_rtm

pytestmark = pytest.mark.gpu


def _solver(w):
    mesh = ridg.Mesh(w.xyz, w.tets, default_bc=w.default_bc)
    return ridg.Solver(mesh, w.N, w.c, w.rho, dtype="f32", cfl=w.cfl, n_levels_max=w.n_levels_max)


def test_server_results_equal_standalone_shots():
    w = tiny_layered_rtm(N=3, t_final=0.006)
    s = _solver(w)
    x0 = np.asarray(w.source_xyz, dtype=float)
    sources = [tuple(x0 + np.array([dx, 0.0, 0.0])) for dx in (0.0, 20.0, -30.0)]
    records = [w.t_final, 0.004, w.t_final]  # different record lengths: the arena is reused and grown
    alone = [s.rtm_shot(src, w.f0, w.t_peak, 1.0, w.receivers, tf) for src, tf in zip(sources, records)]
    with ridg.Server(s, max_queued=4) as sv:
        tickets = [sv.submit(src, w.f0, w.t_peak, 1.0, w.receivers, tf) for src, tf in zip(sources, records)]
        served = [sv.wait(t, timeout=120) for t in tickets]
    for (tr, ip, iq), (tr2, ip2, iq2, tm) in zip(alone, served):
        assert np.array_equal(tr, tr2) and np.array_equal(ip, ip2) and np.array_equal(iq, iq2)
        assert 0.0 <= tm["queued_s"] <= tm["total_s"] and 0.0 < tm["run_s"] <= tm["total_s"]
    # first in, first out: each request waited at least as long as the one before it ran
    assert served[1][3]["queued_s"] >= served[0][3]["run_s"] * 0.5
    # the solver is usable again once the server is gone
    tr, _, _ = s.rtm_shot(sources[0], w.f0, w.t_peak, 1.0, w.receivers, w.t_final)
    assert np.array_equal(tr, alone[0][0])


def test_server_busy_timeout_and_errors():
    w = tiny_layered_rtm(N=3, t_final=0.006)
    s = _solver(w)
    long_record = 1.5  # keeps the worker busy for a while
    with ridg.Server(s, max_queued=1) as sv:
        t1 = sv.submit(w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, long_record, want_images=False)
        time.sleep(0.2)  # the worker has taken t1
        t2 = sv.submit((1e6, 0.0, 0.0), w.f0, w.t_peak, 1.0, w.receivers, w.t_final)  # source outside the mesh
        with pytest.raises(ridg.RidgError) as e:
            sv.submit(w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final)
        assert e.value.code == -8  # queue full
        with pytest.raises(ridg.RidgError) as e:
            sv.wait(t1, timeout=0.0)
        assert e.value.code == -6  # still running; the ticket stays valid
        tr1, ip1, iq1, tm1 = sv.wait(t1, timeout=300)
        assert ip1 is None and np.isfinite(tr1).all() and np.abs(tr1).max() > 0
        with pytest.raises(ridg.RidgError) as e:
            sv.wait(t2, timeout=300)
        assert e.value.code == -7  # the request's own error
        with pytest.raises(ridg.RidgError) as e:
            sv.wait(t2, timeout=1.0)
        assert e.value.code == -1  # released ticket
        # the server carries on after a failed request
        t3 = sv.submit(w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final)
        tr3, _, _, _ = sv.wait(t3, timeout=300)
        assert np.isfinite(tr3).all()


def test_server_sampled_source_equals_standalone_shot():
    """A request with a sampled source: the server keeps its own copy of the samples."""
    w = tiny_layered_rtm(N=3, t_final=0.004)
    s = _solver(w)
    dt_s = 0.4 * s.info.dt_local
    wav = np.sin(np.arange(int(w.t_final / dt_s)) * dt_s * 2 * np.pi * w.f0) ** 3
    alone = s.rtm_shot(w.source_xyz, 0.0, 0.0, 2.0, w.receivers, w.t_final, wavelet=wav, wavelet_dt=dt_s)
    with ridg.Server(s, max_queued=2) as sv:
        t = sv.submit(w.source_xyz, 0.0, 0.0, 2.0, w.receivers, w.t_final, wavelet=wav.copy(), wavelet_dt=dt_s)
        served = sv.wait(t, timeout=120)
    for a, b in zip(alone, served[:3]):
        assert np.array_equal(a, b)


def _stream_solver(w, torch, N=None):
    st = torch.cuda.Stream()
    mesh = ridg.Mesh(w.xyz, w.tets, default_bc=w.default_bc)
    s = ridg.Solver(mesh, w.N if N is None else N, w.c, w.rho, dtype="f32", cfl=w.cfl, n_levels_max=w.n_levels_max,
                    stream=st.cuda_stream)
    s._stream = st  # keep the stream alive with the solver
    return s


def test_slots_run_concurrently_and_match_standalone_shots():
    """Two slots of one model on their own streams: requests submitted together start on both slots
    at once, and every result equals the same shot run alone."""
    torch = pytest.importorskip("torch")
    w = tiny_layered_rtm(N=3, t_final=0.006)
    s1, s2 = _stream_solver(w, torch), _stream_solver(w, torch)
    x0 = np.asarray(w.source_xyz, dtype=float)
    sources = [tuple(x0 + np.array([dx, 0.0, 0.0])) for dx in (0.0, 20.0, -30.0, 35.0)]
    alone = [s1.rtm_shot(src, w.f0, w.t_peak, 1.0, w.receivers, w.t_final) for src in sources]
    with ridg.Server([s1, s2], max_queued=8) as sv:
        tickets = [sv.submit(src, w.f0, w.t_peak, 1.0, w.receivers, w.t_final) for src in sources]
        served = [sv.wait(t, timeout=300) for t in tickets]
    for (tr, ip, iq), (tr2, ip2, iq2, tm) in zip(alone, served):
        assert np.array_equal(tr, tr2) and np.array_equal(ip, ip2) and np.array_equal(iq, iq2)
    tms = [x[3] for x in served]
    assert {tm["slot"] for tm in tms} == {0, 1}
    a, b = tms[0], tms[1]  # the first two requests ran on different slots at the same time
    assert a["slot"] != b["slot"] and a["start_s"] < b["end_s"] and b["start_s"] < a["end_s"]


def test_slots_of_two_models():
    """Requests go to the slots of their own model (different meshes and orders)."""
    torch = pytest.importorskip("torch")
    w3 = tiny_layered_rtm(N=3, t_final=0.004)
    w2 = tiny_layered_rtm(N=2, t_final=0.004)
    s3, s2 = _stream_solver(w3, torch), _stream_solver(w2, torch)
    a3 = s3.rtm_shot(w3.source_xyz, w3.f0, w3.t_peak, 1.0, w3.receivers, w3.t_final)
    a2 = s2.rtm_shot(w2.source_xyz, w2.f0, w2.t_peak, 1.0, w2.receivers, w2.t_final)
    with ridg.Server([s3, s2], max_queued=8, models=[0, 1]) as sv:
        t = [sv.submit(w2.source_xyz, w2.f0, w2.t_peak, 1.0, w2.receivers, w2.t_final, model=1),
             sv.submit(w3.source_xyz, w3.f0, w3.t_peak, 1.0, w3.receivers, w3.t_final, model=0),
             sv.submit(w2.source_xyz, w2.f0, w2.t_peak, 1.0, w2.receivers, w2.t_final, model=1)]
        r = [sv.wait(x, timeout=300) for x in t]
        with pytest.raises(ValueError):
            sv.submit(w2.source_xyz, w2.f0, w2.t_peak, 1.0, w2.receivers, w2.t_final, model=2)
    assert [x[3]["slot"] for x in r] == [1, 0, 1]
    for got, ref in zip(r, [a2, a3, a2]):
        assert all(np.array_equal(g, e) for g, e in zip(got[:3], ref))
    with pytest.raises(ridg.RidgError) as e:
        ridg.Server([s3, s2], models=[0, 0])  # different orders under one model number
    assert e.value.code == -1


def test_admission_by_device_memory():
    """A request whose boundary-trace arena cannot fit in device memory completes with RIDG_E_OOM
    after the idle slots have given back their buffers; the server then serves the next request."""
    torch = pytest.importorskip("torch")
    w = tiny_layered_rtm(N=3, t_final=0.004)
    s1, s2 = _stream_solver(w, torch), _stream_solver(w, torch)
    rec = w.receivers[:1]
    with ridg.Server([s1, s2], max_queued=4) as sv:
        sv.wait(sv.submit(w.source_xyz, w.f0, w.t_peak, 1.0, rec, w.t_final), timeout=300)
        # about 1e8 fine steps of boundary records: far more than the device holds
        big = sv.submit(w.source_xyz, w.f0, w.t_peak, 1.0, rec, 2000.0, want_images=False)
        with pytest.raises(ridg.RidgError) as e:
            sv.wait(big, timeout=600)
        assert e.value.code == -3
        tr, ip, iq, _ = sv.wait(sv.submit(w.source_xyz, w.f0, w.t_peak, 1.0, rec, w.t_final), timeout=300)
        assert np.isfinite(tr).all() and np.abs(ip).max() > 0
