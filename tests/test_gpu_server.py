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
