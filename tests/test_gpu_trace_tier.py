"""Boundary-trace records beyond a device budget (ridg_set_trace_budget; Sec. 4.3 moves the records
from the device to host memory): the records of consecutive fine steps go to pinned host memory in
chunks of half the budget during the forward run and come back, one chunk ahead, in reverse order
during the backward run.

* Every budget (three chunks, several, and the smallest allowed, about one fine step per chunk) gives
  the shot with every record on the device bit for bit, in FP64 and FP32, on a three-level mesh and
  on the box with isolated fast inclusions; the stats count the chunks (at least three: two chunks
  of half the budget would hold every record) and the bytes that went to host memory (all but the
  last two chunks, which never leave the device).
* An image window that ends the backward run early, and a second shot with another source that
  reuses the host memory, match their all-device shots as well.
* A budget below twice one fine step's records, or negative, is refused; the solver stays usable."""

import numpy as np
import pytest

from paper_1506_00907_gb300 import ridg
from synth import inclusion_box, tiny_layered_rtm

pytestmark = pytest.mark.gpu


def _case(name, dtype):
    w = inclusion_box() if name == "inclusions" else tiny_layered_rtm(N=3, t_final=0.003)
    mesh = ridg.Mesh(w.xyz, w.tets, default_bc=w.default_bc)
    s = ridg.Solver(mesh, w.N, w.c, w.rho, dtype=dtype, cfl=w.cfl, n_levels_max=w.n_levels_max)
    return w, s


def _record_bytes(s, dtype):
    nfpp = 16 if (s.info.N + 1) * (s.info.N + 2) // 2 <= 16 else 32
    return 2 * nfpp * (8 if dtype == "f64" else 4)


def _same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("name", ["tiny", "inclusions"])
def test_tiered_records_give_the_all_device_shot(name, dtype):
    w, s = _case(name, dtype)
    args = (w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final)
    ref = s.rtm_shot(*args)
    st = s.shot_stats()
    full = st.boundary_trace_bytes
    assert st.trace_chunks == 1 and st.host_trace_bytes == 0
    assert np.abs(ref[0]).max() > 0 and np.abs(ref[1]).max() > 0
    # the step that advances every level records every boundary face
    smallest = 2 * s.info.n_boundary_faces * _record_bytes(s, dtype)
    seen = []
    for budget in (int(0.8 * full), int(0.2 * full), smallest):
        budget = max(budget, smallest)
        s.set_trace_budget(budget)
        out = s.rtm_shot(*args)
        st = s.shot_stats()
        assert _same(out, ref), budget
        assert st.boundary_trace_bytes == full and st.trace_chunks >= 3
        assert 0 < st.host_trace_bytes < full
        seen.append(int(st.trace_chunks))
    assert 3 <= seen[0] <= seen[1] <= seen[2] and seen[2] > seen[0]
    s.set_trace_budget(full)  # a budget that holds every record: no tier
    assert _same(s.rtm_shot(*args), ref) and s.shot_stats().trace_chunks == 1
    s.close()


def test_tiered_records_with_window_and_second_shot():
    dtype = "f32"
    w, s = _case("tiny", dtype)
    t_img = 0.5 * w.t_final
    other = (w.source_xyz[0] + 30.0, w.source_xyz[1], w.source_xyz[2])
    ref_win = s.rtm_shot(w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final, t_image_start=t_img)
    ref_other = s.rtm_shot(other, w.f0, w.t_peak, 1.0, w.receivers, w.t_final)
    full = s.shot_stats().boundary_trace_bytes
    s.set_trace_budget(max(int(0.1 * full), 2 * s.info.n_boundary_faces * _record_bytes(s, dtype)))
    out = s.rtm_shot(w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final, t_image_start=t_img)
    assert s.shot_stats().trace_chunks > 2
    assert _same(out, ref_win)
    assert _same(s.rtm_shot(other, w.f0, w.t_peak, 1.0, w.receivers, w.t_final), ref_other)
    s.close()


def test_budget_below_one_step_is_refused():
    dtype = "f64"
    w, s = _case("tiny", dtype)
    args = (w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final)
    ref = s.rtm_shot(*args)
    smallest = 2 * s.info.n_boundary_faces * _record_bytes(s, dtype)
    s.set_trace_budget(smallest - 1)
    with pytest.raises(ridg.RidgError):
        s.rtm_shot(*args)
    with pytest.raises(ridg.RidgError):
        s.set_trace_budget(-1)
    s.set_trace_budget(0)
    assert _same(s.rtm_shot(*args), ref)
    s.close()
