"""Environment switches read when a solver is created.

* RIDG_DEBUG=1 checks the solver's tables on the host before they are uploaded (indices in range,
  symmetric connectivity, inverse slot maps, boundary-face numbering, face-node permutations): the
  check passes on single-level, multi-level and partitioned meshes, and the shot is unchanged.
* RIDG_PROFILE=<every> turns on the CUDA-event profiling of ridg_set_profiling."""

import numpy as np
import pytest

from oracle.partition import partition
from oracle.rtm import make_problem
from paper_1506_00907_gb300 import ridg
from synth import inclusion_box, tiny_layered_rtm

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["tiny", "inclusions"])
def test_debug_table_checks_pass_and_change_nothing(name, monkeypatch):
    w = inclusion_box() if name == "inclusions" else tiny_layered_rtm(N=3, t_final=0.002)
    mesh = ridg.Mesh(w.xyz, w.tets, default_bc=w.default_bc)
    args = (w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final)
    kw = dict(dtype="f32", cfl=w.cfl, n_levels_max=w.n_levels_max)
    ref = ridg.Solver(mesh, w.N, w.c, w.rho, **kw).rtm_shot(*args)
    monkeypatch.setenv("RIDG_DEBUG", "1")
    out = ridg.Solver(mesh, w.N, w.c, w.rho, **kw).rtm_shot(*args)
    assert all(np.array_equal(a, b) for a, b in zip(out, ref))
    # parts with ghost slots
    prob = make_problem(w.xyz, w.tets, w.c, w.rho, w.N, default_bc=w.default_bc, cfl=w.cfl,
                        n_levels_max=w.n_levels_max)
    part = partition(prob.geo, prob.levels, prob.n_levels, 3)
    g = ridg.Group(mesh, w.N, w.c, w.rho, part, **kw)
    assert all(np.array_equal(a, b) for a, b in zip(g.rtm_shot(*args), ref))


def test_profile_switch_turns_on_event_timing(monkeypatch):
    w = tiny_layered_rtm(N=3, t_final=0.002)
    mesh = ridg.Mesh(w.xyz, w.tets, default_bc=w.default_bc)
    args = (w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final)
    s = ridg.Solver(mesh, w.N, w.c, w.rho, dtype="f32", cfl=w.cfl, n_levels_max=w.n_levels_max)
    s.rtm_shot(*args)
    assert s.shot_stats().prof_forward_launches == 0
    monkeypatch.setenv("RIDG_PROFILE", "1")
    s = ridg.Solver(mesh, w.N, w.c, w.rho, dtype="f32", cfl=w.cfl, n_levels_max=w.n_levels_max)
    s.rtm_shot(*args)
    st = s.shot_stats()
    assert st.prof_forward_launches > 0 and st.prof_backward_launches > 0
    assert st.prof_forward_ms > 0 and st.prof_backward_ms > 0
