"""Failure detection by host-side fault injection (no GPU fault): each failure point fires once
through the error path of the failure it stands for, the call reports its status, and the solver,
server or part group works afterwards with the results of an undisturbed run.

* a device allocation while a solver is created: RIDG_E_OOM;
* the boundary-trace arena of a shot: RIDG_E_OOM;
* the shot server's memory admission: the request completes with RIDG_E_OOM, the next one is served;
* a part group's interface transfer: RIDG_E_CUDA, every other part's thread released (no host wait
  is left hanging)."""

import numpy as np
import pytest

from oracle.partition import partition
from oracle.rtm import make_problem
from paper_1506_00907_gb300 import ridg
from synth import inclusion_box, tiny_layered_rtm

pytestmark = pytest.mark.gpu

OOM, CUDA = -3, -4


def _tiny():
    w = tiny_layered_rtm(N=3, t_final=0.002)
    return w, ridg.Mesh(w.xyz, w.tets, default_bc=w.default_bc)


def _solver(w, mesh, **kw):
    return ridg.Solver(mesh, w.N, w.c, w.rho, dtype="f32", cfl=w.cfl, n_levels_max=w.n_levels_max, **kw)


@pytest.fixture(autouse=True)
def _disarm():
    ridg.inject_fault("none")
    yield
    ridg.inject_fault("none")


def test_allocation_failure_while_creating_a_solver():
    w, mesh = _tiny()
    ridg.inject_fault("alloc", 2)
    with pytest.raises(ridg.RidgError) as e:
        _solver(w, mesh)
    assert e.value.code == OOM and "injected" in str(e.value)
    assert ridg.fault_armed() == 0
    args = (w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final)
    a = _solver(w, mesh).rtm_shot(*args)
    b = _solver(w, mesh).rtm_shot(*args)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))


def test_arena_failure_during_a_shot():
    w, mesh = _tiny()
    s, ref = _solver(w, mesh), _solver(w, mesh)
    args = (w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final)
    ridg.inject_fault("arena")
    with pytest.raises(ridg.RidgError) as e:
        s.rtm_shot(*args)
    assert e.value.code == OOM
    tr, ip, iq = s.rtm_shot(*args)
    tr0, ip0, iq0 = ref.rtm_shot(*args)
    assert np.array_equal(tr, tr0) and np.array_equal(ip, ip0) and np.array_equal(iq, iq0)


def test_admission_refusal_in_the_shot_server():
    w, mesh = _tiny()
    s, ref = _solver(w, mesh), _solver(w, mesh)
    args = (w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final)
    tr0, ip0, iq0 = ref.rtm_shot(*args)
    with ridg.Server([s], max_queued=4) as sv:
        ridg.inject_fault("admission")
        t = sv.submit(*args)
        with pytest.raises(ridg.RidgError) as e:
            sv.wait(t)
        assert e.value.code == OOM
        tr, ip, iq, _ = sv.wait(sv.submit(*args))
    assert np.array_equal(tr, tr0) and np.array_equal(ip, ip0) and np.array_equal(iq, iq0)


@pytest.mark.timeout(600)
def test_interface_transfer_failure_in_a_part_group():
    w = inclusion_box()
    prob = make_problem(w.xyz, w.tets, w.c, w.rho, w.N, default_bc=w.default_bc, cfl=w.cfl,
                        n_levels_max=w.n_levels_max)
    mesh = ridg.Mesh(w.xyz, w.tets, default_bc=w.default_bc)
    part = partition(prob.geo, prob.levels, prob.n_levels, 3)
    g = ridg.Group(mesh, w.N, w.c, w.rho, part, cfl=w.cfl, n_levels_max=w.n_levels_max)
    args = (w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final)
    ridg.inject_fault("exchange", 7)
    with pytest.raises(ridg.RidgError) as e:
        g.rtm_shot(*args)
    assert e.value.code == CUDA and "injected" in str(e.value)
    tr, ip, iq = g.rtm_shot(*args)
    tr0, ip0, iq0 = ridg.Solver(mesh, w.N, w.c, w.rho, cfl=w.cfl, n_levels_max=w.n_levels_max).rtm_shot(*args)
    assert np.array_equal(tr, tr0) and np.array_equal(ip, ip0) and np.array_equal(iq, iq0)
