"""Domain decomposition (Sec. 4.2) on CPU ranks: the partitioned oracle against the unpartitioned one.

* The partition balances the weights 2^(l-1) and keeps every element of the finest level, with its
  face neighbours, inside one part (lumping).
* Two gloo ranks each run a whole RTM shot (forward with recording, overshoot, backward source and
  receiver runs with both images) on their own part of a three-level mesh, exchanging interface
  traces at the end of every fine step except those that update the finest level only; the union of
  their fields, traces and images equals the unpartitioned oracle's bit for bit.
* Shot-parallel flow: each rank migrates its own shots with the oracle standing in for the library,
  and the image all-reduce gives the sum of the shots."""

import functools
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle.partition import PartMRAB, element_weights, partition
from oracle.rtm import make_problem, rtm_shot
from paper_1506_00907_gb300.shots import reduce_images, shots_of_rank
from synth import inclusion_box, tiny_layered_rtm


def _problem(name="inclusions"):
    """The 648-element box whose few finest elements are isolated (as in the paper's survey), or the
    tiny layered mesh whose finest level is most of the mesh (its lumps are too heavy to keep whole,
    so finest elements lie at the interface)."""
    w = inclusion_box() if name == "inclusions" else tiny_layered_rtm(N=2, t_final=0.002)
    return w, make_problem(w.xyz, w.tets, w.c, w.rho, w.N, default_bc=w.default_bc, cfl=w.cfl,
                           n_levels_max=w.n_levels_max)


def test_partition_balances_weights_and_keeps_finest_lumps_inside():
    w, prob = _problem()
    g, lev, L = prob.geo, prob.levels, prob.n_levels
    assert L == 3 and np.sum(lev == L) < 0.01 * w.K
    wt = element_weights(lev)
    for n_parts in (2, 3, 4):
        part = partition(g, lev, L, n_parts)
        assert set(np.unique(part)) == set(range(n_parts))
        loads = np.bincount(part, weights=wt, minlength=n_parts)
        # balanced within a few per cent (lumps of a finest element and its neighbours stay whole)
        assert loads.max() - loads.min() <= 0.03 * loads.sum(), loads
        for k in np.nonzero(lev == L)[0]:
            for k2 in g.nbr[k]:
                assert k2 < 0 or part[k2] == part[k]
    # a finest level that is most of the mesh: its lump is not kept whole, the weights still balance
    w, prob = _problem("tiny")
    part = partition(prob.geo, prob.levels, prob.n_levels, 4)
    loads = np.bincount(part, weights=element_weights(prob.levels))
    assert loads.max() < 1.1 * loads.mean()


class GlooComm:
    """Array transfers between ranks with torch.distributed point-to-point calls (gloo)."""

    def exchange(self, sends, recv_shapes):
        reqs, got = [], {}
        for r in sorted(recv_shapes):
            t = torch.empty(recv_shapes[r], dtype=torch.float64)
            reqs.append(dist.irecv(t, src=r))
            got[r] = t
        for r in sorted(sends):
            reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(sends[r])), dst=r))
        for q in reqs:
            q.wait()
        return {r: t.numpy() for r, t in got.items()}


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _part_worker(rank, world, port, name, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, prob = _problem(name)
        part = partition(prob.geo, prob.levels, prob.n_levels, world)
        steppers = []

        def stepper(*a, **k):
            s = PartMRAB(*a, **k, part=part, rank=rank, comm=GlooComm())
            steppers.append(s)
            return s

        res = rtm_shot(prob, w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final, stepper=stepper)
        out[rank] = {"part": part, "traces": res.traces, "image_p": res.image_p, "image_q": res.image_q,
                     "q_final": res.q_final, "q_back": res.q_source_back, "dof": res.dof_updates,
                     "messages": sum(s.messages for s in steppers), "silent": sum(s.silent_steps for s in steppers)}
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name", ["inclusions", "tiny"])
def test_partitioned_shot_equals_unpartitioned_two_ranks(name):
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_part_worker, args=(world, _free_port(), name, out), nprocs=world, start_method="spawn")
    w, prob = _problem(name)
    ref = rtm_shot(prob, w.source_xyz, w.f0, w.t_peak, 1.0, w.receivers, w.t_final)
    part = out[0]["part"]
    assert np.array_equal(part, out[1]["part"])
    rec_owner = np.array([part[prob.geo.locate(x)[0]] for x in w.receivers])
    traces = np.zeros_like(ref.traces)
    img_p, img_q = np.zeros_like(ref.image_p), np.zeros_like(ref.image_q)
    q_final, q_back = np.zeros_like(ref.q_final), np.zeros_like(ref.q_source_back)
    for r in range(world):
        o, own = out[r], part == r
        traces[rec_owner == r] = o["traces"][rec_owner == r]
        img_p[own], img_q[own] = o["image_p"][own], o["image_q"][own]
        q_final[own], q_back[own] = o["q_final"][own], o["q_back"][own]
        assert np.all(o["image_p"][~own] == 0.0)  # a part images only its own elements
        assert o["messages"] > 0
        # finest-only steps transfer nothing exactly when lumping kept the finest elements inside
        assert (o["silent"] > 0) == (name == "inclusions")
    assert np.abs(ref.image_p).max() > 0 and np.abs(ref.traces).max() > 0
    for a, b in ((traces, ref.traces), (img_p, ref.image_p), (img_q, ref.image_q), (q_final, ref.q_final),
                 (q_back, ref.q_source_back)):
        assert np.array_equal(a, b)
    assert out[0]["dof"] + out[1]["dof"] == ref.dof_updates


@functools.lru_cache(maxsize=None)
def _shot_images(i):
    w, prob = _problem("tiny")
    x = (w.source_xyz[0] + 20.0 * (i - 1), w.source_xyz[1], w.source_xyz[2])
    res = rtm_shot(prob, x, w.f0, w.t_peak, 1.0, w.receivers, 0.001)
    return res.image_p, res.image_q


def _shots_worker(rank, world, port, n_shots, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        img_p = torch.zeros(_shot_images(0)[0].shape, dtype=torch.float64)
        img_q = torch.zeros_like(img_p)
        for i in shots_of_rank(n_shots, rank, world):
            p, q = _shot_images(i)
            img_p += torch.from_numpy(p)
            img_q += torch.from_numpy(q)
        reduce_images([img_p, img_q])
        out[rank] = (img_p.numpy().copy(), img_q.numpy().copy())
    finally:
        dist.destroy_process_group()


def test_shot_parallel_images_are_the_sum_of_the_shots_two_ranks():
    world, n_shots = 2, 3
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_shots_worker, args=(world, _free_port(), n_shots, out), nprocs=world, start_method="spawn")
    exp_p = sum(_shot_images(i)[0] for i in range(n_shots))
    exp_q = sum(_shot_images(i)[1] for i in range(n_shots))
    for r in range(world):
        p, q = out[r]
        assert np.allclose(p, exp_p, rtol=1e-13, atol=0) and np.allclose(q, exp_q, rtol=1e-13, atol=0)
        assert np.abs(p).max() > 0


def test_library_partition_equals_the_oracle_partition():
    """ridg_partition (host code of the library, its own implementation) gives the oracle's parts."""
    from paper_1506_00907_gb300 import ridg

    for name in ("inclusions", "tiny"):
        w, prob = _problem(name)
        m = ridg.Mesh(w.xyz, w.tets, default_bc=w.default_bc)
        for n_parts in (1, 2, 3, 4, 7):
            lib_part = ridg.partition(m, w.N, w.c, n_parts, cfl=w.cfl, n_levels_max=w.n_levels_max)
            assert np.array_equal(lib_part, partition(prob.geo, prob.levels, prob.n_levels, n_parts))
    with pytest.raises(ridg.RidgError):
        ridg.partition(m, w.N, w.c, 0)
