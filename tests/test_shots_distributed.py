"""Shot-parallel host logic on CPU ranks (gloo, world size 2): shot partition and image reduction."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1506_00907_gb300.shots import reduce_images, shots_of_rank


def test_shot_partition_covers_every_shot_once():
    for n, world in ((29, 2), (29, 4), (3, 8), (0, 2)):
        got = sorted(i for r in range(world) for i in shots_of_rank(n, r, world))
        assert got == list(range(n))
    with pytest.raises(ValueError):
        shots_of_rank(3, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(100 + rank)
        img_p = torch.tensor(rng.standard_normal((7, 5)))
        img_q = torch.tensor(rng.standard_normal((7, 5)))
        reduce_images([img_p, img_q])
        out[rank] = (img_p.numpy().copy(), img_q.numpy().copy())
    finally:
        dist.destroy_process_group()


def test_image_reduction_two_ranks():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
    exp_p = sum(np.random.default_rng(100 + r).standard_normal((7, 5)) for r in range(world))
    rngs = [np.random.default_rng(100 + r) for r in range(world)]
    exp_q = 0
    for g in rngs:
        g.standard_normal((7, 5))
        exp_q = exp_q + g.standard_normal((7, 5))
    for r in range(world):
        p, q = out[r]
        assert np.allclose(p, exp_p) and np.allclose(q, exp_q)
