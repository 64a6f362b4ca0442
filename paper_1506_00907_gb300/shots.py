"""Shot-parallel execution across GPUs (one process per GPU).

Shots of a survey are independent (the image is the sum over shots of Eqs. imageP/imageQ), so
the natural multi-GPU form is one shot per rank at a time and one reduction of the images: no
data-path exchange happens while a shot runs.
"""

from __future__ import annotations


def shots_of_rank(n_shots: int, rank: int, world: int):
    """Indices of the shots rank `rank` of `world` migrates (round robin)."""
    if world < 1 or not (0 <= rank < world) or n_shots < 0:
        raise ValueError("bad shot partition")
    return list(range(rank, n_shots, world))


def reduce_images(images, group=None):
    """Sum per-rank images in place over the process group (torch.distributed all-reduce).

    `images` is an iterable of tensors of identical shape on every rank (FP64 images on the GPU
    with NCCL, or CPU tensors with gloo)."""
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized():
        return images
    for img in images:
        dist.all_reduce(img, op=dist.ReduceOp.SUM, group=group)
    return images
