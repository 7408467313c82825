"""Multi-process helpers: one process per GPU, torch.distributed underneath.

The rasterizer partitions by camera: each camera's forward and backward are
independent of the others, and the only exchange a multi-GPU optimisation
step needs is the sum over ranks of the per-primitive gradients (one
all-reduce per step, after the render backward and before the parameter
update).  Primitives cannot be split spatially, since compositing needs one
global depth order per pixel.

These helpers are backend-agnostic (NCCL for device tensors, gloo for host
tensors) and contain no rendering arithmetic.
"""
from __future__ import annotations

from typing import Dict, List, Sequence


def _dist():
    import torch.distributed as dist
    return dist


def world() -> int:
    dist = _dist()
    return dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1


def rank() -> int:
    dist = _dist()
    return dist.get_rank() if dist.is_available() and dist.is_initialized() else 0


def balanced_shards(cameras: Sequence, n_ranks: int) -> List[List[int]]:
    """Camera indices per rank, balancing pixel counts: cameras in
    descending pixel count go to the rank with the fewest pixels so far
    (ties to the lower rank).  Every camera lands on exactly one rank."""
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    order = sorted(range(len(cameras)), key=lambda i: (-cameras[i].width * cameras[i].height, i))
    load = [0] * n_ranks
    shards: List[List[int]] = [[] for _ in range(n_ranks)]
    for i in order:
        r = min(range(n_ranks), key=lambda k: (load[k], k))
        shards[r].append(i)
        load[r] += cameras[i].width * cameras[i].height
    return [sorted(s) for s in shards]


def my_cameras(cameras: Sequence, r: int = None, n: int = None) -> List:
    r = rank() if r is None else r
    n = world() if n is None else n
    return [cameras[i] for i in balanced_shards(cameras, n)[r]]


def allreduce_gradients(grads: Dict[str, "object"], group=None) -> Dict[str, "object"]:
    """Sum every gradient tensor over ranks, in place, in sorted key order
    (so all ranks issue the same collectives)."""
    dist = _dist()
    if world() == 1:
        return grads
    for k in sorted(grads):
        dist.all_reduce(grads[k], op=dist.ReduceOp.SUM, group=group)
    return grads


def max_over_ranks(x: float, device=None) -> float:
    import torch
    dist = _dist()
    if world() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device=None) -> float:
    import torch
    dist = _dist()
    if world() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier():
    if world() > 1:
        _dist().barrier()
