"""Work split across GPUs (one process per GPU).

Every row of a batch is an independent DFT (Eq. (1) per row), so a multi-GPU
run gives each rank a disjoint share of the rows and needs no collective on the
data path.  A uniform batch is split into contiguous blocks; a ragged batch is
balanced by the work of each transform, taken as N log2 N (the Cooley-Tukey
operation count, Section IV), with a deterministic longest-first greedy
assignment.  The only cross-rank operation is the timing reduction of the
benchmark (the maximum over ranks).
"""
from __future__ import annotations

import math

import numpy as np


def shard_uniform(batch: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous block (start, count) of `batch` rows for `rank` of `world`;
    counts differ by at most one."""
    if world < 1 or not 0 <= rank < world or batch < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(batch, world)
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


def transform_cost(n: int) -> float:
    return float(n) * max(1.0, math.log2(n))


def shard_ragged(lengths, world: int) -> list[np.ndarray]:
    """Indices of the transforms of every rank: longest first, each to the
    currently least-loaded rank (ties to the lowest rank).  Every index appears
    exactly once; each rank's indices are returned in increasing order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    lengths = np.asarray(lengths, dtype=np.int64)
    order = sorted(range(lengths.size), key=lambda t: (-int(lengths[t]), t))
    load = [0.0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for t in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(t)
        load[r] += transform_cost(int(lengths[t]))
    return [np.array(sorted(p), dtype=np.int64) for p in parts]


def max_over_ranks(value: float, dist=None) -> float:
    """The maximum of `value` over all ranks of the default process group
    (the value itself without one).  Works on any backend: the tensor lives on
    the backend's device (CUDA for NCCL, CPU for gloo)."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(value)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
