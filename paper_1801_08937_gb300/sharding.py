"""Host-side partitioning of one map-making problem over several ranks.

W is block diagonal over stationary (detector, interval) blocks, so
A = P^T W P is a sum of per-block terms: rank r can own a contiguous range
of whole blocks and compute its partial P_r^T W_r P_r x with no halo
exchange; one sum over ranks of the n = 3 n_pix map values completes A x.
Maps, M_BD blocks (also sums over blocks), Z and AZ are replicated, so the
PCG inner products stay local.  Independent problems (the paper's
divide-and-conquer of data subsets) need no exchange at all and run as
replicas.
"""
from __future__ import annotations

import numpy as np


def partition_blocks(block_off, world: int):
    """Contiguous block ranges [b0, b1) per rank with balanced sample counts."""
    block_off = np.asarray(block_off, dtype=np.int64)
    n_blocks = block_off.shape[0] - 1
    if world < 1:
        raise ValueError("world must be >= 1")
    total = int(block_off[-1])
    cuts = [0]
    for r in range(1, world):
        target = total * r / world
        b = int(np.searchsorted(block_off, target, side="left"))
        b = min(max(b, cuts[-1]), n_blocks)
        cuts.append(b)
    cuts.append(n_blocks)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def shard(pix, psi, block_off, block_band, b0: int, b1: int):
    """Pointing arrays and block table of blocks [b0, b1), offsets rebased to 0."""
    block_off = np.asarray(block_off, dtype=np.int64)
    t0, t1 = int(block_off[b0]), int(block_off[b1])
    return (np.asarray(pix)[t0:t1], np.asarray(psi)[t0:t1], block_off[b0:b1 + 1] - t0,
            np.asarray(block_band)[b0:b1], (t0, t1))


def max_over_ranks(value: float, dist=None) -> float:
    """Largest value over the ranks of a torch.distributed group (the value itself when alone)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64)
    if dist.get_backend() == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
