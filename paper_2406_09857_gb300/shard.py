"""Partition of one enclosure across ranks (one GPU each), with no exchange of data.

The boxes of the finest grid that Algorithm 3 returns do not depend on how coarser boxes were
pruned: interval Horner with outward rounding is inclusion-isotone and the grid is exact, so a
box of level L passes C0 only if each of its ancestors does, and the survivors of level L are
exactly the level-L boxes that pass.  With N = 2^s ranks, rank r therefore starts Algorithm 3
at level s from every box of that level whose x_1 index is r (an x_1-slab of the domain, all
other indices free) and runs it to depth L on the full grid; its survivors are the single-GPU
survivors with x_1 index in [r 2^(L-s), (r+1) 2^(L-s)), and the ranks' results concatenated in
rank order are the single-GPU result in lexicographic order.  Levels below s are skipped and
level s is evaluated unpruned, which changes the work but not the result.
"""
from __future__ import annotations

import numpy as np


def log2_exact(n: int) -> int:
    if n < 1 or n & (n - 1):
        raise ValueError("the number of ranks must be a power of two, got %d" % n)
    return n.bit_length() - 1


def rank_start(k: int, depth: int, rank: int, world: int):
    """(start level s, int32 [2^(s(k-1)), k] lex-sorted boxes of level s with x_1 index = rank)."""
    s = log2_exact(world)
    if s > depth:
        raise ValueError("%d ranks need depth >= %d" % (world, s))
    if not 0 <= rank < world:
        raise ValueError("rank %d outside [0, %d)" % (rank, world))
    side = 1 << s
    rest = np.stack(np.meshgrid(*[np.arange(side, dtype=np.int32)] * (k - 1), indexing="ij"),
                    axis=-1).reshape(-1, k - 1) if k > 1 else np.zeros((1, 0), dtype=np.int32)
    t = np.empty((rest.shape[0], k), dtype=np.int32)
    t[:, 0] = rank
    t[:, 1:] = rest
    return s, t
