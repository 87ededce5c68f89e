"""Partition of one enclosure across ranks (one GPU each), with no exchange of data.

The boxes of the finest grid that Algorithm 3 returns do not depend on the order in which
coarser boxes were pruned: interval Horner with outward rounding is inclusion-isotone and
the grid is exact, so a box of level L survives iff it passes C0 at level L and at each of its
ancestors, and every ancestor of a passing box passes.  Splitting the domain along x_1 into N
(a power of two) equal slabs and enclosing slab r at depth L - log2(N) therefore gives exactly
the level-L survivors whose x_1 index lies in [r 2^(L - log2 N), (r+1) 2^(L - log2 N)); the
slabs concatenated in rank order are the single-GPU result in lexicographic order.  Only the
coarsest log2(N) levels, where each rank holds one slab, are not evaluated.
"""
from __future__ import annotations

import numpy as np


def log2_exact(n: int) -> int:
    if n < 1 or n & (n - 1):
        raise ValueError("the number of ranks must be a power of two, got %d" % n)
    return n.bit_length() - 1


def rank_problem(domain, depth: int, rank: int, world: int):
    """(sub-domain, sub-depth, x_1 index offset) of rank ``rank`` out of ``world``."""
    s = log2_exact(world)
    if s > depth:
        raise ValueError("%d ranks need depth >= %d" % (world, s))
    dom = np.asarray(domain, dtype=np.float64).reshape(-1).copy()
    lo, hi = dom[0], dom[1]
    w = (hi - lo) / world  # exact on dyadic domains (division by a power of two)
    dom[0] = lo + rank * w
    dom[1] = lo + (rank + 1) * w
    return dom, depth - s, rank << (depth - s)


def to_global(tuples: np.ndarray, offset: int) -> np.ndarray:
    out = np.array(tuples, dtype=np.int32, copy=True)
    if out.size:
        out[:, 0] += offset
    return out
