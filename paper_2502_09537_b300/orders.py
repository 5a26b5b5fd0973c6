"""Update orders of the grid points for DP-AVF2 (Sec. 3 of arXiv 2502.09537).

Every order of the points defines a DP-AVF scheme (Eqs. LapP, order1, order2):
in a point's update the neighbours that come earlier enter at the new level.
An order here is a permutation of the linear indices 0 .. N^d - 1 of the grid
(C order, last axis fastest), as ``Solver.set_order`` and the oracle take it;
the base half visits the points in the order, the adjoint half in reverse.
"""
from __future__ import annotations

from typing import List

import numpy as np


def lexicographic(dim: int, N: int) -> np.ndarray:
    """Eq. order1 generalised: increasing linear index, i.e. every point after
    its lower neighbours along each axis (S = W = 1, E = N = 0 in 2D)."""
    return np.arange(N ** dim, dtype=np.int64)


def reverse_lexicographic(dim: int, N: int) -> np.ndarray:
    """Eq. order2: decreasing linear index (S = W = 0, E = N = 1 in 2D)."""
    return np.arange(N ** dim, dtype=np.int64)[::-1].copy()


def checkerboard(dim: int, N: int, red_first: bool = True) -> np.ndarray:
    """Algorithm 3's order: one colour's points (in increasing index), then the
    other's.  A point is red when its 1-based index sum is odd."""
    idx = np.indices((N,) * dim).reshape(dim, -1)
    red = ((idx.sum(axis=0) + dim) & 1) == 1
    first = red if red_first else ~red
    lin = np.arange(N ** dim, dtype=np.int64)
    return np.concatenate([lin[first], lin[~first]])


def block_split_2d(N: int, nblocks: int) -> np.ndarray:
    """Algorithm 2's order on an N x N grid (the paper's CPU-parallel split):
    the boundary row j_0 = 0, then blocks of rows separated by single rows
    j_1 < ... < j_nblocks = N - 1, each block's rows in increasing j and each
    row in increasing k, and finally the separator rows j_1 .. j_nblocks.
    Blocks are as equal as possible.  Rows are the first axis (the paper's j),
    so blocks are independent of one another: no point of one block
    neighbours a point of another."""
    inner = N - 1 - nblocks  # rows outside j_0 and the separators
    if nblocks < 1 or inner < nblocks:
        raise ValueError("need at least one row per block: N >= 2 nblocks + 1")
    sizes = [inner // nblocks + (1 if b < inner % nblocks else 0) for b in range(nblocks)]
    seps: List[int] = []
    blocks: List[List[int]] = []
    j = 1
    for b in range(nblocks):
        blocks.append(list(range(j, j + sizes[b])))
        j += sizes[b]
        seps.append(j)
        j += 1
    assert seps[-1] == N - 1
    rows = [0] + [r for blk in blocks for r in blk] + seps
    k = np.arange(N, dtype=np.int64)
    return np.concatenate([r * N + k for r in rows])


def random_order(dim: int, N: int, seed: int) -> np.ndarray:
    """A seeded uniformly random permutation (any order is a valid scheme)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.permutation(N ** dim).astype(np.int64)
