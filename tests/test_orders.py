"""Update orders (Sec. 3, Eqs. LapP/order1/order2; Algorithms 1-3): the level
schedule the library derives from an order, checked on the host, and the
fact it rests on, checked on the oracle.

The GPU runs an order as levels: a point's level is one more than the largest
level of its neighbours that precede it in the order.  Two facts make that
exact: (1) points of one level are never neighbours, and (2) the serial
DP-AVF2 result depends on the order only through which neighbour of each
point comes first -- so any order with the same levels, in particular the
level-sorted one, gives bitwise the same serial result.  (2) is checked on
the oracle itself, independently of the GPU path.
"""
import numpy as np
import pytest

from paper_2502_09537_b300 import orders
from paper_2502_09537_b300.inputs import Problem, random_state
from paper_2502_09537_b300.solver import KGSError, order_schedule


def _neighbours(dim, N, p):
    c = np.unravel_index(p, (N,) * dim)
    out = []
    for a in range(dim):
        for dlt in (-1, 1):
            q = list(c)
            q[a] = (q[a] + dlt) % N
            out.append(int(np.ravel_multi_index(q, (N,) * dim)))
    return out


def _levels_brute(dim, N, order):
    pos = np.empty(N ** dim, dtype=np.int64)
    pos[order] = np.arange(N ** dim)
    lv = np.zeros(N ** dim, dtype=np.int64)
    for t, p in enumerate(order.tolist()):
        earlier = [lv[q] + 1 for q in _neighbours(dim, N, p) if pos[q] < t]
        lv[p] = max(earlier, default=0)
    return lv


@pytest.mark.parametrize("dim,N", [(1, 10), (2, 6), (2, 8), (3, 4)])
def test_lexicographic_levels_are_the_index_sums(dim, N):
    lv, n = order_schedule(dim, N, orders.lexicographic(dim, N))
    assert n == 1 + dim * (N - 1)
    assert np.array_equal(lv, np.indices((N,) * dim).sum(axis=0))


@pytest.mark.parametrize("dim,N", [(1, 8), (2, 6), (3, 4)])
def test_checkerboard_has_two_levels_red_first(dim, N):
    lv, n = order_schedule(dim, N, orders.checkerboard(dim, N))
    assert n == 2
    red = ((np.indices((N,) * dim).sum(axis=0) + dim) & 1) == 1
    assert np.array_equal(lv == 0, red)
    lv, n = order_schedule(dim, N, orders.checkerboard(dim, N, red_first=False))
    assert n == 2 and np.array_equal(lv == 0, ~red)


@pytest.mark.parametrize("dim,N,seed", [(1, 12, 1), (2, 6, 2), (2, 8, 3), (3, 4, 4)])
def test_schedule_matches_brute_force_and_levels_are_independent(dim, N, seed):
    order = orders.random_order(dim, N, 2502_09537 + seed)
    lv, n = order_schedule(dim, N, order)
    want = _levels_brute(dim, N, order)
    assert np.array_equal(lv.ravel(), want)
    assert n == want.max() + 1
    flat = lv.ravel()
    for p in range(N ** dim):
        for q in _neighbours(dim, N, p):
            assert flat[p] != flat[q]


def test_block_split_order_structure():
    N, nb = 24, 3
    o = orders.block_split_2d(N, nb)
    assert np.array_equal(np.sort(o), np.arange(N * N))
    rows = (o // N).reshape(N, N)[:, 0].tolist()   # each row is visited whole, k ascending
    assert np.array_equal((o % N).reshape(N, N), np.tile(np.arange(N), (N, 1)))
    assert rows[0] == 0
    seps = rows[-nb:]
    assert seps[-1] == N - 1 and all(b - a >= 2 for a, b in zip([0] + seps, seps))
    # blocks (the rows between separators) never touch one another
    block_of = {}
    for b, (lo, hi) in enumerate(zip([0] + seps[:-1], seps)):
        for r in range(lo + 1, hi):
            block_of[r] = b
    for r, b in block_of.items():
        for r2 in ((r - 1) % N, (r + 1) % N):
            assert block_of.get(r2, b) == b
    with pytest.raises(ValueError):
        orders.block_split_2d(6, 3)


def test_schedule_rejects_non_permutations():
    o = orders.lexicographic(2, 6)
    bad = o.copy()
    bad[3] = bad[4]
    with pytest.raises(KGSError):
        order_schedule(2, 6, bad)
    bad = o.copy()
    bad[0] = 36
    with pytest.raises(KGSError):
        order_schedule(2, 6, bad)
    with pytest.raises(ValueError):
        order_schedule(2, 6, o[:-1])
    with pytest.raises(KGSError):
        order_schedule(2, 5, np.arange(25))   # odd N


@pytest.mark.parametrize("dim,N,seed", [(1, 16, 5), (2, 8, 6), (3, 4, 7)])
def test_oracle_depends_on_the_order_only_through_its_levels(orc, dim, N, seed):
    """Serial DP-AVF2 in a random order equals serial DP-AVF2 in that order's
    level-sorted form (levels ascending, ties in any order) bitwise; a
    different order (lexicographic) gives a different scheme."""
    prob = Problem(dim, N, 10.0, 1.0, 0.7, 1.1, 0.9, 0.01)
    order = orders.random_order(dim, N, 2502_09537 + seed)
    lv, _ = order_schedule(dim, N, order)
    rng = np.random.Generator(np.random.PCG64(seed))
    tie = rng.permutation(N ** dim)
    by_level = np.lexsort((tie, lv.ravel())).astype(np.int64)
    st = random_state(prob, 2502_09537 + 50 + seed)
    a = tuple(np.array(x, copy=True) for x in st)
    b = tuple(np.array(x, copy=True) for x in st)
    c = tuple(np.array(x, copy=True) for x in st)
    orc.steps_order(prob, *a, order, 5)
    orc.steps_order(prob, *b, by_level, 5)
    orc.steps_order(prob, *c, orders.lexicographic(dim, N), 5)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert any(not np.array_equal(x, z) for x, z in zip(a, c))


def test_package_checkerboard_is_the_oracles(orc):
    for dim, N in [(1, 8), (2, 6), (3, 4)]:
        for red_first in (True, False):
            assert np.array_equal(orders.checkerboard(dim, N, red_first),
                                  orc.checkerboard_order(dim, N, red_first))
