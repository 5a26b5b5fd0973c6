"""The oracle's colour convention, pinned to the paper's figures.

A black-first checkerboard (or one that colours by 0-based index sums in 1D or
3D) is another valid DP-AVF2 scheme: it conserves the energy, is second order
and reversible, so the physics pins cannot tell it from the paper's.  What
fixes the convention is the paper itself:

  * the 2D checkerboard figure of Sec. 4.2 (its 16 nodes, read into
    tests/golden/gpu2d_colours.txt), with the bottom-left node blue;
  * the 3D checkerboard figure of Sec. 4.2 (its colour rule on 0-based
    lattice indices, tests/golden/gpu3d_colours.txt);
  * Algorithm 3: red is (j + k) mod 2 == 1 on 1-based indices, red first in
    the base half, blue first in the adjoint half;
  * the 1D configuration's "red/black (odd/even)": red = odd 1-based j.

The tests check that the figures agree with Algorithm 3's rule under the
stated reading, that the oracle's red set and colour order are exactly the
figures', that its steps are the in-place sweep in that hand-written order,
and that two planted mistakes (black first; 0-based colour sums) each fail.
"""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _grid_rows(lines):
    return [l.split() for l in lines if l.strip() and not l.startswith("#")]


def figure_2d_red():
    """Red points of the 2D figure as 1-based (j, k): column j from the left,
    row k from the bottom (rows in the file run top first)."""
    with open(os.path.join(GOLDEN, "gpu2d_colours.txt")) as f:
        rows = _grid_rows(f.read().splitlines())
    assert len(rows) == 4 and all(len(r) == 4 for r in rows)
    red = set()
    for r, row in enumerate(rows):
        k = 4 - r
        for c, col in enumerate(row):
            assert col in ("R", "B")
            if col == "R":
                red.add((c + 1, k))
    return red


def figure_3d_red():
    """Red points of the 3D figure as 1-based (j, k, l) = lattice (x, y, z) + 1."""
    with open(os.path.join(GOLDEN, "gpu3d_colours.txt")) as f:
        lines = [l for l in f.read().splitlines() if l.strip() and not l.startswith("#")]
    red, z = set(), None
    rows_seen = 0
    for l in lines:
        if l.startswith("z "):
            z = int(l.split()[1])
            rows_seen = 0
            continue
        yy = 3 - rows_seen
        rows_seen += 1
        for x, col in enumerate(l.split()):
            assert col in ("R", "B")
            if col == "R":
                red.add((x + 1, yy + 1, z + 1))
    assert len(red) == 32
    return red


def linear(idx1, N):
    """0-based linear index (axis 0 slowest) of a 1-based index tuple."""
    i = 0
    for a in idx1:
        i = i * N + (a - 1)
    return i


def test_2d_figure_is_algorithm_3_rule():
    """Under the reading (1,1) = bottom-left, the figure's red nodes are
    exactly Algorithm 3's (j + k) mod 2 == 1; the other corner reading
    ((1,1) = top-left) would make red (j + k) even, contradicting it."""
    red = figure_2d_red()
    assert red == {(j, k) for j in range(1, 5) for k in range(1, 5) if (j + k) % 2 == 1}
    assert (1, 1) not in red


def test_3d_figure_is_the_1_based_odd_rule():
    red = figure_3d_red()
    rule = {(j, k, l) for j in range(1, 5) for k in range(1, 5) for l in range(1, 5)
            if (j + k + l) % 2 == 1}
    assert red == rule


def colour_pin_failures(order_fn):
    """Every way order_fn(dim, N) departs from the paper's checkerboard order:
    its first half must be the red points (2D and 3D figures at N = 4, the
    rule carried to N = 6, 1D red = odd 1-based j), each colour's points in
    increasing order.  Returns a list of failure descriptions."""
    fails = []
    cases = [(1, 4, {(j,) for j in (1, 3)}),
             (1, 6, {(j,) for j in (1, 3, 5)}),
             (2, 4, figure_2d_red()),
             (3, 4, figure_3d_red()),
             (2, 6, {(j, k) for j in range(1, 7) for k in range(1, 7) if (j + k) % 2}),
             (3, 6, {(j, k, l) for j in range(1, 7) for k in range(1, 7) for l in range(1, 7)
                     if (j + k + l) % 2})]
    for dim, N, red in cases:
        order = np.asarray(order_fn(dim, N))
        M = N ** dim
        want_red = sorted(linear(p, N) for p in red)
        want_black = sorted(set(range(M)) - set(want_red))
        if list(order[: M // 2]) != want_red:
            fails.append(f"dim {dim} N {N}: first half is not the red points in order")
        if list(order[M // 2:]) != want_black:
            fails.append(f"dim {dim} N {N}: second half is not the blue points in order")
    return fails


def test_oracle_order_is_the_figures(orc):
    assert colour_pin_failures(orc.checkerboard_order) == []


def test_black_first_mutant_fails_the_colour_pin(orc):
    fails = colour_pin_failures(lambda d, n: orc.checkerboard_order(d, n, red_first=False))
    assert len(fails) == 12  # every case, both halves


def test_zero_based_colour_mutant_fails_the_colour_pin(orc):
    """Colouring by the 0-based index sum is the same in 2D and the opposite
    in 1D and 3D: the 2D pins pass it, the 1D and 3D pins fail it."""
    fails = colour_pin_failures(lambda d, n: orc.checkerboard_order(d, n, mut=orc.MUT_COLOUR_0BASED))
    assert fails and all(not f.startswith("dim 2") for f in fails)
    assert {f.split(":")[0] for f in fails} == {"dim 1 N 4", "dim 1 N 6", "dim 3 N 4", "dim 3 N 6"}


def _state(dim, N, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return tuple(np.ascontiguousarray(rng.uniform(-0.7, 0.7, (N,) * dim)) for _ in range(4))


@pytest.mark.parametrize("dim,N,hand", [
    (1, 4, [0, 2, 1, 3]),      # red = 1-based j in {1, 3} = 0-based {0, 2}
    (1, 6, [0, 2, 4, 1, 3, 5]),
])
def test_checkerboard_steps_are_the_hand_written_red_first_sweep_1d(orc, dim, N, hand):
    """steps_checkerboard is Algorithm 1's in-place sweep over the order
    written out by hand from the 1D rule (red = odd 1-based j, red first):
    bitwise equal to it, and different from the black-first sweep."""
    from paper_2502_09537_b300.inputs import Problem
    prob = Problem(dim, N, 2.5, 1.1, 0.9, 1.2, 0.8, 0.05)
    st = _state(dim, N, 7 + N)
    a = tuple(x.copy() for x in st)
    orc.steps_checkerboard(prob, *a, 3)
    b = tuple(x.copy() for x in st)
    orc.steps_order(prob, *b, np.array(hand), 3)
    c = tuple(x.copy() for x in st)
    black_first = hand[N // 2:] + hand[: N // 2]
    orc.steps_order(prob, *c, np.array(black_first), 3)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert not all(np.array_equal(x, y) for x, y in zip(a, c))


def test_checkerboard_steps_are_the_2d_figure_sweep(orc):
    """In 2D the sweep order is built from the figure itself: its red nodes
    (lexicographic), then its blue ones; the oracle's checkerboard steps are
    bitwise that sweep."""
    from paper_2502_09537_b300.inputs import Problem
    N = 4
    red = sorted(linear(p, N) for p in figure_2d_red())
    blue = sorted(set(range(N * N)) - set(red))
    prob = Problem(2, N, 3.0, 1.1, 0.9, 1.2, 0.8, 0.05)
    st = _state(2, N, 11)
    a = tuple(x.copy() for x in st)
    orc.steps_checkerboard(prob, *a, 3)
    b = tuple(x.copy() for x in st)
    orc.steps_order(prob, *b, np.array(red + blue), 3)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
