"""General update orders on the GPU (Sec. 3; Algorithms 1-3) against the oracle.

kgs_set_order runs any order of the points as a level schedule.  Checked
here: the checkerboard given as an order is bitwise the fused colour passes
(same pointwise arithmetic, same neighbour values); orders with the same
levels are bitwise equal; the lexicographic order (Eq. order1), its reverse
(Eq. order2), Algorithm 2's block order, the black-first checkerboard and
random orders match the oracle's serial DP-AVF2 in that order (float64 bar
1e-12, as for the checkerboard); energy is conserved in the lexicographic
order; the order can be reset and bad orders are rejected.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2502_09537_b300 import orders  # noqa: E402
from paper_2502_09537_b300.inputs import Problem, random_state  # noqa: E402
from paper_2502_09537_b300.solver import (KGS_FP32, KGS_FP64, KGS_OPT_GRAPH, KGSError,  # noqa: E402
                                          Solver, order_schedule)

FP64_BAR = 1e-12


def _copy(st):
    return tuple(np.array(a, dtype=np.float64, copy=True) for a in st)


def _gpu(prob, st, order, splits, precision=KGS_FP64, graph=1):
    with Solver.from_problem(prob, precision) as s:
        s.set_option(KGS_OPT_GRAPH, graph)
        s.set_state(*_copy(st))
        if order is not None:
            s.set_order(order)
        for n in splits:
            s.step(n)
        return s.get_state(), s.order_levels()


def _rel(a, b):
    return max(np.abs(x - y).max() / max(np.abs(y).max(), 1e-300) for x, y in zip(a, b))


def _bitwise(a, b):
    return all(np.array_equal(x.view(np.uint64), y.view(np.uint64)) for x, y in zip(a, b))


@pytest.mark.parametrize("precision", [KGS_FP64, KGS_FP32])
@pytest.mark.parametrize("dim,N", [(1, 64), (2, 32), (3, 10)])
def test_checkerboard_as_an_order_is_the_colour_passes(dim, N, precision):
    prob = Problem(dim, N, 8.0, 1.0, 0.8, 1.2, 0.9, 0.02)
    st = random_state(prob, 2502_09537 + 60 + dim)
    ref, lv0 = _gpu(prob, st, None, [7], precision)
    got, lv = _gpu(prob, st, orders.checkerboard(dim, N), [7], precision)
    assert lv0 == 2 and lv == 2
    assert _bitwise(got, ref)
    # the same levels in another order within each level
    perm = orders.checkerboard(dim, N)
    red = perm[: N ** dim // 2][::-1]
    black = perm[N ** dim // 2:][::-1]
    got2, _ = _gpu(prob, st, np.concatenate([red, black]), [3, 4], precision, graph=0)
    assert _bitwise(got2, ref)


@pytest.mark.parametrize("name,dim,N,nsteps", [
    ("lexicographic", 1, 64, 40),
    ("lexicographic", 2, 24, 60),
    ("reverse_lexicographic", 2, 20, 60),
    ("lexicographic", 3, 8, 30),
    ("black_first", 2, 16, 50),
    ("block_split", 2, 26, 40),
    ("random", 2, 12, 40),
    ("random", 3, 6, 20),
])
def test_order_matches_oracle(orc, name, dim, N, nsteps):
    prob = Problem(dim, N, 10.0, 1.0, 0.8, 1.1, 0.9, 0.01)
    st = random_state(prob, 2502_09537 + 70 + N)
    if name == "lexicographic":
        order = orders.lexicographic(dim, N)
    elif name == "reverse_lexicographic":
        order = orders.reverse_lexicographic(dim, N)
    elif name == "black_first":
        order = orders.checkerboard(dim, N, red_first=False)
    elif name == "block_split":
        order = orders.block_split_2d(N, 4)
    else:
        order = orders.random_order(dim, N, 2502_09537 + 80 + N)
    want = _copy(st)
    orc.steps_order(prob, *want, order, nsteps)
    got, lv = _gpu(prob, st, order, [nsteps])
    assert lv == order_schedule(dim, N, order)[1]
    assert _rel(got, want) <= FP64_BAR, _rel(got, want)
    # split calls (graph replays vs direct launches) give bitwise the same state
    got2, _ = _gpu(prob, st, order, [1, nsteps - 1], graph=0)
    assert _bitwise(got, got2)


def test_energy_conserved_in_lexicographic_order(orc):
    prob = Problem(2, 32, 16.0, 1.0, 1.0, 1.0, 1.0, 0.01)
    st = random_state(prob, 2502_09537 + 90)
    with Solver.from_problem(prob) as s:
        s.set_state(*_copy(st))
        s.set_order(orders.lexicographic(2, 32))
        E0, S0, _ = s.invariants()
        s.step(2000)
        E1, S1, _ = s.invariants()
    assert abs(E1 - E0) / max(S0, S1) < 1e-13


def test_reset_and_bad_orders():
    prob = Problem(2, 16, 8.0, 1.0, 1.0, 1.0, 1.0, 0.01)
    st = random_state(prob, 2502_09537 + 91)
    ref, _ = _gpu(prob, st, None, [5])
    with Solver.from_problem(prob) as s:
        s.set_state(*_copy(st))
        s.set_order(orders.lexicographic(2, 16))
        assert s.order_levels() == 31
        bad = orders.lexicographic(2, 16)
        bad[0] = 1
        with pytest.raises(KGSError):
            s.set_order(bad)
        assert s.order_levels() == 31          # unchanged by the rejected order
        s.set_orders(orders.lexicographic(2, 16), orders.reverse_lexicographic(2, 16))
        assert s.order_levels() == 62          # two sweeps per half step
        with pytest.raises(KGSError):
            s.set_order(bad)
        with pytest.raises(KGSError):
            s.set_orders(orders.lexicographic(2, 16), bad)
        assert s.order_levels() == 62          # per-variable orders kept by both rejections
        s.set_order(None)
        assert s.order_levels() == 2
        s.step(5)
        assert _bitwise(s.get_state(), ref)


@pytest.mark.parametrize("precision", [KGS_FP64, KGS_FP32])
@pytest.mark.parametrize("name,dim,N", [("lexicographic", 2, 24), ("lexicographic", 3, 8),
                                        ("random", 2, 14), ("block_split", 2, 26)])
def test_persistent_levels_are_bitwise_the_per_level_launches(name, dim, N, precision):
    """KGS_OPT_ORDER_MODE 2 (all levels of a step in one cooperative launch,
    a grid barrier after each level), 1 (one launch per level) and 3 (one
    launch per level on natural order) compute bitwise the same state; so does
    the automatic choice."""
    from paper_2502_09537_b300.solver import KGS_OPT_ORDER_MODE
    prob = Problem(dim, N, 10.0, 1.0, 0.8, 1.1, 0.9, 0.01)
    st = random_state(prob, 2502_09537 + 110 + N)
    order = {"lexicographic": orders.lexicographic(dim, N),
             "random": orders.random_order(dim, N, 2502_09537 + 111),
             "block_split": orders.block_split_2d(N, 4) if dim == 2 else None}[name]
    out = {}
    for mode in (1, 2, 3, 0):
        with Solver.from_problem(prob, precision) as s:
            s.set_option(KGS_OPT_ORDER_MODE, mode)
            s.set_state(*_copy(st))
            s.set_order(order)
            s.step(7)
            s.step(5)
            out[mode] = s.get_state()
    assert _bitwise(out[1], out[2]) and _bitwise(out[1], out[3]) and _bitwise(out[1], out[0])


def test_barrier_timeout_is_reported_and_the_context_survives():
    """A grid barrier that cannot complete (the test hook makes it wait for a
    CTA that does not exist) gives up after its 2 s bound: kgs_step returns
    KGS_ERR_TIMEOUT, the handle refuses further work, and the device stays
    usable for a new handle."""
    from paper_2502_09537_b300.solver import (KGS_ERR_TIMEOUT, KGS_OPT_ORDER_MODE,
                                              KGS_OPT_TEST_BARRIER_STALL)
    prob = Problem(2, 16, 8.0, 1.0, 1.0, 1.0, 1.0, 0.01)
    st = random_state(prob, 2502_09537 + 120)
    with Solver.from_problem(prob) as s:
        s.set_state(*_copy(st))
        s.set_order(orders.lexicographic(2, 16))
        s.set_option(KGS_OPT_ORDER_MODE, 2)
        s.set_option(KGS_OPT_TEST_BARRIER_STALL, 1)
        with pytest.raises(KGSError) as ei:
            s.step(1)
        assert ei.value.status == KGS_ERR_TIMEOUT
        with pytest.raises(KGSError) as ei:
            s.get_state()
        assert ei.value.status == KGS_ERR_TIMEOUT
    ref, _ = _gpu(prob, st, orders.lexicographic(2, 16), [3])
    want = _copy(st)
    from oracle import steps_order
    steps_order(prob, *want, orders.lexicographic(2, 16), 3)
    assert _rel(ref, want) <= FP64_BAR


@pytest.mark.parametrize("precision", [KGS_FP64, KGS_FP32])
@pytest.mark.parametrize("N,reverse", [(64, False), (96, False), (160, False), (64, True), (128, True)])
def test_lexicographic_sweep_is_bitwise_the_level_schedule(N, reverse, precision):
    """KGS_OPT_ORDER_MODE 4 (a doacross sweep: one warp per strip of 32 rows,
    lanes one column apart, strips chained by progress counters) computes the
    lexicographic order and its reverse bitwise as the per-level launches do
    (modes 3 and 1); auto takes the sweep."""
    from paper_2502_09537_b300.solver import KGS_OPT_ORDER_MODE
    prob = Problem(2, N, 11.0, 1.0, 0.8, 1.1, 0.9, 0.01)
    st = random_state(prob, 2502_09537 + 130 + N + int(reverse))
    order = orders.reverse_lexicographic(2, N) if reverse else orders.lexicographic(2, N)
    out = {}
    for mode in (4, 3, 1, 0):
        with Solver.from_problem(prob, precision) as s:
            s.set_option(KGS_OPT_ORDER_MODE, mode)
            s.set_state(*_copy(st))
            s.set_order(order)
            s.step(4)
            s.step(3)
            out[mode] = s.get_state()
    assert _bitwise(out[4], out[3]) and _bitwise(out[4], out[1]) and _bitwise(out[4], out[0])
    if precision == KGS_FP64:
        want = _copy(st)
        from oracle import steps_order
        steps_order(prob, *want, order, 7)
        assert _rel(out[4], want) <= FP64_BAR


def test_lexicographic_sweep_wait_timeout_is_reported():
    """A strip's wait that cannot complete (the test hook makes every strip
    wait for progress the strip before it never reaches) gives up after its
    2 s bound; the handle reports KGS_ERR_TIMEOUT at the next synchronising
    call and from then on, and a new handle works."""
    from paper_2502_09537_b300.solver import (KGS_ERR_TIMEOUT, KGS_OPT_ORDER_MODE,
                                              KGS_OPT_TEST_BARRIER_STALL)
    prob = Problem(2, 64, 8.0, 1.0, 1.0, 1.0, 1.0, 0.01)
    st = random_state(prob, 2502_09537 + 140)
    with Solver.from_problem(prob) as s:
        s.set_state(*_copy(st))
        s.set_order(orders.lexicographic(2, 64))
        s.set_option(KGS_OPT_ORDER_MODE, 4)
        s.set_option(KGS_OPT_TEST_BARRIER_STALL, 1)
        s.step(1)
        with pytest.raises(KGSError) as ei:
            s.get_state()
        assert ei.value.status == KGS_ERR_TIMEOUT
        with pytest.raises(KGSError) as ei:
            s.step(1)
        assert ei.value.status == KGS_ERR_TIMEOUT
    a, _ = _gpu(prob, st, orders.lexicographic(2, 64), [2])
    b, _ = _gpu(prob, st, None, [2])   # the checkerboard, for contrast
    want = _copy(st)
    from oracle import steps_order
    steps_order(prob, *want, orders.lexicographic(2, 64), 2)
    assert _rel(a, want) <= FP64_BAR and not _bitwise(a, b)


def _orders2_pair(dim, N, k):
    lex, rev = orders.lexicographic(dim, N), orders.reverse_lexicographic(dim, N)
    cb = orders.checkerboard(dim, N)
    r1 = orders.random_order(dim, N, 2502_09537 + 401 + dim)
    return [(lex, rev), (cb, r1), (rev, cb)][k]


@pytest.mark.parametrize("mode", [0, 1, 3])
@pytest.mark.parametrize("dim,N,k", [(1, 40, 0), (2, 18, 0), (2, 18, 1), (2, 64, 2), (3, 8, 1)])
def test_per_variable_orders_match_oracle(orc, dim, N, k, mode):
    """kgs_set_orders (one order for Psi, another for (U,V)) against the
    oracle's two-sweep form (float64 bar 1e-12), per-level launches on the
    colour-split layout (mode 1) and on the natural-order copy (3, auto)."""
    from paper_2502_09537_b300.solver import KGS_OPT_ORDER_MODE
    prob = Problem(dim, N, 9.0, 1.1, 0.9, 1.2, 0.8, 0.01)
    st = random_state(prob, 2502_09537 + 410 + dim + k, 0.6)
    op, ou = _orders2_pair(dim, N, k)
    with Solver.from_problem(prob) as s:
        s.set_option(KGS_OPT_ORDER_MODE, mode)
        s.set_state(*_copy(st))
        s.set_orders(op, ou)
        s.step(7)
        s.step(5)
        got = s.get_state()
    want = _copy(st)
    orc.steps_orders2(prob, *want, op, ou, 12)
    assert _rel(got, want) <= FP64_BAR


@pytest.mark.parametrize("precision", [KGS_FP64, KGS_FP32])
def test_equal_per_variable_orders_are_bitwise_one_order(precision):
    """With the same order for both variables the two-sweep form is the
    per-point form: bitwise kgs_set_order's result; kgs_set_order afterwards
    returns to one order."""
    prob = Problem(2, 22, 9.0, 1.1, 0.9, 1.2, 0.8, 0.01)
    st = random_state(prob, 2502_09537 + 420, 0.6)
    o = orders.random_order(2, 22, 2502_09537 + 421)
    one, _ = _gpu(prob, st, o, [6, 4], precision)
    with Solver.from_problem(prob, precision) as s:
        s.set_state(*_copy(st))
        s.set_orders(o, o)
        s.step(6)
        s.step(4)
        same = s.get_state()
    assert _bitwise(one, same)
    op, ou = _orders2_pair(2, 22, 1)
    with Solver.from_problem(prob, precision) as s:
        s.set_state(*_copy(st))
        s.set_orders(op, ou)
        assert s.order_levels() > 2
        s.set_order(o)
        s.step(6)
        s.step(4)
        reset = s.get_state()
    assert _bitwise(one, reset)


def test_energy_conserved_with_per_variable_orders():
    prob = Problem(2, 24, 8.0, 1.0, 1.1, 0.9, 1.2, 0.02)
    st = random_state(prob, 2502_09537 + 430, 0.6)
    op, ou = _orders2_pair(2, 24, 0)
    with Solver.from_problem(prob) as s:
        s.set_state(*_copy(st))
        s.set_orders(op, ou)
        E0, S0, _ = s.invariants()
        worst = 0.0
        for _ in range(5):
            s.step(200)
            E, S, _ = s.invariants()
            worst = max(worst, abs(E - E0) / max(S0, S))
    assert worst <= 1e-13, worst
