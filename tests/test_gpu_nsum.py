"""The float64 neighbour sum of the colour passes against the exact sum.

Every FP64 colour pass forms S = the sum of a field over the 2d neighbours
(Eq. scheme1's discrete Laplacian without the centre term).  The kernels form
it in an exact integer accumulator and round once, so on its fast path the
result must be bitwise the correctly rounded sum, which Python's math.fsum
returns (Shewchuk's exact summation); on the rare fallback it must be the
left-to-right float64 sum.  Rows cover wide exponent spreads, exact and near
cancellation, ties in the last place, signed zeros, specials and values of the
size the solver sees.
"""
import math

import numpy as np
import pytest

from paper_2502_09537_b300.solver import probe_nsum

pytestmark = pytest.mark.gpu


def _rows(k, n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.normal(size=(n, k))
    c = n // 8
    x[c:2 * c] *= 2.0 ** rng.integers(-90, 90, size=(c, k))
    x[2 * c:3 * c, 1] = -x[2 * c:3 * c, 0]
    x[3 * c:4 * c, 1] = -x[3 * c:4 * c, 0] * (1 + rng.integers(-9, 9, size=c) * 2.0 ** -52)
    x[3 * c:4 * c, 0] *= 2.0 ** -60
    x[4 * c:5 * c] = (rng.integers(-2 ** 20, 2 ** 20, size=(c, k)) * 2.0 ** -20
                      + rng.integers(0, 3, size=(c, k)) * 2.0 ** -74)
    x[5 * c:5 * c + c // 4] = 0.0
    x[5 * c + c // 4:5 * c + c // 2] = -0.0
    x[5 * c + c // 2:6 * c, ::2] = 0.0
    specials = np.array([np.inf, -np.inf, np.nan, 5e-324, 1e-310, 1.7976931348623157e308,
                         2.2250738585072014e-308])
    x[6 * c:7 * c, 0] = rng.choice(specials, size=c)
    x[7 * c:] = 1e-4 * rng.normal(size=(n - 7 * c, k))
    return x


def _expected(row, exact):
    if exact:
        s = math.fsum(row)
        if s == 0.0:  # IEEE: a zero sum is -0 only when every term is -0
            s = -0.0 if all(v == 0.0 and math.copysign(1.0, v) < 0 for v in row) else 0.0
        return s
    s = float(row[0])
    for v in row[1:]:
        s = s + float(v)
    return s


@pytest.mark.parametrize("k", [2, 4, 6])
def test_neighbour_sum_is_correctly_rounded(k):
    x = _rows(k, 1 << 16, 2502_09537 + 40 + k)
    got, exact = probe_nsum(x)
    assert not (exact == -1).any(), "nsum disagrees with its two halves"
    bad = []
    for i in range(x.shape[0]):
        want = _expected(x[i].tolist(), exact[i] == 1)
        if math.isnan(want) and math.isnan(got[i]):
            continue
        if np.float64(want).view(np.uint64) != np.float64(got[i]).view(np.uint64):
            bad.append((x[i].tolist(), want, float(got[i]), int(exact[i])))
    assert not bad, bad[:5]
    # the fast path takes every row of finite normal values within 71 binades
    assert exact.mean() > 0.7


def test_neighbour_sum_fast_path_on_solver_like_values():
    rng = np.random.Generator(np.random.PCG64(2502_09537 + 47))
    base = np.exp(-rng.uniform(0, 30, size=(1 << 16, 1)))
    x = base * (1 + 0.05 * rng.normal(size=(1 << 16, 4))) + 1e-4 * rng.normal(size=(1 << 16, 4))
    got, exact = probe_nsum(x)
    assert exact.mean() > 0.999
    want = np.array([math.fsum(r) for r in x.tolist()])
    sel = exact == 1
    assert np.array_equal(got[sel].view(np.uint64), want[sel].view(np.uint64))


def test_neighbour_sum_empty():
    got, exact = probe_nsum(np.zeros((0, 4)))
    assert got.shape == (0,) and exact.shape == (0,)
