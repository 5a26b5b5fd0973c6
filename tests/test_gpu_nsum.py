"""The float64 neighbour sums of the colour passes against exact arithmetic.

Every FP64 colour pass forms S = the sum of a field over the 2d neighbours
(Eq. scheme1's discrete Laplacian without the centre term) and beta S.  The
kernels form S in an exact integer accumulator and round once, so on that path
S must be bitwise the correctly rounded sum, which Python's math.fsum returns
(Shewchuk's exact summation), and beta S must be bitwise beta times the exact
sum rounded once, which Python's Fraction arithmetic gives (float() of a
Fraction is correctly rounded).  On the rare fallback they must be the
left-to-right float64 sum and its rounded product with beta.  Rows cover wide
exponent spreads, exact and near cancellation, ties in the last place, signed
zeros, specials and values of the size the solver sees.
"""
import math
from fractions import Fraction

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


def _neg_zeros(row):
    return all(v == 0.0 and math.copysign(1.0, v) < 0 for v in row)


def _expected(row, exact):
    if exact:
        s = math.fsum(row)
        if s == 0.0:  # IEEE: a zero sum is -0 only when every term is -0
            s = -0.0 if _neg_zeros(row) else 0.0
        return s
    s = float(row[0])
    for v in row[1:]:
        s = s + float(v)
    return s


def _expected_scaled(row, beta, exact):
    if exact:
        f = Fraction(beta) * sum(Fraction(v) for v in row)
        if f == 0:
            return math.copysign(0.0, (-1.0 if _neg_zeros(row) else 1.0) * math.copysign(1.0, beta))
        return float(f)
    return beta * _expected(row, False)


def _biased_exponent(x):
    return (int(np.float64(x).view(np.uint64)) >> 52) & 0x7FF


def _fast_path_expected(row):
    """Whether the exact accumulator must take the row: finite values whose
    nonzero members lie within 31 binades of the largest (a subnormal counts
    as exponent 1), and an exact sum that is zero or has a normal exponent."""
    if not all(math.isfinite(v) for v in row):
        return False
    es = [max(_biased_exponent(v), 1) for v in row]
    nz = [e for e, v in zip(es, row) if v != 0.0]
    if nz and max(es) - min(nz) > 31:
        return False
    f = sum(Fraction(v) for v in row)
    if f == 0:
        return True
    a = abs(f)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if a < Fraction(2) ** e:
        e -= 1
    return 1 <= e + 1023 <= 0x7FE


def _same(a, b):
    if math.isnan(a) and math.isnan(b):
        return True
    return np.float64(a).view(np.uint64) == np.float64(b).view(np.uint64)


@pytest.mark.parametrize("k,beta", [(2, 1.0), (4, 0.30517578125), (4, -0.1234567890123), (6, 7.3e5)])
def test_neighbour_sum_is_correctly_rounded(k, beta):
    x = _rows(k, 1 << 15, 2502_09537 + 40 + k)
    got, scaled, exact = probe_nsum(x, beta)
    assert not (exact == -1).any(), "nsum entry points disagree with their halves"
    bad = []
    for i in range(x.shape[0]):
        row = x[i].tolist()
        want = _expected(row, bool(exact[i] & 1))
        want2 = _expected_scaled(row, beta, bool(exact[i] & 2))
        if not _same(want, got[i]) or not _same(want2, scaled[i]):
            bad.append((row, want, float(got[i]), want2, float(scaled[i]), int(exact[i])))
    assert not bad, bad[:5]
    # the exact path takes exactly the rows it should
    want_fast = np.array([_fast_path_expected(r) for r in x.tolist()])
    assert np.array_equal((exact & 1) == 1, want_fast)
    assert want_fast.mean() > 0.6 and ((exact & 2) > 0).mean() > 0.55


def test_neighbour_sum_fast_path_on_solver_like_values():
    rng = np.random.Generator(np.random.PCG64(2502_09537 + 47))
    base = np.exp(-rng.uniform(0, 30, size=(1 << 15, 1)))
    x = base * (1 + 0.05 * rng.normal(size=(1 << 15, 4))) + 1e-4 * rng.normal(size=(1 << 15, 4))
    beta = 0.5 * 5e-4 / (2 * (40.0 / 2048) ** 2)
    got, scaled, exact = probe_nsum(x, beta)
    assert (exact == 3).mean() > 0.999
    sel = exact == 3
    want = np.array([math.fsum(r) for r in x.tolist()])
    want2 = np.array([float(Fraction(beta) * sum(Fraction(v) for v in r)) for r in x.tolist()])
    assert np.array_equal(got[sel].view(np.uint64), want[sel].view(np.uint64))
    assert np.array_equal(scaled[sel].view(np.uint64), want2[sel].view(np.uint64))


def test_neighbour_sum_zero_or_subnormal_beta_falls_back():
    x = np.array([[1.0, 2.0, 3.0, 4.0], [-0.0, -0.0, -0.0, -0.0]])
    for beta in (0.0, -0.0, 5e-324):
        got, scaled, exact = probe_nsum(x, beta)
        assert (exact & 2).sum() == 0
        assert _same(scaled[0], beta * 10.0) and _same(scaled[1], beta * -0.0)


def test_neighbour_sum_empty():
    got, scaled, exact = probe_nsum(np.zeros((0, 4)))
    assert got.shape == (0,) and scaled.shape == (0,) and exact.shape == (0,)


def _ulps(a, b):
    ia = np.float64(a).view(np.int64)
    ib = np.float64(b).view(np.int64)
    return abs(int(ia) - int(ib))


def test_psi_weight_within_one_ulp_of_exact():
    """w = 1/(1 + r^2) (Eq. scheme1's Psi update in increment form) as the FP64
    passes form it on the integer pipes: within one ulp of the exact value
    everywhere, correctly rounded almost everywhere."""
    from paper_2502_09537_b300.solver import probe_psi_weight
    rng = np.random.Generator(np.random.PCG64(2502_09537 + 48))
    r = np.concatenate([
        rng.choice([-1.0, 1.0], size=60000) * 2.0 ** rng.uniform(-32, 31, size=60000),
        rng.uniform(-3, 3, size=20000),
        np.array([0.0, -0.0, 5e-324, 1e-300, 2.0 ** -27, -2.0 ** -27, 2.0 ** -26.999, 1.0, -1.0,
                  2.0, 2.0 ** 29, 2.0 ** 30, -2.0 ** 31, 1e10, 2.0 ** 510, 2.0 ** 520, 1e200,
                  np.inf, -np.inf])])
    r = np.concatenate([r, rng.choice([-1.0, 1.0], size=6000) * 2.0 ** rng.uniform(30, 545, size=6000)])
    w = probe_psi_weight(r)
    assert math.isnan(probe_psi_weight(np.array([np.nan]))[0])
    worst, exact, where = 0, 0, None
    for ri, wi in zip(r.tolist(), w.tolist()):
        if math.isinf(ri):
            assert wi == 0.0
            continue
        want = float(Fraction(1) / (1 + Fraction(ri) ** 2))
        u = _ulps(wi, want)
        if u > worst:
            worst, where = u, (ri, wi, want)
        exact += u == 0
    assert worst <= 1, where
    assert exact / (r.size - 2) > 0.999
