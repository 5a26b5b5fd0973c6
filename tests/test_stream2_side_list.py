"""The host-built side list of the two-steps-per-launch kernel
(kgs_stream2_side_list, no device needed) against the dependency regions
worked out here from the checkerboard's neighbour rule, for every height of a
grid's last row of tiles.

One step pair's passes B1, R1, B2, R2 run on planes a, a-1, a-2, a-3; R2
updates the tile on its plane; a pass's region on a plane is what the next
pass reads there (its own points, their in-plane neighbours of the pass's
colour) and on the planes on either side (the same positions).  A point of
colour c on a plane whose parity with the tile's first row is P, in tile row
y and colour column k, has its last-axis neighbours at columns k - 1 + zp
and k + zp, zp = (c ^ P ^ y) & 1 (red = even coordinate sum in 3D, c = 0)."""
import numpy as np
import pytest

from paper_2502_09537_b300 import build as kbuild
from paper_2502_09537_b300 import solver

TY, TH, SIDE = 23, 32, 96
RED, BLACK = 0, 1


@pytest.fixture(scope="module")
def side_list():
    kbuild.build()
    solver.load_library()
    return solver.stream2_side_list


def reads(points, colour, P):
    out = set()
    for y, k in points:
        zp = (colour ^ P ^ y) & 1
        out |= {(y - 1, k), (y + 1, k), (y, k - 1 + zp), (y, k + zp)}
    return out


def regions(ty, q):
    """B1's region on a plane of parity q, R1's on q ^ 1, B2's on q, and the tile."""
    T = {(y, k) for y in range(ty) for k in range(TH)}

    def d3(P):
        return T | reads(T, RED, P)

    def d2(P):
        return d3(P) | d3(P ^ 1) | reads(d3(P), BLACK, P)

    def d1(P):
        return d2(P) | d2(P ^ 1) | reads(d2(P), RED, P)
    return d1(q), d2(q ^ 1), d3(q), T


def expected(ty, q):
    D1, D2, D3, T = regions(ty, q)
    main = {(y, k) for y in range(-3, ty + 3) for k in range(TH)}
    side = [(int(p in D2) + int(p in D3) + 1, p) for p in D1 - main]
    return D1, D2, D3, T, main, side


@pytest.mark.parametrize("ty", list(range(1, TY + 1)))
def test_regions_fit_the_thread_layout(ty):
    """Main threads (tile rows -3 .. ty + 2, the 32 columns) take a prefix of
    the passes that depends on the row only; every other point is a side
    point with at most three passes; everything B1 reads lies in the staged
    box (rows -4 .. ty + 3, columns -2 .. 33)."""
    for q in (0, 1):
        D1, D2, D3, T, main, side = expected(ty, q)
        assert T <= D3 <= D2 <= D1
        assert main <= D1
        for y, k in main:
            depth = sum((y, k) in D for D in (D1, D2, D3, T))
            assert depth == 1 + (-2 <= y <= ty + 1) + (-1 <= y <= ty) + (0 <= y < ty)
        assert len(side) <= SIDE and all(d <= 3 for d, _ in side)
        box = reads(D1, BLACK, q) | D1
        assert all(-4 <= y <= ty + 3 and -2 <= k <= TH + 1 for y, k in box)


@pytest.mark.parametrize("N", [64, 512, 576] + list(range(46, 92, 2)))
def test_library_side_list_is_the_regions(side_list, N):
    """Every last-tile height (N = 46 .. 90 covers N mod 23 = 0 .. 22): the
    library's entries are the side points, each with its passes, the points
    with more passes first."""
    pos, n = side_list(N)
    kinds = [(0, TY)] + ([(1, N % TY)] if N % TY else [])
    for kind, ty in kinds:
        for q in (0, 1):
            *_, side = expected(ty, q)
            got = []
            for e in pos[kind, q, :n[kind, q]]:
                assert e & 0x8000
                got.append((((e >> 11) & 3) + 1, ((e & 31) - 4, ((e >> 5) & 63) - 2)))
            assert n[kind, q] == len(side)
            assert sorted(got) == sorted(side)
            depths = [d for d, _ in got]
            assert depths == sorted(depths, reverse=True)
            assert (pos[kind, q, n[kind, q]:] == 0).all()
    if N % TY == 0:
        assert (n[1] == 0).all()


def test_side_list_rejects_bad_arguments(side_list):
    lib = solver.load_library()
    buf = np.zeros(400, dtype=np.uint16)
    assert lib.kgs_stream2_side_list(63, buf.ctypes.data, 400) == -1
    assert lib.kgs_stream2_side_list(2, buf.ctypes.data, 400) == -1
    assert lib.kgs_stream2_side_list(64, buf.ctypes.data, 387) == -1
    assert lib.kgs_stream2_side_list(64, None, 400) == -1
