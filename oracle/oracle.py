"""ctypes wrapper of the FP64 CPU oracle (``kgs_oracle.c``).

TEST INFRASTRUCTURE: imported only by the tests, the smoke check and the
benchmark's CPU-baseline legs.  Every function works in place on float64
numpy arrays of shape ``(N,) * dim`` (C order, index ``[ix][iy][iz]``).

Functions and the passages of arXiv 2502.09537 they follow:
  steps_order            Algorithm 1 (in-place DP-AVF2 sweep over any order),
                         Eqs. scheme1, dp-avf-kj-adj, dp-comp
  checkerboard_order     Sec. 4.2 / Algorithm 3 colour rule (red = odd 1-based
                         index sum), red points first
  steps_checkerboard     Algorithm 1 with the checkerboard order
  steps_checkerboard_omp the same, one colour's points split over threads
  invariants             E_h (Sec. 2, Eq. ene-origin) with forward differences,
                         its absolute-term scale, and the mass h^d sum |Psi|^2
"""
import ctypes
import os

import numpy as np

from . import build as _build

MUT_ADJ_LITERAL = 1
MUT_NO_REVERSE = 2
MUT_RHO_OLD_BASE = 4
MUT_ALPHA_2D = 8
MUT_NO_ADJ_SWAP = 16
MUT_COLOUR_0BASED = 32

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        common = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                  ctypes.c_double, ctypes.c_double, ctypes.c_double]
        lib.orc_steps_order.argtypes = common + [ctypes.c_double, _dp, _dp, _dp, _dp,
                                                 _i64p, ctypes.c_int64, ctypes.c_int]
        lib.orc_steps_order.restype = None
        lib.orc_steps_orders2.argtypes = common + [ctypes.c_double, _dp, _dp, _dp, _dp,
                                                   _i64p, _i64p, ctypes.c_int64, ctypes.c_int]
        lib.orc_steps_orders2.restype = None
        lib.orc_steps_checkerboard.argtypes = common + [ctypes.c_double, _dp, _dp, _dp, _dp,
                                                        ctypes.c_int64]
        lib.orc_steps_checkerboard.restype = None
        lib.orc_steps_checkerboard_omp.argtypes = common + [ctypes.c_double, _dp, _dp, _dp, _dp,
                                                            ctypes.c_int64, ctypes.c_int]
        lib.orc_steps_checkerboard_omp.restype = None
        lib.orc_checkerboard_order.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int, _i64p]
        lib.orc_checkerboard_order.restype = None
        lib.orc_checkerboard_order_mut.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int,
                                                   ctypes.c_int, _i64p]
        lib.orc_checkerboard_order_mut.restype = None
        lib.orc_invariants.argtypes = common + [_dp, _dp, _dp, _dp, _dp]
        lib.orc_invariants.restype = None
        lib.orc_max_threads.argtypes = []
        lib.orc_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _check_state(dim, N, arrays):
    shape = (N,) * dim
    for a in arrays:
        if not (isinstance(a, np.ndarray) and a.dtype == np.float64
                and a.flags.c_contiguous and a.shape == shape):
            raise ValueError(f"oracle state must be C-contiguous float64 of shape {shape}")


def checkerboard_order(dim: int, N: int, red_first: bool = True, mut: int = 0) -> np.ndarray:
    """The checkerboard update order: one colour's points in lexicographic
    order, then the other's; red first (the paper's order) unless red_first is
    False.  mut may plant MUT_COLOUR_0BASED (tests of the colour pins)."""
    order = np.empty(N ** dim, dtype=np.int64)
    _load().orc_checkerboard_order_mut(dim, N, 1 if red_first else 0, mut,
                                       order.ctypes.data_as(_i64p))
    return order


def steps_order(prob, P, Q, U, V, order, nsteps: int, mut: int = 0) -> None:
    """Advance (P,Q,U,V) in place by nsteps DP-AVF2 steps in the given update order."""
    dim, N, L, k1, k2, mu, gamma, tau = prob
    _check_state(dim, N, (P, Q, U, V))
    order = np.ascontiguousarray(order, dtype=np.int64)
    if order.shape != (N ** dim,) or not np.array_equal(np.sort(order), np.arange(N ** dim)):
        raise ValueError("order must be a permutation of 0..N^d-1")
    _load().orc_steps_order(dim, N, L, k1, k2, mu, gamma, tau, _ptr(P), _ptr(Q), _ptr(U),
                            _ptr(V), order.ctypes.data_as(_i64p), nsteps, mut)


def _permutation(order, M):
    order = np.ascontiguousarray(order, dtype=np.int64)
    if order.shape != (M,) or not np.array_equal(np.sort(order), np.arange(M)):
        raise ValueError("order must be a permutation of 0..N^d-1")
    return order


def steps_orders2(prob, P, Q, U, V, order_psi, order_uv, nsteps: int, mut: int = 0) -> None:
    """Advance (P,Q,U,V) in place by nsteps DP-AVF2 steps with one update order
    for Psi and another for (U,V) (the remark after Eq. dp-avf-kj-adj): per
    step the Psi sweep in order_psi, the (U,V) sweep in order_uv, then both
    reversed, (U,V) first (orc_steps_orders2 states the reading)."""
    dim, N, L, k1, k2, mu, gamma, tau = prob
    _check_state(dim, N, (P, Q, U, V))
    op = _permutation(order_psi, N ** dim)
    ou = _permutation(order_uv, N ** dim)
    _load().orc_steps_orders2(dim, N, L, k1, k2, mu, gamma, tau, _ptr(P), _ptr(Q), _ptr(U), _ptr(V),
                              op.ctypes.data_as(_i64p), ou.ctypes.data_as(_i64p), nsteps, mut)


def steps_checkerboard(prob, P, Q, U, V, nsteps: int) -> None:
    dim, N, L, k1, k2, mu, gamma, tau = prob
    _check_state(dim, N, (P, Q, U, V))
    _load().orc_steps_checkerboard(dim, N, L, k1, k2, mu, gamma, tau, _ptr(P), _ptr(Q),
                                   _ptr(U), _ptr(V), nsteps)


def steps_checkerboard_omp(prob, P, Q, U, V, nsteps: int, nthreads: int = 0) -> None:
    dim, N, L, k1, k2, mu, gamma, tau = prob
    _check_state(dim, N, (P, Q, U, V))
    _load().orc_steps_checkerboard_omp(dim, N, L, k1, k2, mu, gamma, tau, _ptr(P), _ptr(Q),
                                       _ptr(U), _ptr(V), nsteps, nthreads)


def invariants(prob, P, Q, U, V):
    """Return (E_h, S_E, mass) of the state."""
    dim, N, L, k1, k2, mu, gamma, _tau = prob
    _check_state(dim, N, (P, Q, U, V))
    out = np.zeros(3)
    _load().orc_invariants(dim, N, L, k1, k2, mu, gamma, _ptr(P), _ptr(Q), _ptr(U), _ptr(V),
                           _ptr(out))
    return float(out[0]), float(out[1]), float(out[2])


def max_threads() -> int:
    return int(_load().orc_max_threads())


__all__ = [n for n in dir() if not n.startswith("_") and n not in ("ctypes", "os", "np")]
