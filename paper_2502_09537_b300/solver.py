"""Thin ctypes binding of libkgs (the C ABI declared in ``include/kgs.h``).

Argument marshalling only: every step of the DP-AVF2 path runs in the CUDA
kernels of ``libkgs.so``.  There is no CPU fallback: if the library is missing
or no GPU is present the calls raise.

State arguments are four float64 arrays (P, Q, U, V) of shape (N,)*d in C
order: numpy arrays (host) or CUDA torch tensors (device; passed by pointer).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# KGS_LIBRARY may name another build of the same ABI (the index-checking
# libkgs_debug.so of build.build(debug_bounds=True)).
LIB_PATH = os.environ.get("KGS_LIBRARY") or os.path.join(HERE, "libkgs.so")

KGS_OK = 0
KGS_HOST = 0
KGS_DEVICE = 1
KGS_HOST_ASYNC = 2
KGS_FP64 = 64
KGS_FP32 = 32
KGS_OPT_KERNEL = 1
KGS_OPT_GRAPH = 2
KGS_OPT_THREADS = 3
KGS_OPT_PPT = 4
KGS_OPT_TILE_T1 = 5
KGS_OPT_TILE_T2 = 6
KGS_OPT_TILE_LX = 7
KGS_OPT_TILE_PASSES = 8
KGS_OPT_TILE_THREADS = 9
KGS_OPT_SLAB_PLANES = 10
KGS_OPT_ORDER_MODE = 11
KGS_OPT_TEST_BARRIER_STALL = 12
KGS_OPT_WAVE_LAG = 13
KGS_OPT_WAVE_CHUNK = 14
KGS_OPT_PDL = 15
KGS_OPT_STREAM_CHUNK = 16
KGS_OPT_STREAM_PREFETCH = 17
KGS_ERR_ARG = -1
KGS_ERR_TIMEOUT = -6

# Every function the header declares, with its ctypes signature.
_c_int64 = ctypes.c_int64
_c_dbl = ctypes.c_double
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
SIGNATURES = {
    "kgs_create": (_vp, [ctypes.c_int, _c_int64] + [_c_dbl] * 6),
    "kgs_create_ex": (_vp, [ctypes.c_int, _c_int64] + [_c_dbl] * 6 + [ctypes.c_int, ctypes.c_int]),
    "kgs_set_state": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, ctypes.c_int, _vp]),
    "kgs_get_state": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, ctypes.c_int, _vp]),
    "kgs_step": (ctypes.c_int, [_vp, _c_int64, _vp]),
    "kgs_invariants": (ctypes.c_int, [_vp, _dp, _vp]),
    "kgs_energy": (ctypes.c_int, [_vp, _dp]),
    "kgs_mass": (ctypes.c_int, [_vp, _dp]),
    "kgs_set_tau": (ctypes.c_int, [_vp, _c_dbl]),
    "kgs_set_option": (ctypes.c_int, [_vp, ctypes.c_int, _c_int64]),
    "kgs_launch_count": (_c_int64, [_vp]),
    "kgs_destroy": (None, [_vp]),
    "kgs_order_schedule": (ctypes.c_int, [ctypes.c_int, _c_int64, _vp, _vp, ctypes.POINTER(_c_int64)]),
    "kgs_set_order": (ctypes.c_int, [_vp, _vp]),
    "kgs_set_orders": (ctypes.c_int, [_vp, _vp, _vp]),
    "kgs_order_levels": (ctypes.c_int, [_vp, ctypes.POINTER(_c_int64)]),
    "kgs_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "kgs_last_error": (ctypes.c_char_p, []),
    "kgs_last_status": (ctypes.c_int, []),
    "kgs_invariants_noalloc": (ctypes.c_int, [ctypes.c_int, _c_int64] + [_c_dbl] * 5
                               + [_vp, _vp, _vp, _vp, _vp, _vp]),
    "kgs_batch_create": (_vp, [ctypes.c_int, _c_int64]),
    "kgs_batch_add": (_c_int64, [_vp, ctypes.c_int, _c_int64] + [_c_dbl] * 6 + [ctypes.c_int]),
    "kgs_batch_remove": (ctypes.c_int, [_vp, _c_int64]),
    "kgs_batch_free_bytes": (_c_int64, [_vp]),
    "kgs_batch_set_state": (ctypes.c_int, [_vp, _c_int64, _vp, _vp, _vp, _vp, ctypes.c_int, _vp]),
    "kgs_batch_get_state": (ctypes.c_int, [_vp, _c_int64, _vp, _vp, _vp, _vp, ctypes.c_int, _vp]),
    "kgs_batch_step_each": (ctypes.c_int, [_vp, ctypes.POINTER(_c_int64), _vp]),
    "kgs_batch_step": (ctypes.c_int, [_vp, _c_int64, _vp]),
    "kgs_batch_invariants": (ctypes.c_int, [_vp, _c_int64, _dp, _vp]),
    "kgs_batch_set_option": (ctypes.c_int, [_vp, ctypes.c_int, _c_int64]),
    "kgs_batch_launch_count": (_c_int64, [_vp]),
    "kgs_batch_destroy": (None, [_vp]),
    # include/kgs_probe.h
    "kgs_probe_fma_rate": (ctypes.c_int, [ctypes.c_int, _c_int64, ctypes.c_int, _vp, _dp, _dp]),
    "kgs_probe_nsum": (ctypes.c_int, [ctypes.c_int, _c_int64, _vp, _c_dbl, _vp, _vp, _vp, _vp]),
    "kgs_probe_psi_weight": (ctypes.c_int, [_c_int64, _vp, _vp, _vp]),
    "kgs_debug_bounds": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint32)]),
    "kgs_stream2_side_list": (ctypes.c_int, [_c_int64, _vp, _c_int64]),
}

_lib = None


class KGSError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libkgs status {status}: {msg}")
        self.status = status


def load_library():
    """Load libkgs.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libkgs not built at {LIB_PATH}; run "
                              "`python -m paper_2502_09537_b300.build`")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def debug_bounds():
    """(checking build?, flag bits set since the last call) of kgs_debug_bounds."""
    f = ctypes.c_uint32()
    r = load_library().kgs_debug_bounds(ctypes.byref(f))
    if r < 0:
        raise KGSError(r, "kgs_debug_bounds failed")
    return bool(r), int(f.value)


def stream2_side_list(N: int):
    """The two-step kernel's side list for an N^3 grid (kgs_stream2_side_list):
    entries (2, 2, 96) uint16 by tile kind and plane parity, and the list
    lengths (2, 2)."""
    buf = np.zeros(388, dtype=np.uint16)
    r = load_library().kgs_stream2_side_list(N, buf.ctypes.data, buf.size)
    if r < 0:
        raise KGSError(r, "kgs_stream2_side_list failed")
    return buf[:384].reshape(2, 2, 96).astype(np.int64), buf[384:].reshape(2, 2).astype(np.int64)


def last_error() -> str:
    return load_library().kgs_last_error().decode()


def _check(status: int):
    if status != KGS_OK:
        raise KGSError(status, last_error())


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


def _as_buffers(arrays: Sequence, N: int, dim: int):
    """Return (where, pointers, keepalive) for four state arrays."""
    shape = (N,) * dim
    if all(isinstance(a, np.ndarray) for a in arrays):
        out = []
        for a in arrays:
            if a.shape != shape or a.dtype != np.float64 or not a.flags.c_contiguous:
                raise ValueError(f"host state arrays must be C-contiguous float64 {shape}")
            out.append(a)
        return KGS_HOST, [a.ctypes.data for a in out], out
    import torch
    out = []
    for a in arrays:
        if not (isinstance(a, torch.Tensor) and a.is_cuda and a.dtype == torch.float64
                and tuple(a.shape) == shape and a.is_contiguous()):
            raise ValueError(f"device state tensors must be contiguous CUDA float64 {shape}")
        out.append(a)
    return KGS_DEVICE, [a.data_ptr() for a in out], out


class Solver:
    """One periodic KGS problem advanced by the DP-AVF2 checkerboard scheme."""

    def __init__(self, dim: int, N: int, L: float, kappa1: float, kappa2: float, mu: float,
                 gamma: float, tau: float, precision: int = KGS_FP64, device: int = -1):
        lib = load_library()
        self._lib = lib
        h = lib.kgs_create_ex(dim, N, L, kappa1, kappa2, mu, gamma, tau, precision, device)
        if not h:
            raise KGSError(lib.kgs_last_status(), last_error())
        self._h = ctypes.c_void_p(h)
        self.dim, self.N, self.L, self.precision = dim, N, L, precision

    @classmethod
    def from_problem(cls, prob, precision: int = KGS_FP64, device: int = -1) -> "Solver":
        return cls(prob.dim, prob.N, prob.L, prob.kappa1, prob.kappa2, prob.mu, prob.gamma,
                   prob.tau, precision, device)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.kgs_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # state ---------------------------------------------------------------
    def set_state(self, P, Q, U, V, stream=None, asynchronous=False):
        """Copy a state in.  asynchronous=True with host arrays queues the copy
        on `stream` and returns at once (KGS_HOST_ASYNC): the arrays (pinned,
        for the copy to overlap other work) must stay unchanged until the
        stream has passed it."""
        where, ptrs, _keep = _as_buffers((P, Q, U, V), self.N, self.dim)
        if asynchronous and where == KGS_HOST:
            where = KGS_HOST_ASYNC
        _check(self._lib.kgs_set_state(self._h, *ptrs, where, _stream_ptr(stream)))

    def get_state(self, out=None, stream=None, asynchronous=False):
        """Return (P, Q, U, V).  With out=None, new numpy arrays; otherwise fills
        the four given numpy arrays or CUDA tensors.  asynchronous=True with
        host arrays queues the copy on `stream` (KGS_HOST_ASYNC): the arrays
        hold the state once the stream has passed it."""
        if out is None:
            out = tuple(np.empty((self.N,) * self.dim) for _ in range(4))
        where, ptrs, _keep = _as_buffers(out, self.N, self.dim)
        if asynchronous and where == KGS_HOST:
            where = KGS_HOST_ASYNC
        _check(self._lib.kgs_get_state(self._h, *ptrs, where, _stream_ptr(stream)))
        return tuple(out)

    # stepping ------------------------------------------------------------
    def step(self, nsteps: int, stream=None):
        _check(self._lib.kgs_step(self._h, int(nsteps), _stream_ptr(stream)))

    def set_tau(self, tau: float):
        _check(self._lib.kgs_set_tau(self._h, float(tau)))

    def set_option(self, option: int, value: int):
        _check(self._lib.kgs_set_option(self._h, int(option), int(value)))

    def set_order(self, order=None):
        """Update order of the following steps: a permutation of the linear
        indices 0 .. N^d - 1 (visited in this order by the base half, in the
        reverse order by the adjoint half), or None for the checkerboard."""
        if order is None:
            _check(self._lib.kgs_set_order(self._h, None))
            return
        o = _order_array(order, self.N ** self.dim)
        _check(self._lib.kgs_set_order(self._h, o.ctypes.data))

    def set_orders(self, order_psi, order_uv):
        """One update order for Psi and another for (U,V) (kgs_set_orders):
        each half step sweeps the variables in their own orders, (U,V) first
        and both reversed in the adjoint half."""
        M = self.N ** self.dim
        op = _order_array(order_psi, M)
        ou = _order_array(order_uv, M)
        _check(self._lib.kgs_set_orders(self._h, op.ctypes.data, ou.ctypes.data))

    def order_levels(self) -> int:
        """Parallel levels per half step of the current order (2 for the checkerboard)."""
        n = ctypes.c_int64()
        _check(self._lib.kgs_order_levels(self._h, ctypes.byref(n)))
        return n.value

    # diagnostics ---------------------------------------------------------
    def invariants(self, stream=None):
        """(E_h, S_E, mass) in float64."""
        out = (ctypes.c_double * 3)()
        _check(self._lib.kgs_invariants(self._h, ctypes.cast(out, _dp), _stream_ptr(stream)))
        return float(out[0]), float(out[1]), float(out[2])

    def energy(self) -> float:
        e = ctypes.c_double()
        _check(self._lib.kgs_energy(self._h, ctypes.byref(e)))
        return e.value

    def mass(self) -> float:
        m = ctypes.c_double()
        _check(self._lib.kgs_mass(self._h, ctypes.byref(m)))
        return m.value

    @property
    def launch_count(self) -> int:
        return int(self._lib.kgs_launch_count(self._h))


def _order_array(order, M: int) -> np.ndarray:
    o = np.ascontiguousarray(order, dtype=np.int64).ravel()
    if o.size != M:
        raise ValueError(f"an order has N^d = {M} entries (got {o.size})")
    return o


def order_schedule(dim: int, N: int, order):
    """(level of every point by linear index, number of levels) of an update
    order, computed by the library on the host (kgs_order_schedule)."""
    lib = load_library()
    o = _order_array(order, N ** dim)
    level = np.empty(o.size, dtype=np.int32)
    n = ctypes.c_int64()
    _check(lib.kgs_order_schedule(int(dim), int(N), o.ctypes.data, level.ctypes.data, ctypes.byref(n)))
    return level.reshape((N,) * dim), n.value


def probe_fma_rate(precision: int = 64, iters: int = 4096, blocks_per_sm: int = 8, stream=None):
    """Measured FMA rate of the FP64 (or FP32) pipe in FMA/s (include/kgs_probe.h)."""
    lib = load_library()
    ms, rate = ctypes.c_double(), ctypes.c_double()
    st = lib.kgs_probe_fma_rate(precision, iters, blocks_per_sm, _stream_ptr(stream),
                                ctypes.byref(ms), ctypes.byref(rate))
    if st != 0:
        raise KGSError(st, "FMA probe failed")
    return rate.value, ms.value


def probe_nsum(x, beta: float = 1.0, stream=None):
    """The colour passes' float64 neighbour sums of each row of x (shape
    (n, k), k in {2, 4, 6}): (S, beta*S, exact) where bit 0 of exact[i] says S
    of row i came from the exact integer accumulator (correctly rounded) and
    bit 1 that beta*S did (beta times the exact sum, rounded once); otherwise
    the left-to-right float64 sum (times beta) was taken."""
    import numpy as np
    lib = load_library()
    x = np.ascontiguousarray(x, dtype=np.float64)
    if x.ndim != 2:
        raise ValueError("x must be (n, k)")
    n, k = x.shape
    out = np.empty(n, dtype=np.float64)
    scaled = np.empty(n, dtype=np.float64)
    exact = np.empty(n, dtype=np.int32)
    st = lib.kgs_probe_nsum(k, n, x.ctypes.data, float(beta), out.ctypes.data, scaled.ctypes.data,
                            exact.ctypes.data, _stream_ptr(stream))
    if st != 0:
        raise KGSError(st, "neighbour-sum probe failed")
    return out, scaled, exact


def probe_psi_weight(r, stream=None):
    """w = 1 / (1 + r^2) for each value of r as the float64 colour passes form it."""
    import numpy as np
    lib = load_library()
    r = np.ascontiguousarray(r, dtype=np.float64).ravel()
    w = np.empty_like(r)
    st = lib.kgs_probe_psi_weight(r.size, r.ctypes.data, w.ctypes.data, _stream_ptr(stream))
    if st != 0:
        raise KGSError(st, "Psi weight probe failed")
    return w


KGS_BATCH_OPT_CTAS_PER_SM = 1
KGS_BATCH_OPT_GRAPH = 2
KGS_BATCH_OPT_PERSISTENT = 3
KGS_BATCH_OPT_TEST_STALL = 4
KGS_BATCH_OPT_CTAS_LIST = 16  # + 3 p + (dim - 1), p = 0 FP64 / 1 FP32


class Batch:
    """Independent KGS instances stepped together (kgs_batch_* of kgs.h)."""

    def __init__(self, capacity_bytes: int, device: int = -1):
        lib = load_library()
        self._lib = lib
        h = lib.kgs_batch_create(device, int(capacity_bytes))
        if not h:
            raise KGSError(lib.kgs_last_status(), last_error())
        self._h = ctypes.c_void_p(h)
        self._shape = {}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.kgs_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def add(self, prob, precision: int = KGS_FP64) -> int:
        i = self._lib.kgs_batch_add(self._h, prob.dim, prob.N, prob.L, prob.kappa1, prob.kappa2,
                                    prob.mu, prob.gamma, prob.tau, precision)
        if i < 0:
            raise KGSError(int(i), last_error())
        self._shape[int(i)] = (prob.N, prob.dim)
        return int(i)

    def remove(self, i: int):
        _check(self._lib.kgs_batch_remove(self._h, i))
        self._shape.pop(i, None)

    def free_bytes(self) -> int:
        return int(self._lib.kgs_batch_free_bytes(self._h))

    def set_state(self, i: int, P, Q, U, V, stream=None):
        N, dim = self._shape[i]
        where, ptrs, _keep = _as_buffers((P, Q, U, V), N, dim)
        _check(self._lib.kgs_batch_set_state(self._h, i, *ptrs, where, _stream_ptr(stream)))

    def get_state(self, i: int, out=None, stream=None):
        N, dim = self._shape[i]
        if out is None:
            out = tuple(np.empty((N,) * dim) for _ in range(4))
        where, ptrs, _keep = _as_buffers(out, N, dim)
        _check(self._lib.kgs_batch_get_state(self._h, i, *ptrs, where, _stream_ptr(stream)))
        return tuple(out)

    def step(self, nsteps: int, stream=None):
        _check(self._lib.kgs_batch_step(self._h, int(nsteps), _stream_ptr(stream)))

    def step_each(self, nsteps, stream=None):
        arr = (ctypes.c_int64 * len(nsteps))(*[int(n) for n in nsteps])
        _check(self._lib.kgs_batch_step_each(self._h, arr, _stream_ptr(stream)))

    def invariants(self, i: int, stream=None):
        out = (ctypes.c_double * 3)()
        _check(self._lib.kgs_batch_invariants(self._h, i, ctypes.cast(out, _dp), _stream_ptr(stream)))
        return float(out[0]), float(out[1]), float(out[2])

    def set_option(self, option: int, value: int):
        _check(self._lib.kgs_batch_set_option(self._h, int(option), int(value)))

    @property
    def launch_count(self) -> int:
        return int(self._lib.kgs_batch_launch_count(self._h))
