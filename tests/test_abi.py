"""The C ABI without a GPU: the library builds for sm_103a, loads, exports every
function include/kgs.h declares, and rejects invalid arguments before touching
CUDA.  Compute calls are exercised by the GPU tests."""
import ctypes
import os
import re

import pytest

from paper_2502_09537_b300 import build as kbuild
from paper_2502_09537_b300 import solver

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in ("kgs.h", "kgs_probe.h")]


def declared_functions():
    text = "".join(open(h).read() for h in HEADERS)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w\s\*]*?\b(kgs_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    kbuild.build()
    return solver.load_library()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["kgs_create", "kgs_create_ex", "kgs_set_state", "kgs_get_state",
                     "kgs_step", "kgs_energy", "kgs_mass", "kgs_invariants", "kgs_destroy",
                     "kgs_set_tau", "kgs_strerror", "kgs_last_error", "kgs_last_status"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert names
    for n in names:
        assert hasattr(lib, n), n
        assert n in solver.SIGNATURES, f"binding lacks {n}"


def test_debug_bounds_library_exports_the_same_abi():
    """The index-checking build (KGS_DEBUG_BOUNDS) exports every declared
    function too, and kgs_debug_bounds tells the two builds apart without a
    GPU call reaching a device (the normal build answers 0 before any)."""
    path = kbuild.build(debug_bounds=True)
    dbg = ctypes.CDLL(path)
    for n in declared_functions():
        assert hasattr(dbg, n), n
    out = os.popen(f"/usr/local/cuda/bin/cuobjdump --list-elf {path} 2>&1").read()
    assert "sm_103a" in out


def test_library_is_built_for_sm103a(lib):
    out = os.popen(f"/usr/local/cuda/bin/cuobjdump --list-elf {kbuild.LIB} 2>&1").read()
    assert "sm_103a" in out


@pytest.mark.parametrize("args,status", [
    ((0, 16, 1.0, 1, 1, 1, 1, 0.1), -1),          # dim
    ((4, 16, 1.0, 1, 1, 1, 1, 0.1), -1),
    ((2, 15, 1.0, 1, 1, 1, 1, 0.1), -2),          # odd N
    ((2, 2, 1.0, 1, 1, 1, 1, 0.1), -2),           # N < 4
    ((1, (1 << 30) + 2, 1.0, 1, 1, 1, 1, 0.1), -7),  # too large
    ((2, 65536, 1.0, 1, 1, 1, 1, 0.1), -7),
    ((3, 8192, 1.0, 1, 1, 1, 1, 0.1), -7),
    ((2, 16, 0.0, 1, 1, 1, 1, 0.1), -1),          # L
    ((2, 16, -1.0, 1, 1, 1, 1, 0.1), -1),
    ((2, 16, 1.0, float("nan"), 1, 1, 1, 0.1), -1),
    ((2, 16, 1.0, 1, float("inf"), 1, 1, 0.1), -1),
    ((2, 16, 1.0, 1, 1, 1, 1, 0.0), -1),          # tau
    ((2, 16, 1.0, 1, 1, 1, 1, float("nan")), -1),
])
def test_create_rejects_invalid_arguments(lib, args, status):
    h = lib.kgs_create(*args)
    assert not h
    assert lib.kgs_last_status() == status
    assert lib.kgs_last_error()


def test_create_rejects_bad_precision(lib):
    assert not lib.kgs_create_ex(2, 16, 1.0, 1, 1, 1, 1, 0.1, 16, -1)
    assert lib.kgs_last_status() == -1


def test_null_handle_calls_fail_cleanly(lib):
    out = (ctypes.c_double * 3)()
    assert lib.kgs_step(None, 1, None) == -1
    assert lib.kgs_invariants(None, ctypes.cast(out, ctypes.POINTER(ctypes.c_double)), None) == -1
    assert lib.kgs_set_tau(None, 0.1) == -1
    assert lib.kgs_set_state(None, None, None, None, None, 0, None) == -1
    assert lib.kgs_launch_count(None) == -1
    lib.kgs_destroy(None)


def test_strerror_covers_every_status(lib):
    for st in range(0, -8, -1):
        assert lib.kgs_strerror(st) and lib.kgs_strerror(st) != b"unknown status"
    assert lib.kgs_strerror(-99) == b"unknown status"


def test_valid_create_without_gpu_fails_loudly(lib):
    """No CPU fallback: with no device, a valid problem is refused with
    KGS_ERR_CUDA (on a GPU machine this test is skipped)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    h = lib.kgs_create(2, 16, 1.0, 1, 1, 1, 1, 0.1)
    assert not h
    assert lib.kgs_last_status() == -4
    with pytest.raises(solver.KGSError):
        solver.Solver(2, 16, 1.0, 1, 1, 1, 1, 0.1)


def test_binding_constants_match_the_header():
    """Every KGS_* constant the Python binding defines has the value
    include/kgs.h gives it."""
    text = open(HEADERS[0]).read()
    defines = {m.group(1): int(m.group(2))
               for m in re.finditer(r"^#define\s+(KGS_\w+)\s+(-?\d+)\b", text, flags=re.M)}
    names = [n for n in dir(solver) if n.startswith("KGS_")]
    assert len(names) > 10
    for n in names:
        assert n in defines, f"{n} not in kgs.h"
        assert getattr(solver, n) == defines[n], n
