"""Index checks on the GPU (the stand-in for a memory checker): tiny and
ragged grids through the colour-pass, streamed-plane and batch kernels of the
index-checking build (libkgs_debug.so, KGS_DEBUG_BOUNDS), in a child process
that loads that build; no check may fire, and the states equal the normal
build's bit for bit (the checks only add comparisons)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2502_09537_b300 import solver
from paper_2502_09537_b300.inputs import Problem, random_state
from paper_2502_09537_b300.solver import Batch, KGS_FP32, KGS_FP64, KGS_OPT_KERNEL, Solver
checking, flags0 = solver.debug_bounds()
cases = []
for dim, N in ((1, 4), (1, 6), (1, 130), (2, 4), (2, 6), (2, 66), (3, 4), (3, 6), (3, 18), (3, 64)):
    for prec in (KGS_FP64, KGS_FP32):
        for kernel in (1, 4, 5, 7, 8):
            if kernel == 5 and dim < 2:
                continue
            prob = Problem(dim, N, 5.0, 1.0, 0.9, 1.1, 1.2, 0.01)
            st = random_state(prob, 40 + N + dim, 0.5)
            with Solver.from_problem(prob, prec) as s:
                s.set_option(KGS_OPT_KERNEL, kernel)
                s.set_state(*st)
                s.step(3)
                cases.append(((dim, N, prec, kernel), [float(np.sum(np.abs(a))) for a in s.get_state()]))
with Batch(1 << 26) as b:
    probs = [(Problem(1, 6, 3.0, 1, 1, 1, 1, 0.01), KGS_FP64), (Problem(2, 10, 3.0, 1, 1, 1, 1, 0.01), KGS_FP32),
             (Problem(3, 6, 3.0, 1, 1, 1, 1, 0.01), KGS_FP64), (Problem(3, 8, 3.0, 1, 1, 1, 1, 0.01), KGS_FP32)]
    ids = [b.add(p, prec) for p, prec in probs]
    for i, (p, _) in zip(ids, probs):
        b.set_state(i, *random_state(p, 7 + i, 0.5))
    b.step_each([3, 0, 5, 2])
    for i in ids:
        cases.append((("batch", i), [float(np.sum(np.abs(a))) for a in b.get_state(i)]))
checking, flags = solver.debug_bounds()
print(json.dumps({"checking": checking, "flags0": flags0, "flags": flags, "lib": solver.LIB_PATH,
                  "cases": cases}))
"""


def run_child(lib_path):
    env = dict(os.environ, KGS_LIBRARY=lib_path)
    out = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-3000:]
    return json.loads(out.stdout.strip().splitlines()[-1])


def test_no_index_check_fires_and_states_match_the_normal_build():
    from paper_2502_09537_b300 import build as kbuild
    dbg = run_child(kbuild.build(debug_bounds=True))
    assert dbg["checking"] is True and dbg["lib"].endswith("libkgs_debug.so")
    assert dbg["flags0"] == 0 and dbg["flags"] == 0, dbg["flags"]
    ref = run_child(kbuild.build())
    assert ref["checking"] is False and ref["flags"] == 0
    assert len(dbg["cases"]) == len(ref["cases"])
    for (ka, va), (kb, vb) in zip(dbg["cases"], ref["cases"]):
        assert ka == kb and va == vb, (ka, va, vb)
