"""FP64 CPU oracle of the DP-AVF2 checkerboard scheme (arXiv 2502.09537).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library; see ``kgs_oracle.c`` for the
passages of the paper each function follows.
"""
from .oracle import (  # noqa: F401
    MUT_ADJ_LITERAL, MUT_NO_REVERSE, MUT_RHO_OLD_BASE, MUT_ALPHA_2D, MUT_NO_ADJ_SWAP,
    MUT_COLOUR_0BASED,
    checkerboard_order, steps_order, steps_orders2, steps_checkerboard, steps_checkerboard_omp,
    invariants, max_threads,
)
