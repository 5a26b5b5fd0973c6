"""B300-native DP-AVF2 checkerboard solver for the periodic Klein-Gordon-Schroedinger
equations (arXiv 2502.09537).

The compute path lives in ``libkgs.so`` (hand-written sm_103a CUDA behind a C ABI,
declared in ``include/kgs.h``); ``solver`` is a thin ctypes binding over it.
Importing this package does not load the library; ``solver`` does, and raises if
it is missing.
"""
