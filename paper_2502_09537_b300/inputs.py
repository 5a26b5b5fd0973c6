"""Seeded synthetic initial data shaped like the paper's workloads.

This module holds no arithmetic of the DP-AVF2 scheme: it only evaluates
initial conditions on the grid and draws seeded noise.  It is the one module
both the CUDA path's tests and the CPU oracle's tests take inputs from.

Grid (Sec. 2 of arXiv 2502.09537): N points per direction on the periodic
domain [-L/2, L/2)^d, x_j = -L/2 + j h, h = L/N, j = 0..N-1.  Arrays are
float64, C order, shape (N,)*d, index [ix][iy][iz].

Noise is drawn with numpy's PCG64, seed = 2502_09537 + config index, in the
field order P, Q, U, V.
"""
from __future__ import annotations

import math
from typing import Callable, List, NamedTuple, Tuple

import numpy as np

SEED_BASE = 2502_09537


class Problem(NamedTuple):
    """Parameters of one periodic KGS problem (Eq. kgs): dimension, points per
    direction, period L, kappa1, kappa2, mu, gamma and the time step tau."""
    dim: int
    N: int
    L: float
    kappa1: float
    kappa2: float
    mu: float
    gamma: float
    tau: float

    @property
    def h(self) -> float:
        return self.L / self.N

    @property
    def points(self) -> int:
        return self.N ** self.dim


class Workload(NamedTuple):
    name: str
    prob: Problem
    nsteps: int
    state: Tuple[np.ndarray, np.ndarray, np.ndarray, np.ndarray]  # P, Q, U, V


def coords(prob: Problem) -> List[np.ndarray]:
    """Open-mesh coordinate arrays x, y, z (broadcastable to (N,)*d)."""
    x = -prob.L / 2 + prob.h * np.arange(prob.N, dtype=np.float64)
    out = []
    for a in range(prob.dim):
        shape = [1] * prob.dim
        shape[a] = prob.N
        out.append(x.reshape(shape))
    return out


def _full(a, prob):
    return np.array(np.broadcast_to(a, (prob.N,) * prob.dim), dtype=np.float64, order="C", copy=True)


def _r2(prob: Problem) -> np.ndarray:
    r2 = 0.0
    for c in coords(prob):
        r2 = r2 + c * c
    return r2


def _add_noise(fields, rng, kind: str, amp: float):
    out = []
    for f in fields:
        if kind == "uniform":
            n = rng.uniform(-amp, amp, size=f.shape)
        else:
            n = rng.normal(0.0, amp, size=f.shape)
        out.append(np.ascontiguousarray(f + n))
    return tuple(out)


def soliton_1d(N: int = 512, nsteps: int = 2000, noise: bool = True) -> Workload:
    """1D, x in [-40,40), kappas = mu = gamma = 1, tau = 1e-3:
    psi0 = 1.5 sech^2(x/sqrt2) e^{0.5 i x}, u0 = -0.75 sech^2(x/sqrt2), v0 = 0,
    plus uniform noise of amplitude 1e-4 on every field (config index 0)."""
    prob = Problem(1, N, 80.0, 1.0, 1.0, 1.0, 1.0, 1e-3)
    (x,) = coords(prob)
    s2 = 1.0 / np.cosh(x / math.sqrt(2.0)) ** 2
    P = 1.5 * s2 * np.cos(0.5 * x)
    Q = 1.5 * s2 * np.sin(0.5 * x)
    U = -0.75 * s2
    V = np.zeros_like(x)
    fields = tuple(_full(f, prob) for f in (P, Q, U, V))
    if noise:
        rng = np.random.Generator(np.random.PCG64(SEED_BASE + 0))
        fields = _add_noise(fields, rng, "uniform", 1e-4)
    return Workload(f"kgs1d_soliton_N{N}", prob, nsteps, fields)


def gauss_2d(N: int = 2048, nsteps: int = 1000, noise: bool = True) -> Workload:
    """2D, [-20,20)^2, all parameters 1, tau = 1e-3:
    psi0 = (1+i) exp(-(x^2+y^2)), u0 = exp(-(x^2+y^2)), v0 = 0, plus Gaussian
    noise sigma = 1e-4 (config index 1)."""
    prob = Problem(2, N, 40.0, 1.0, 1.0, 1.0, 1.0, 1e-3)
    g = np.exp(-_r2(prob))
    fields = tuple(_full(f, prob) for f in (g, g, g, 0.0 * g))
    if noise:
        rng = np.random.Generator(np.random.PCG64(SEED_BASE + 1))
        fields = _add_noise(fields, rng, "normal", 1e-4)
    return Workload(f"kgs2d_gauss_N{N}", prob, nsteps, fields)


def gauss_3d(N: int = 512, nsteps: int = 200, noise: bool = True) -> Workload:
    """3D, [-10,10)^3, all parameters 1, tau = 5e-4:
    psi0 = (1+i) exp(-|x|^2), u0 = exp(-|x|^2), v0 = 0, plus Gaussian noise
    sigma = 1e-4 (config index 2)."""
    prob = Problem(3, N, 20.0, 1.0, 1.0, 1.0, 1.0, 5e-4)
    g = np.exp(-_r2(prob))
    fields = tuple(_full(f, prob) for f in (g, g, g, np.zeros(1)))
    if noise:
        rng = np.random.Generator(np.random.PCG64(SEED_BASE + 2))
        fields = _add_noise(fields, rng, "normal", 1e-4)
    return Workload(f"kgs3d_gauss_N{N}", prob, nsteps, fields)


def paper_exp1_2d(N: int, tau: float, t_end: float = 1.0) -> Workload:
    """Sec. 5.1 accuracy example: Omega = (-10,10)^2, kappas = gamma = mu = 1,
    psi0 = (1+i) e^{-(x^2+y^2)}, u0 = tanh(x^2+y^2), v0 = sin(x+y) e^{-2(x^2+y^2)}."""
    prob = Problem(2, N, 20.0, 1.0, 1.0, 1.0, 1.0, tau)
    x, y = coords(prob)
    r2 = x * x + y * y
    g = np.exp(-r2)
    fields = tuple(_full(f, prob) for f in (g, g, np.tanh(r2), np.sin(x + y) * np.exp(-2 * r2)))
    return Workload(f"paper_exp1_N{N}", prob, int(round(t_end / tau)), fields)


def paper_exp2_bumps_2d(N: int, tau: float = 0.01, nsteps: int = 100) -> Workload:
    """Sec. 5.1 parallel example: four bumps at (0,-3), (3,0), (0,3), (-3,0) on
    (-10,10)^2, kappas = gamma = mu = 0.5."""
    prob = Problem(2, N, 20.0, 0.5, 0.5, 0.5, 0.5, tau)
    x, y = coords(prob)
    P = 0.0
    U = 0.0
    for (cx, cy) in ((0.0, -3.0), (3.0, 0.0), (0.0, 3.0), (-3.0, 0.0)):
        d2 = (x - cx) ** 2 + (y - cy) ** 2
        P = P + np.exp(-d2)
        U = U + np.tanh(d2)
    V = np.exp(-x * x - y * y)
    fields = tuple(_full(f, prob) for f in (P, P, U, V))
    return Workload(f"paper_exp2_N{N}", prob, nsteps, fields)


def paper_exp3_ellipsoids_3d(N: int, tau: float = 0.01, nsteps: int = 100) -> Workload:
    """Sec. 5.2 example: (-10,10)^3, kappa1 = -0.4, kappa2 = 0.1, gamma = 0.2,
    mu = 0.1; two shifted bumps in psi with a weak phase tilt, three in u."""
    prob = Problem(3, N, 20.0, -0.4, 0.1, 0.1, 0.2, tau)
    x, y, z = coords(prob)
    psi = 0.0
    for j in (0, 1):
        psi = psi + np.exp(-(x + 2 * (-1) ** j) ** 2 - y * y - z * z) * np.exp(0.01 * j * (x + y + z))
    U = np.exp(-x * x - y * y - (z - 2) ** 2)
    for j in (0, 1):
        U = U + np.exp(-(x + (-1) ** j * math.sqrt(3.0)) ** 2 - y * y - (z + 1) ** 2)
    V = np.exp(-x * x - y * y - z * z)
    fields = tuple(_full(f, prob) for f in (psi, 0.0 * psi, U, V))
    return Workload(f"paper_exp3_N{N}", prob, nsteps, fields)


def random_state(prob: Problem, seed: int, amp: float = 0.5) -> Tuple[np.ndarray, ...]:
    """Smooth-ish random state for small property tests: a few random Fourier
    modes per field plus white noise of amplitude amp/10."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cs = coords(prob)
    out = []
    for _ in range(4):
        f = np.zeros((prob.N,) * prob.dim)
        for _m in range(3):
            phase = rng.uniform(0, 2 * np.pi)
            arg = phase
            for c in cs:
                arg = arg + 2 * np.pi * rng.integers(-2, 3) * c / prob.L
            f = f + amp * rng.uniform(-1, 1) * np.cos(arg)
        f = f + (amp / 10) * rng.uniform(-1, 1, size=f.shape)
        out.append(np.ascontiguousarray(f))
    return tuple(out)


def gaussian_bump(prob: Problem, rng: np.random.Generator) -> Tuple[np.ndarray, ...]:
    """Gaussian-bump data with a random centre and width in [0.5, 2]."""
    cs = coords(prob)
    width = rng.uniform(0.5, 2.0)
    centre = rng.uniform(-prob.L / 4, prob.L / 4, size=prob.dim)
    d2 = 0.0
    for c, x0 in zip(cs, centre):
        d2 = d2 + (c - x0) ** 2
    g = np.exp(-d2 / (width * width))
    return tuple(_full(f, prob) for f in (g, 0.5 * g, g, 0.0 * g))


def batched_instances(seed: int = SEED_BASE + 3, steps: int = 500):
    """96 instances (config index 3): 64 2D grids with N from {128,...,2048}
    (step 128) on [-20,20)^2 and 32 3D grids with N from {64,96,...,256} on
    [-10,10)^3; kappa1, kappa2 ~ U[0.5,2], mu ~ U[0.5,1.5], gamma ~ U[0.5,2],
    tau = 5e-4.  Returns a list of (Problem, nsteps, state_fn) where state_fn()
    builds that instance's Gaussian-bump initial data."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(96):
        if k < 64:
            dim, N, L = 2, int(rng.choice(np.arange(128, 2049, 128))), 40.0
        else:
            dim, N, L = 3, int(rng.choice(np.arange(64, 257, 32))), 20.0
        prob = Problem(dim, N, L, float(rng.uniform(0.5, 2)), float(rng.uniform(0.5, 2)),
                       float(rng.uniform(0.5, 1.5)), float(rng.uniform(0.5, 2)), 5e-4)
        sub = int(rng.integers(0, 2 ** 62))
        out.append((prob, steps, _bump_fn(prob, sub)))
    return out


def _bump_fn(prob: Problem, sub_seed: int) -> Callable[[], Tuple[np.ndarray, ...]]:
    def fn():
        return gaussian_bump(prob, np.random.Generator(np.random.PCG64(sub_seed)))
    return fn
