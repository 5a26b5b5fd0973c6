"""The Sec. 5.1 accuracy example against an independent solution of Eq. (kgs).

Reference: a Fourier pseudo-spectral solution of the continuous equations
(not the oracle's central differences) on a 128^2 grid of the same periodic
box, advanced with Lawson's integrating-factor RK4 (linear Schroedinger and
Klein-Gordon parts exact in Fourier space, the coupling terms by RK4),
dt = 2e-3; halving dt or refining to 192^2 changes it by < 2e-10.

Pin: the oracle (lexicographic order, the one whose accuracy does not carry
the checkerboard's (tau/h^2)^2 term) converges to it at order 2 along the
paper's (h, tau) sequence (h0, tau0) = (5/16, 1/50) halved twice.

The printed values of Table conv2d (tests/golden/conv2d_table.txt) are not
reproduced: at h0 the oracle's error is purely spatial (unchanged with
tau/16) and equals 2.34e-2 (u) and 1.06e-1 (psi) against the printed 7.54e-2
and 7.62e-2; every scheme of that table shares the 5-point central-difference
space discretisation, so the printed experiment must differ from its stated
setup.  The test records the ratios and bounds them loosely (factor 4)."""
import math
import os

import numpy as np

from paper_2502_09537_b300.inputs import Problem, coords, paper_exp1_2d

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "conv2d_table.txt")


def spectral_reference(N=128, T=1.0, dt=2e-3, L=20.0):
    """Fourier pseudo-spectral + Lawson IF-RK4 solution of Eq. (kgs) with
    kappa1 = kappa2 = mu = gamma = 1 from the Sec. 5.1 initial data; returns
    the Fourier coefficients (psi, u, u_t) at time T."""
    k1 = k2 = mu = g = 1.0
    prob = Problem(2, N, L, k1, k2, mu, g, dt)
    x, y = coords(prob)
    r2 = x * x + y * y
    psi = (1 + 1j) * np.exp(-r2)
    u = np.tanh(r2) + 0 * x
    v = np.sin(x + y) * np.exp(-2 * r2)
    k = 2 * np.pi * np.fft.fftfreq(N, d=L / N)
    KX, KY = np.meshgrid(k, k, indexing="ij")
    K2 = KX ** 2 + KY ** 2
    om = np.sqrt(k2 * K2 + mu ** 2)
    X = [np.fft.fft2(psi), np.fft.fft2(u), np.fft.fft2(v)]

    def E(s, P, U, V):  # exact flow of the linear parts over time s
        c, sn = np.cos(om * s), np.sin(om * s)
        return [P * np.exp(-1j * (k1 / 2) * K2 * s), c * U + sn / om * V, -om * sn * U + c * V]

    def nonlinear(P, U, V):
        ps = np.fft.ifft2(P)
        uu = np.fft.ifft2(U).real
        return [np.fft.fft2(1j * g * uu * ps), 0 * U, np.fft.fft2(g * np.abs(ps) ** 2)]

    def axpy(A, a, B):
        return [p + a * q for p, q in zip(A, B)]

    for _ in range(int(round(T / dt))):
        a1 = nonlinear(*X)
        a2 = nonlinear(*E(dt / 2, *axpy(X, dt / 2, a1)))
        a3 = nonlinear(*axpy(E(dt / 2, *X), dt / 2, a2))
        a4 = nonlinear(*axpy(E(dt, *X), dt, E(dt / 2, *a3)))
        e1 = E(dt, *a1)
        e23 = E(dt / 2, *[p + q for p, q in zip(a2, a3)])
        X = [x0 + dt / 6 * (p + 2 * q + r) for x0, p, q, r in zip(E(dt, *X), e1, e23, a4)]
    return X


def on_grid(F, N, Nf):
    """Spectral interpolation of Nf^2 Fourier coefficients onto an N^2 grid
    of the same box (N a multiple or a divisor of Nf)."""
    if N <= Nf:
        return np.fft.ifft2(F)[:: Nf // N, :: Nf // N]
    pad = np.zeros((N, N), complex)
    h = Nf // 2
    dst = np.r_[0:h, N - h:N]
    src = np.r_[0:h, Nf - h:Nf]
    pad[np.ix_(dst, dst)] = F[np.ix_(src, src)]
    return np.fft.ifft2(pad) * (N / Nf) ** 2


def test_exp1_second_order_against_spectral_solution(orc):
    P, U, _ = spectral_reference()
    printed = np.loadtxt(GOLDEN, comments="#")
    eu, ep = [], []
    for lev in range(3):
        N, tau = 64 * 2 ** lev, (1 / 50) / 2 ** lev
        w = paper_exp1_2d(N, tau)
        st = [a.copy() for a in w.state]
        orc.steps_order(w.prob, *st, np.arange(N * N), w.nsteps)
        psi_ref, u_ref = on_grid(P, N, 128), on_grid(U, N, 128).real
        hh = w.prob.h ** 2
        eu.append(math.sqrt(hh * np.sum((st[2] - u_ref) ** 2)))
        ep.append(max(math.sqrt(hh * np.sum((st[0] - psi_ref.real) ** 2)),
                      math.sqrt(hh * np.sum((st[1] - psi_ref.imag) ** 2))))
    ou = [math.log2(eu[i] / eu[i + 1]) for i in range(2)]
    op = [math.log2(ep[i] / ep[i + 1]) for i in range(2)]
    print("Err_u", eu, "orders", ou, "ratio to printed", np.array(eu) / printed[:, 1])
    print("Err_psi", ep, "orders", op, "ratio to printed", np.array(ep) / printed[:, 2])
    assert all(1.8 < o < 2.7 for o in ou + op), (ou, op)
    for mine, theirs in zip(eu + ep, list(printed[:, 1]) + list(printed[:, 2])):
        assert 0.25 < mine / theirs < 4.0
