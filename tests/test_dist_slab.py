"""One grid shared by several ranks as axis-0 slabs (the multi-GPU design of
the colour passes), with gloo ranks on the CPU: the partition, the halo
exchange before every fused colour pass and the all-reduce of the invariants
reproduce the oracle's whole-grid run.  The per-slab pass here is a plain
vectorised numpy restatement of the pointwise update (Eq. scheme1 and its
adjoint, in the colour-pass fusion kgs_step uses), standing in for the GPU
kernels, so the test checks the host logic, not the kernels."""
import os

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2502_09537_b300 import dist as kdist
from paper_2502_09537_b300.inputs import Problem, random_state


def test_slab_partition():
    for N, world in [(10, 3), (64, 4), (7, 7), (9, 1)]:
        parts = kdist.slab_planes(N, world)
        assert sum(n for _, n in parts) == N
        assert [p for p, _ in parts] == list(np.cumsum([0] + [n for _, n in parts])[:-1])
        assert max(n for _, n in parts) - min(n for _, n in parts) <= 1
    with pytest.raises(ValueError):
        kdist.slab_planes(4, 5)
    assert kdist.fused_pass_sequence(1) == [0, 1, 3]
    assert kdist.fused_pass_sequence(3) == [0, 1, 2, 1, 2, 1, 3]


def _coef(prob):
    dim, N, L, k1, k2, mu, gamma, tau = prob
    s, h2 = tau / 2.0, (L / N) ** 2
    beta = s * k1 / (2 * h2)
    A = dim * s * k2 / h2 + s * mu * mu / 2
    return dict(s=s, beta=beta, alpha=dim * beta, g=s * gamma / 2, A=A, B=s * k2 / h2, E=s * gamma,
                det=1 + A * s / 2)


def _nsum(F, n, dim):
    """Sum over the 2d neighbours of the slab's planes 1..n (halo planes 0, n+1)."""
    S = F[0:n] + F[2:n + 2]
    for ax in range(1, dim):
        S = S + np.roll(F[1:n + 1], 1, axis=ax) + np.roll(F[1:n + 1], -1, axis=ax)
    return S


def _red_mask(slab):
    idx = np.indices((slab.n,) + (slab.N,) * (slab.dim - 1))
    total = idx.sum(axis=0) + slab.p0 + slab.dim
    return (total % 2) == 1          # red: 1-based index sum odd


def _numpy_pass(prob):
    c = _coef(prob)

    def psi(P, Q, U, SP, SQ, m):
        r = c["alpha"] - c["g"] * U
        z = P + 1j * Q
        dz = (2 * r * z - c["beta"] * (SP + 1j * SQ)) / (1j - r)
        P[m] += dz.real[m]
        Q[m] += dz.imag[m]

    def uv(P, Q, U, V, SU, m):
        rho = P * P + Q * Q
        rhs = c["B"] * SU - 2 * c["A"] * U - c["A"] * c["s"] * V + c["E"] * rho
        dV = rhs / c["det"]
        dU = c["s"] * V + c["s"] / 2 * dV
        U[m] += dU[m]
        V[m] += dV[m]

    def pass_fn(mode, slab, P, Q, U, V):
        n, dim = slab.n, slab.dim
        Pa, Qa, Ua, Va = (x.numpy() for x in (P, Q, U, V))
        SP, SQ, SU = _nsum(Pa, n, dim), _nsum(Qa, n, dim), _nsum(Ua, n, dim)
        red = _red_mask(slab)
        m = ~red if mode == kdist.PASS_BLACK_FUSED else red
        p, q, u, v = Pa[1:n + 1], Qa[1:n + 1], Ua[1:n + 1], Va[1:n + 1]

        def base():
            psi(p, q, u, SP, SQ, m)
            uv(p, q, u, v, SU, m)

        def adjoint():
            uv(p, q, u, v, SU, m)
            psi(p, q, u, SP, SQ, m)

        if mode == kdist.PASS_RED_BASE:
            base()
        elif mode == kdist.PASS_BLACK_FUSED:
            base()
            adjoint()
        elif mode == kdist.PASS_RED_FUSED:
            adjoint()
            base()
        else:
            adjoint()

    return pass_fn


def _numpy_partials(prob):
    dim, N, L, k1, k2, mu, gamma, _ = prob
    h = L / N

    def partial_fn(slab, P, Q, U, V):
        n = slab.n
        Pa, Qa, Ua, Va = (x.numpy() for x in (P, Q, U, V))
        p, q, u, v = Pa[1:n + 1], Qa[1:n + 1], Ua[1:n + 1], Va[1:n + 1]
        gp = (Pa[2:n + 2] - p) ** 2 + (Qa[2:n + 2] - q) ** 2
        gu = (Ua[2:n + 2] - u) ** 2
        for ax in range(1, dim):
            gp = gp + (np.roll(p, -1, axis=ax) - p) ** 2 + (np.roll(q, -1, axis=ax) - q) ** 2
            gu = gu + (np.roll(u, -1, axis=ax) - u) ** 2
        t1, t2 = 0.5 * k1 * gp / h ** 2, 0.5 * k2 * gu / h ** 2
        t34 = 0.5 * (v * v + mu * mu * u * u)
        rho = p * p + q * q
        t5 = gamma * rho * u
        hd = h ** dim
        return (hd * float(np.sum(t1 + t2 + t34 - t5)),
                hd * float(np.sum(np.abs(t1) + np.abs(t2) + t34 + np.abs(t5))),
                hd * float(np.sum(rho)))

    return partial_fn


def _worker(rank, world, port, prob, nsteps, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    st = random_state(prob, 2502_09537 + 500 + prob.dim, 0.6)
    slab = kdist.Slab(prob.dim, prob.N, rank, world)
    P, Q, U, V = (slab.take(torch.from_numpy(a.copy())) for a in st)
    slab.run(P, Q, U, V, nsteps, _numpy_pass(prob))
    inv = slab.invariants(P, Q, U, V, _numpy_partials(prob))
    out.put((rank, slab.p0, [x[1:slab.n + 1].numpy().copy() for x in (P, Q, U, V)], inv))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [1, 2, 3])
@pytest.mark.parametrize("dim,N", [(2, 12), (3, 6), (2, 10)])
def test_slabs_reproduce_the_whole_grid(orc, dim, N, world):
    """(2, 10) on 3 ranks: slabs of 4, 3 and 3 planes, so the ranks' first
    planes differ in parity and the colouring must come from global indices."""
    prob = Problem(dim, N, 7.0, 1.1, 0.9, 1.2, 0.8, 0.02)
    nsteps = 9
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29600 + (os.getpid() + 17 * world + 5 * dim + N) % 900
    procs = [ctx.Process(target=_worker, args=(r, world, port, prob, nsteps, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got = [np.concatenate([r[2][f] for r in res], axis=0) for f in range(4)]
    want = [a.copy() for a in random_state(prob, 2502_09537 + 500 + dim, 0.6)]
    orc.steps_checkerboard(prob, *want, nsteps)
    err = max(np.abs(x - y).max() / np.abs(y).max() for x, y in zip(got, want))
    assert err <= 1e-12, err
    Eo, So, Mo = orc.invariants(prob, *want)
    for _, _, _, (E, S, M) in res:       # every rank holds the reduced sums
        assert abs(E - Eo) <= 1e-13 * So and abs(S - So) <= 1e-13 * So and abs(M - Mo) <= 1e-13 * Mo
