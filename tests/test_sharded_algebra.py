"""The row-partitioned algebra of the analysis, on CPU ranks (two gloo processes).

The analysis shards by observation rows: each rank holds a contiguous block of the rows of V, D
and r, and the matching block of state rows (H takes every stride-th state row, so a block of
observations maps to a block of state rows with no halo).  Step 1 is local.  Each level needs only
the dots of v_k with the active columns, v_k^T [Z, u_k, u_{k+1..N}]: a 2N-vector summed over the
ranks (one all-reduce per level), after which every rank updates its own rows.  M = V^T Z /
sqrt(N - 1) is one N x N all-reduce, and X_A = X_B + dX_B M is local.  This test runs that
partitioned recurrence with numpy on each rank and gloo all-reduces in FP64, and checks the gathered
Z, gamma, M and X_A against the FP64 oracle of the whole problem.  It is the algebra a row-sharded
multi-GPU analysis would run; the library itself runs one GPU per analysis (replicas)."""
import math
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NSTATE, STRIDE, NENS, SEED = 150, 3, 7, 8080
NOBS = (NSTATE - 1) // STRIDE + 1


def _problem():
    import synth
    dXB = synth.normal_matrix(SEED, 1, NSTATE, NENS, row_scale=synth.uniform(SEED, 2, NSTATE, 0.5, 2.0))
    XB = dXB + 3.0
    r = synth.uniform(SEED, 3, NOBS, 0.5, 1.5)
    D = synth.normal_matrix(SEED, 4, NOBS, NENS)
    return XB, dXB, r, D


def _allreduce(x):
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.numpy()


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    XB, dXB, r, D = _problem()
    # observation rows [j0, j1) of this rank; state rows [j0 * stride, j1 * stride) (the last rank
    # also takes the trailing unobserved state rows)
    per = (NOBS + world - 1) // world
    j0, j1 = rank * per, min(NOBS, (rank + 1) * per)
    i0, i1 = j0 * STRIDE, (NSTATE if rank == world - 1 else j1 * STRIDE)
    scale = 1.0 / math.sqrt(NENS - 1)
    V = dXB[:, i0:i1:STRIDE][:, : j1 - j0] * scale          # (N, local nobs): H dX_B / sqrt(N - 1)
    Dl, rl = D[:, j0:j1], r[j0:j1]
    U, Z = V / rl, Dl / rl                                   # Step 1 (eq. SM-step-1), local rows
    gamma = np.zeros(NENS)
    for k in range(NENS):                                    # Step 2 (eqs. SM-step-2-*)
        part = np.concatenate([[V[k] @ U[k]], Z @ V[k], U[k + 1:] @ V[k]])
        tot = _allreduce(part)                               # the level's one exchange
        gamma[k] = 1.0 + tot[0]
        h = U[k] / gamma[k]
        Z = Z - np.outer(tot[1:1 + NENS], h)
        U[k + 1:] = U[k + 1:] - np.outer(tot[1 + NENS:], h)
    M = _allreduce(V @ Z.T) * scale                          # M[m, e] = v_m^T z_e / sqrt(N - 1)
    XA = XB[:, i0:i1] + M.T @ dXB[:, i0:i1]                  # X_A = X_B + dX_B M, local state rows
    zs = [None] * world
    xs = [None] * world
    dist.all_gather_object(zs, Z)
    dist.all_gather_object(xs, XA)
    if rank == 0:
        q.put((np.concatenate(zs, axis=1), np.concatenate(xs, axis=1), gamma, M))
    dist.destroy_process_group()


def test_row_sharded_recurrence_matches_the_oracle():
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 31500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(rk, 2, port, q)) for rk in range(2)]
    for p in procs:
        p.start()
    Z, XA, gamma, M = q.get(timeout=180)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    XB, dXB, r, D = _problem()
    V = oracle.observe_deviations(dXB, NOBS, STRIDE)
    ref = oracle.analysis(r, V, D, XB, dXB)
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)  # noqa: E731
    assert rel(Z, ref["Z"]) <= 1e-12
    np.testing.assert_allclose(gamma, ref["gamma"], rtol=1e-12)
    assert rel(M, ref["M"]) <= 1e-12
    assert rel(XA, ref["XA"]) <= 1e-12


def _panel_worker(rank, world, port, q, b):
    """The panel form of the recurrence (b levels per exchange): per panel P the ranks sum
    G = V_P^T U_P (b x b) and A = V_P^T [U_trailing, Z] (b x ncols) in one all-reduce; the b x b
    factor is then the same on every rank (gamma_m = 1 + (G beta_m)_m, h_m = U_P beta_m / gamma_m,
    beta_j -= (beta_m / gamma_m)(G beta_j)_m), and each rank applies X -= U_P B (I + L)^{-1} A to its
    rows, L the strictly lower part of G B."""
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    XB, dXB, r, D = _problem()
    per = (NOBS + world - 1) // world
    j0, j1 = rank * per, min(NOBS, (rank + 1) * per)
    scale = 1.0 / math.sqrt(NENS - 1)
    V = dXB[:, j0 * STRIDE:NSTATE:STRIDE][:, : j1 - j0] * scale
    Dl, rl = D[:, j0:j1], r[j0:j1]
    U, Z = V / rl, Dl / rl
    gamma = np.zeros(NENS)
    for k0 in range(0, NENS, b):
        bp = min(b, NENS - k0)
        P = slice(k0, k0 + bp)
        X = np.concatenate([U[k0 + bp:], Z])                 # trailing columns of U, then Z
        red = _allreduce(np.concatenate([(V[P] @ U[P].T).ravel(), (V[P] @ X.T).ravel()]))
        G = red[: bp * bp].reshape(bp, bp)                   # G[l, m] = v_l^T u_m
        A = red[bp * bp:].reshape(bp, X.shape[0])            # A[l, c] = v_l^T x_c
        beta = np.eye(bp)                                    # u_m (current) = U_P beta[:, m]
        B = np.zeros((bp, bp))
        for m in range(bp):
            gamma[k0 + m] = 1.0 + (G @ beta[:, m])[m]
            B[:, m] = beta[:, m] / gamma[k0 + m]
            for j in range(m + 1, bp):
                beta[:, j] -= B[:, m] * (G @ beta[:, j])[m]
        L = np.tril(G @ B, -1)
        C = np.linalg.solve(np.eye(bp) + L, A)               # the level coefficients c = (I + L)^{-1} a
        X = X - (U[P].T @ (B @ C)).T
        U[k0 + bp:] = X[: NENS - k0 - bp]
        Z = X[NENS - k0 - bp:]
    zs = [None] * world
    dist.all_gather_object(zs, Z)
    if rank == 0:
        q.put((np.concatenate(zs, axis=1), gamma))
    dist.destroy_process_group()


@pytest.mark.parametrize("b", [1, 3, 7])
def test_row_sharded_panel_recurrence_matches_the_oracle(b):
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 32500 + (os.getpid() + 17 * b) % 1000
    procs = [ctx.Process(target=_panel_worker, args=(rk, 2, port, q, b)) for rk in range(2)]
    for p in procs:
        p.start()
    Z, gamma = q.get(timeout=180)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    XB, dXB, r, D = _problem()
    V = oracle.observe_deviations(dXB, NOBS, STRIDE)
    Zref, gref = oracle.ism_solve(r, V, D, return_gamma=True)
    assert np.linalg.norm(Z - Zref) / np.linalg.norm(Zref) <= 1e-12
    np.testing.assert_allclose(gamma, gref, rtol=1e-12)
