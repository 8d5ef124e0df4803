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
