"""Row-sharded analysis through the C ABI (enkf_rows_*): two ranks, each holding a block of
observation rows and a block of state rows on the same GPU, exchange the dots of every
level of Step 2 (Sec. 3.1, eqs. SM-step-2-h/Z/u) and the final Gram over gloo (host
round trips), and their Z, gamma, M and X_A are compared with the FP64 oracle of the
whole problem.  No kernel waits on another rank: every exchange happens on the host
between launches.  Bars as for the plain paths (tests/bars.py): FP64 1e-10 on every
result; FP32 1e-5 on Z and X_A, 1e-4 on M and the increment."""
import math
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SEED = 21302
STRIDE = 3


def _problem(nobs, nens):
    sys.path.insert(0, ROOT)
    import synth
    nstate = nobs * STRIDE + 2
    s = synth.uniform(SEED, 1, nstate, 0.5, 2.0)
    dXB = synth.normal_matrix(SEED, 2, nstate, nens, row_scale=s)
    XB = dXB + 2.0
    r = synth.uniform(SEED, 3, nobs, 0.5, 1.5)
    D = synth.normal_matrix(SEED, 4, nobs, nens)
    V = dXB[:, ::STRIDE][:, :nobs] / math.sqrt(nens - 1)
    return XB, dXB, r, D, V


def _worker(rank, world, port, nobs, nens, split, dtype_name, outdir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_1302_3876_gb300 import enkf, sharded
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    enkf.load(build_if_missing=False)
    dt = {"fp64": (np.float64, torch.float64), "fp32": (np.float32, torch.float32)}[dtype_name]
    XB, dXB, r, D, V = _problem(nobs, nens)
    nstate = dXB.shape[1]
    # observation rows [j0, j1) of this rank; state rows [i0, i1) (an uneven split of each)
    j0, j1 = (0, split) if rank == 0 else (split, nobs)
    i0, i1 = (0, split * STRIDE + 1) if rank == 0 else (split * STRIDE + 1, nstate)
    dev = torch.device("cuda", 0)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a.astype(dt[0]))).to(dev)  # noqa: E731

    def all_reduce(x):
        h = x.cpu()
        dist.all_reduce(h, op=dist.ReduceOp.SUM)
        x.copy_(h)

    XA = torch.empty(nens, i1 - i0, dtype=dt[1], device=dev)
    out = sharded.sharded_analysis(t(r[j0:j1]), t(V[:, j0:j1]), t(D[:, j0:j1]), t(dXB[:, i0:i1]), t(XB[:, i0:i1]),
                                   XA, all_reduce)
    torch.cuda.synchronize()
    np.savez(os.path.join(outdir, f"rank{rank}.npz"), Z=out["Z"].double().cpu().numpy(),
             XA=XA.double().cpu().numpy(), M=out["M"].double().cpu().numpy().reshape(nens, nens).T,
             gamma=out["gamma"].cpu().numpy())
    dist.barrier()
    dist.destroy_process_group()


def _run(nobs, nens, split, dtype_name, tmp_path):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    port = 32500 + (os.getpid() + nobs + nens) % 1000
    procs = [ctx.Process(target=_worker, args=(rk, 2, port, nobs, nens, split, dtype_name, str(tmp_path)))
             for rk in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    parts = [np.load(os.path.join(tmp_path, f"rank{rk}.npz")) for rk in range(2)]
    return {"Z": np.concatenate([p["Z"] for p in parts], axis=1),
            "XA": np.concatenate([p["XA"] for p in parts], axis=1),
            "M": parts[0]["M"], "M1": parts[1]["M"], "gamma": parts[0]["gamma"]}


@pytest.mark.parametrize("dtype_name,nobs,nens,split", [("fp64", 3001, 24, 1025), ("fp64", 700, 96, 333),
                                                        ("fp32", 3001, 24, 1025), ("fp32", 5000, 64, 4097)])
def test_two_ranks_match_the_oracle(dtype_name, nobs, nens, split, tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1302_3876_gb300 import enkf
    from tests import bars as B
    from tests.util import rel
    enkf.load(build_if_missing=True)           # build before the ranks start
    got = _run(nobs, nens, split, dtype_name, tmp_path)
    XB, dXB, r, D, V = _problem(nobs, nens)
    npdt = np.float64 if dtype_name == "fp64" else np.float32
    rd = lambda a: a.astype(npdt).astype(np.float64)  # noqa: E731
    XBr, dXr, rr, Dr, Vr = rd(XB), rd(dXB), rd(r), rd(D), rd(V)
    Z, gamma = oracle.ism_solve_refined(rr, Vr, Dr, return_gamma=True)
    M = oracle.vtz(Vr, Z)
    XA = oracle.analysis_update(XBr, dXr, M)
    errs = {"Z": rel(got["Z"], Z), "M": rel(got["M"], M), "XA": rel(got["XA"], XA),
            "increment": rel(got["XA"] - XBr, XA - XBr)}
    print(f"sharded {dtype_name} nobs={nobs} nens={nens} split={split}: " +
          ", ".join(f"{k} {v:.2e}" for k, v in errs.items()))
    mode = enkf.ENKF_FP64 if dtype_name == "fp64" else enkf.ENKF_FP32
    B.check(errs, mode, label=f"sharded {dtype_name}")
    np.testing.assert_allclose(got["gamma"], gamma, rtol=1e-12 if dtype_name == "fp64" else 1e-5)
    assert np.array_equal(got["M"], got["M1"])       # every rank assembles the same M
