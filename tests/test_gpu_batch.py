"""Parity of the batched analyses (enkf_ism_batch) with the oracle, per problem.

FP32 storage with FP64 level denominators, no refinement: the FP32 bars of
tests/bars.py per problem, Z within 1e-5 relative and M within 1e-4 (M = V^T Z is the
part of Z in range(V), damped by 1/gamma).  A batched problem returns Z and M only (no
X_A, hence no increment).  Every panel width the autotuner can pick is checked, the
captured graph is replayed on new data in place, and every one of the 8192 problems
of the full workload is checked once."""
import numpy as np
import pytest

import oracle
import synth
from tests import bars as B
from tests.util import rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1302_3876_gb300 import enkf  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    enkf.load(build_if_missing=True)


def run_batch(base, descs, out_floats, tune=False, force_widths=None, replay_same=False):
    plan, wsb = enkf.enkf_ism_batch_plan(descs)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    tin = torch.from_numpy(base).cuda()
    tout = torch.full((out_floats,), float("nan"), dtype=torch.float32, device="cuda")
    widths = None
    if tune:
        widths = enkf.enkf_ism_batch_autotune(plan, tin, tout, ws)
    st = enkf.enkf_ism_batch(plan, tin, tout, ws, sync=True)
    assert st == 0
    out = tout.cpu().numpy()
    if replay_same:
        tout.fill_(float("nan"))
        enkf.enkf_ism_batch(plan, tin, tout, ws, sync=True)
        np.testing.assert_array_equal(tout.cpu().numpy(), out)
    enkf.enkf_ism_batch_plan_destroy(plan)
    return out, widths


def check_problem(base, out, d):
    n, N = d["nobs"], d["nens"]
    r = base[d["r"]:d["r"] + n].astype(np.float64)
    V = base[d["V"]:d["V"] + n * N].astype(np.float64).reshape(N, n)
    D = base[d["D"]:d["D"] + n * N].astype(np.float64).reshape(N, n)
    Z, gamma = oracle.ism_solve_refined(r, V, D, return_gamma=True)
    M = oracle.vtz(V, Z)
    Zd = out[d["Z"]:d["Z"] + n * N].astype(np.float64).reshape(N, n)
    Md = out[d["M"]:d["M"] + N * N].astype(np.float64).reshape(N, N).T
    ez, em = rel(Zd, Z), rel(Md, M)
    B.check({"Z": ez, "M": em}, enkf.ENKF_FP32, label=f"problem nobs={n} nens={N} gamma_max={gamma.max():.0f}")
    return ez, em


def small_batch(nprob=96, seed=777):
    rng_n = synth.uniform(seed, 50, nprob, np.log(1.0), np.log(3000.0))
    nobs = np.maximum(1, np.rint(np.exp(rng_n))).astype(np.int64)
    choices = np.array([4, 8, 32, 64, 96, 128])
    nens = choices[(synth.u64(seed, 51, nprob) % np.uint64(len(choices))).astype(np.int64)]
    edge = [1, 2, 3, 31, 33, 4096][:nprob]
    nobs[:len(edge)] = edge
    return synth.batch_local_packed(nprob, seed, nens_override=nens, nobs_override=nobs)


def test_batch_default_widths():
    base, descs, nout = small_batch()
    out, _ = run_batch(base, descs, nout, replay_same=True)
    for d in descs:
        check_problem(base, out, d)


def test_batch_autotuned_widths_and_every_width(tmp_path, monkeypatch):
    base, descs, nout = small_batch(64, seed=778)
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("ENKF_AUTOTUNE_CACHE", str(cache))
    out, widths = run_batch(base, descs, nout, tune=True)
    assert all(w in (1, 8, 16, 32) for w in widths)
    assert cache.exists() and cache.read_text().strip()
    for d in descs:
        check_problem(base, out, d)
    # a new plan reads the cache; results stay within tolerance
    out2, _ = run_batch(base, descs, nout)
    for d in descs:
        check_problem(base, out2, d)


def test_batch_local_full_workload_every_problem():
    """The 8192-problem batched workload in one launch (the bench's launch configuration);
    every problem against the oracle, with the largest errors printed."""
    base, descs, nout = synth.batch_local_packed(8192)
    out, _ = run_batch(base, descs, nout)
    worst = {"Z": 0.0, "M": 0.0}
    for d in descs:
        ez, em = check_problem(base, out, d)
        worst["Z"], worst["M"] = max(worst["Z"], ez), max(worst["M"], em)
    print(f"batch_local, 8192 problems: largest errors Z {worst['Z']:.2e}, M {worst['M']:.2e}")


def test_batch_rejects_bad_descriptors():
    base, descs, nout = small_batch(4, seed=779)
    bad = [dict(d) for d in descs]
    bad[1]["nens"] = 6
    with pytest.raises(enkf.EnkfError) as e:
        enkf.enkf_ism_batch_plan(bad)
    assert e.value.status == enkf.ENKF_ERR_SHAPE
