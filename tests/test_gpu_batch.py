"""Parity of the batched analyses (enkf_ism_batch) with the oracle, per problem.

FP32 storage with FP64 level denominators: Z within 1e-5 relative; M within
1e-5 * max(1, gamma_max/100) (M = V^T Z carries the conditioning of R + V V^T).
Every panel width the autotuner can pick is checked, and the captured graph is
replayed on new data in place."""
import numpy as np
import pytest

import oracle
import synth
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
    Z, gamma = oracle.ism_solve(r, V, D, return_gamma=True)
    M = oracle.vtz(V, Z)
    Zd = out[d["Z"]:d["Z"] + n * N].astype(np.float64).reshape(N, n)
    Md = out[d["M"]:d["M"] + N * N].astype(np.float64).reshape(N, N).T
    ez, em = rel(Zd, Z), rel(Md, M)
    assert ez <= 1e-5, (n, N, ez)
    assert em <= 1e-5 * max(1.0, gamma.max() / 100.0), (n, N, em, gamma.max())
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


def test_batch_local_full_workload_sampled():
    """The 8192-problem batched workload in one launch; a deterministic sample of
    problems (including the 16 most expensive) against the oracle."""
    base, descs, nout = synth.batch_local_packed(8192)
    out, _ = run_batch(base, descs, nout)
    cost = np.array([d["nobs"] * d["nens"] ** 2 for d in descs])
    idx = list(np.argsort(-cost)[:16]) + list(range(0, 8192, 97))
    for i in sorted(set(int(i) for i in idx)):
        check_problem(base, out, descs[i])


def test_batch_rejects_bad_descriptors():
    base, descs, nout = small_batch(4, seed=779)
    bad = [dict(d) for d in descs]
    bad[1]["nens"] = 6
    with pytest.raises(enkf.EnkfError) as e:
        enkf.enkf_ism_batch_plan(bad)
    assert e.value.status == enkf.ENKF_ERR_SHAPE
