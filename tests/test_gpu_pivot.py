"""Parity of the pivoted solve (Sec. 3.4, enkf_ism_solve_pivot) with the FP64 oracle of the same
recurrence, through the C ABI.  Z is unique (Theorem 3), so Z and M are compared at the plain
path's per-result bars (tests/bars.py: FP64 1e-10; FP32 Z 1e-5, M 1e-4 without refinement).
The pivoted solve returns Z and M only (no X_A, hence no increment).
In FP64 the pivot order and the gamma_k must equal the oracle's; in FP32 the candidates' gamma
carry FP32 rounding, so a near tie may be broken the other way: the order is checked to be a
permutation and each gamma_k >= 1."""
import math

import numpy as np
import pytest

import oracle
import synth
from tests import bars as B
from tests.util import host, rel, rounded, to_dev, vec_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1302_3876_gb300 import enkf  # noqa: E402

DT = {"fp64": (np.float64, torch.float64, 1e-10, enkf.ENKF_FP64),
      "fp32": (np.float32, torch.float32, 1e-5, enkf.ENKF_FP32)}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    enkf.load(build_if_missing=True)


def _problem(seed, nobs, nens, npt):
    r = rounded(synth.uniform(seed, 1, nobs, 0.5, 1.5), npt)
    V = rounded(synth.normal_matrix(seed, 2, nobs, nens, std=1.0 / math.sqrt(max(nens - 1, 1)),
                                    row_scale=synth.uniform(seed, 5, nobs, 0.2, 3.0)), npt)
    D = rounded(synth.normal_matrix(seed, 3, nobs, nens), npt)
    return r, V, D


def _run(prec, r, V, D, ld_pad=0):
    npt, tt, _, mode = DT[prec]
    nens, nobs = V.shape
    ws = torch.empty(max(enkf.enkf_ism_pivot_workspace(nobs, nens, mode), 256), dtype=torch.uint8, device="cuda")
    tV, tD = to_dev(V, npt, nobs + ld_pad), to_dev(D, npt, nobs + ld_pad)
    tZ = to_dev(np.zeros((nens, nobs)), npt, nobs + ld_pad)
    tM = torch.zeros(nens * nens, dtype=tt, device="cuda") if nens >= 2 else None
    tperm = torch.full((nens,), -1, dtype=torch.int32, device="cuda")
    tgam = torch.zeros(nens, dtype=torch.float64, device="cuda")
    st = enkf.enkf_ism_solve_pivot(vec_dev(r, npt), tV, tD, tZ, ws, M=tM, perm=tperm, gamma=tgam)
    torch.cuda.synchronize()
    out = {"status": st, "Z": host(tZ), "perm": tperm.cpu().numpy(), "gamma": tgam.cpu().numpy()}
    if tM is not None:
        out["M"] = host(tM).reshape(nens, nens).T
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("nobs,nens", [(1, 1), (33, 17), (1000, 32), (4099, 64), (20000, 128), (5000, 256)])
def test_pivoted_solve_matches_oracle(prec, nobs, nens):
    _, _, tol, _ = DT[prec]
    r, V, D = _problem(1700 + nobs + nens, nobs, nens, DT[prec][0])
    dev = _run(prec, r, V, D, ld_pad=3)
    Z, gamma, perm = oracle.ism_solve_pivot(r, V, D)
    assert dev["status"] == 0
    assert rel(dev["Z"], Z) <= tol
    if prec == "fp64":
        np.testing.assert_array_equal(dev["perm"], perm)
        np.testing.assert_allclose(dev["gamma"], gamma, rtol=1e-10)
    else:
        assert sorted(dev["perm"].tolist()) == list(range(nens))
        assert np.all(dev["gamma"] >= 1.0 - 1e-6)
        assert dev["gamma"].max() == pytest.approx(gamma.max(), rel=1e-4)
    if nens >= 2:
        M = oracle.vtz(V, Z)
        B.check({"Z": rel(dev["Z"], Z), "M": rel(dev["M"], M)},
                enkf.ENKF_FP64 if prec == "fp64" else enkf.ENKF_FP32, label=f"pivot {prec} ({nobs}, {nens})")


def test_pivoting_reorders_and_keeps_z():
    """The inputs reorder the levels, and Z equals the unpivoted device solve of the same problem."""
    nobs, nens = 3000, 24
    r, V, D = _problem(1801, nobs, nens, np.float64)
    dev = _run("fp64", r, V, D)
    assert dev["perm"].tolist() != list(range(nens))
    plan = enkf.Plan(1, nobs, nens, enkf.ENKF_FP64)
    tZ = to_dev(np.zeros((nens, nobs)), np.float64)
    plan.analysis(vec_dev(r, np.float64), to_dev(V, np.float64), to_dev(D, np.float64), Z=tZ, info=True)
    plan.close()
    assert rel(dev["Z"], host(tZ)) <= 1e-10


def test_pivoted_nonpositive_variance_is_a_numeric_error():
    nobs, nens = 500, 8
    r, V, D = _problem(1802, nobs, nens, np.float32)
    r[123] = -1.0
    with pytest.raises(enkf.EnkfError) as e:
        _run("fp32", r, V, D)
    assert e.value.status == enkf.ENKF_ERR_NUMERIC
