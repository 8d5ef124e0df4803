"""Parity of the tensor-core panel forms and of the refinement with the FP64 oracle.

ENKF_PANEL_BF16 runs the trailing update and the dots on tensor cores with split
BF16 operands (x = hi + lo, three products; each operand kept to ~2^-17);
ENKF_PANEL_FP16 uses one FP16 product (unit roundoff 2^-11); ENKF_PANEL_BF16X3 splits
each operand in three BF16 pieces (six products, operands kept to ~2^-25, the FP32
bars of the plain path).  All store in FP32, accumulate in FP32 and form the level
denominators in FP64.  The bars are per result, fixed, from tests/bars.py (Z, X_A, M
and the increment dX_B M, relative Frobenius error against the oracle on the same
FP32 inputs).  The measured errors are printed so the tables in the design notes can
quote them.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from tests import bars as B
from tests.util import host, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1302_3876_gb300 import enkf  # noqa: E402

NAME = {enkf.ENKF_PANEL_BF16: "PANEL_BF16", enkf.ENKF_PANEL_FP16: "PANEL_FP16",
        enkf.ENKF_PANEL_BF16X3: "PANEL_BF16X3"}
# ~ 2^-17, 2^-11 and 2^-25 operands
GAMMA_REL = {enkf.ENKF_PANEL_BF16: 1e-4, enkf.ENKF_PANEL_FP16: 1e-3, enkf.ENKF_PANEL_BF16X3: 1e-5}
TC_MODES = [enkf.ENKF_PANEL_BF16, enkf.ENKF_PANEL_FP16, enkf.ENKF_PANEL_BF16X3]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    enkf.load(build_if_missing=True)


def problem(seed, nobs, nens, nstate):
    s = synth.uniform(seed, 1, nstate, 0.5, 2.0)
    dXB = synth.normal_matrix(seed, 2, nstate, nens, row_scale=s).astype(np.float32).astype(np.float64)
    r = synth.uniform(seed, 3, nobs, 0.5, 1.5).astype(np.float32).astype(np.float64)
    D = synth.normal_matrix(seed, 4, nobs, nens).astype(np.float32).astype(np.float64)
    V = oracle.observe_deviations(dXB, nobs, max(1, nstate // nobs)).astype(np.float32).astype(np.float64)
    return r, V, D, dXB


def run(mode, r, V, D, dXB, panel_b=0, flags=0):
    nens, nobs = V.shape
    nstate = dXB.shape[1]
    plan = enkf.Plan(nstate, nobs, nens, mode, panel_b=panel_b, flags=flags)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()  # noqa: E731
    tr, tV, tD, tdX = t(r), t(V), t(D), t(dXB)
    tXA = torch.empty_like(tdX)
    tZ = torch.empty_like(tD)
    tM = torch.empty(nens * nens, device="cuda")
    inf = plan.analysis(tr, tV, tD, dXB=tdX, XB=tdX, XA=tXA, Z=tZ, M=tM, info=True)
    assert inf.status == 0
    out = {"Z": host(tZ), "XA": host(tXA), "M": host(tM).reshape(nens, nens).T, "info": inf}
    plan.close()
    return out


_REF = {}


def reference(r, V, D, dXB):
    """The oracle's Z, gamma, M and X_A (cached for the full-size workloads, which several
    tests share)."""
    key = (V.shape, float(r[0]), float(D[0, 0]), float(V[-1, -1]))
    if key in _REF:
        return _REF[key]
    Z, gamma = oracle.ism_solve_refined(r, V, D, return_gamma=True)
    M = oracle.vtz(V, Z)
    out = (Z, gamma, M, oracle.analysis_update(dXB, dXB, M))
    if V.shape[1] >= 200000:   # keep the latest full-size reference only
        _REF.clear()
        _REF[key] = out
    return out


def errors(dev, r, V, D, dXB):
    Z, gamma, M, XA = reference(r, V, D, dXB)
    return {"Z": rel(dev["Z"], Z), "XA": rel(dev["XA"], XA), "M": rel(dev["M"], M),
            "increment": rel(dev["XA"] - dXB, XA - dXB)}, gamma


def check(mode, dev, r, V, D, dXB, label):
    Z, gamma, M, XA = reference(r, V, D, dXB)
    errs = {"Z": rel(dev["Z"], Z), "XA": rel(dev["XA"], XA), "M": rel(dev["M"], M),
            "increment": rel(dev["XA"] - dXB, XA - dXB)}
    print(f"{NAME[mode]} {label}: " + ", ".join(f"{k} {v:.2e}" for k, v in errs.items()) +
          f", gamma_max {gamma.max():.1f}")
    B.check(errs, mode, label=f"{NAME[mode]} {label}")
    # the level denominators inherit the operand precision of the panel Gram
    assert dev["info"].gamma_max == pytest.approx(gamma.max(), rel=GAMMA_REL[mode])


@pytest.mark.parametrize("mode", TC_MODES)
@pytest.mark.parametrize("nobs,nens,panel_b", [(1, 4, 0), (31, 5, 0), (129, 16, 8), (4099, 64, 32), (20000, 48, 16),
                                               (20011, 128, 32), (9000, 256, 32), (5000, 37, 5)])
def test_tensor_core_panel_random(mode, nobs, nens, panel_b):
    nstate = 3 * nobs + 1
    r, V, D, dXB = problem(9000 + nobs + nens, nobs, nens, nstate)
    dev = run(mode, r, V, D, dXB, panel_b)
    check(mode, dev, r, V, D, dXB, f"nobs={nobs} nens={nens} b={panel_b}")


@pytest.mark.parametrize("mode", TC_MODES)
def test_large_single_full_size(mode):
    w = synth.large_single(dtype=np.float32)
    dXB = w["dXB"].astype(np.float64)
    r = w["r"].astype(np.float64)
    D = w["D"].astype(np.float64)
    V = oracle.observe_deviations(dXB, w["nobs"], 4).astype(np.float32).astype(np.float64)
    dev = run(mode, r, V, D, dXB)
    check(mode, dev, r, V, D, dXB, "large_single full size")


def test_panel_single_full_size():
    """Nobs = 2^20, Nens = 256, Nstate = 2^22 (the panel workload), split-BF16 tensor cores."""
    w = synth.panel_single()
    dXB = w["dXB"].astype(np.float64)
    r = w["r"].astype(np.float64)
    D = w["D"].astype(np.float64)
    del w
    V = oracle.observe_deviations(dXB, 1 << 20, 4).astype(np.float32).astype(np.float64)
    dev = run(enkf.ENKF_PANEL_BF16, r, V, D, dXB)
    check(enkf.ENKF_PANEL_BF16, dev, r, V, D, dXB, "panel_single full size")


# ---------------------------------------------------------------------------
# One step of iterative refinement (ENKF_FLAG_REFINE).  The correction applies the
# stored factors, an approximate inverse whose error in range(V) is about
# rho = u * gamma_max (u the precision of the solve's operands), so one step
# multiplies the error of Z and M by about rho.  The refined FP32-class paths
# (PANEL_FP32, PANEL_BF16X3) are held to 1e-5 on every result, split BF16 to its
# refined bars (tests/bars.py), and every refined error must also be below the
# unrefined one where that was above the refined floor.  PANEL_FP16 (u = 2^-11):
# the errors of Z and M must shrink where rho < 1 (the medium cases below); at
# gamma ~ 10^4 it is not effective and is not tested there.
# ---------------------------------------------------------------------------
GAIN_MODES = (enkf.ENKF_PANEL_BF16, enkf.ENKF_PANEL_FP32, enkf.ENKF_PANEL_BF16X3)


@pytest.mark.parametrize("mode", [enkf.ENKF_PANEL_BF16, enkf.ENKF_PANEL_FP16, enkf.ENKF_PANEL_FP32,
                                  enkf.ENKF_PANEL_BF16X3])
@pytest.mark.parametrize("nobs,nens,panel_b", [(129, 16, 8), (20011, 128, 32), (9000, 256, 32), (5000, 37, 5)])
def test_refinement_random(mode, nobs, nens, panel_b):
    nstate = 3 * nobs + 1
    r, V, D, dXB = problem(9100 + nobs + nens, nobs, nens, nstate)
    base, gamma = errors(run(mode, r, V, D, dXB, panel_b), r, V, D, dXB)
    ref, _ = errors(run(mode, r, V, D, dXB, panel_b, flags=enkf.ENKF_FLAG_REFINE), r, V, D, dXB)
    print(f"refine {mode} nobs={nobs} nens={nens} gamma_max={gamma.max():.0f}: before " +
          ", ".join(f"{k} {v:.2e}" for k, v in base.items()) + " | after " +
          ", ".join(f"{k} {v:.2e}" for k, v in ref.items()))
    if mode in GAIN_MODES:
        B.check(ref, mode, refine=True, label=f"refined {NAME.get(mode, mode)}")
        for k in ("Z", "M", "increment"):
            assert ref[k] <= max(2e-6, base[k]), (k, base, ref)
    else:
        assert ref["Z"] <= 0.1 * base["Z"], (base, ref)
        assert ref["M"] <= 0.5 * base["M"], (base, ref)
        assert ref["XA"] <= base["XA"], (base, ref)


@pytest.mark.parametrize("mode", GAIN_MODES)
def test_refinement_large_single_full_size(mode):
    """Nstate 2^21, Nobs 2^19, Nens 128 (gamma ~ 8000): the refined paths at their bars."""
    w = synth.large_single(dtype=np.float32)
    dXB = w["dXB"].astype(np.float64)
    r = w["r"].astype(np.float64)
    D = w["D"].astype(np.float64)
    V = oracle.observe_deviations(dXB, w["nobs"], 4).astype(np.float32).astype(np.float64)
    base, gamma = errors(run(mode, r, V, D, dXB), r, V, D, dXB)
    errs, _ = errors(run(mode, r, V, D, dXB, flags=enkf.ENKF_FLAG_REFINE), r, V, D, dXB)
    print(f"refine {mode} large_single gamma_max={gamma.max():.0f}: before " +
          ", ".join(f"{k} {v:.2e}" for k, v in base.items()) + " | after " +
          ", ".join(f"{k} {v:.2e}" for k, v in errs.items()))
    B.check(errs, mode, refine=True, label="refined large_single")
    B.check(base, mode, refine=False, label="unrefined large_single")


@pytest.mark.parametrize("mode", [enkf.ENKF_PANEL_FP32, enkf.ENKF_PANEL_BF16X3])
def test_refinement_panel_single_full_size(mode):
    """Nstate 2^22, Nobs 2^20, Nens 256: the refined FP32-class panel paths meet 1e-5 on Z,
    M, X_A and the increment at the panel workload."""
    w = synth.panel_single()
    dXB = w["dXB"].astype(np.float64)
    r = w["r"].astype(np.float64)
    D = w["D"].astype(np.float64)
    del w
    V = oracle.observe_deviations(dXB, 1 << 20, 4).astype(np.float32).astype(np.float64)
    errs, gamma = errors(run(mode, r, V, D, dXB, flags=enkf.ENKF_FLAG_REFINE), r, V, D, dXB)
    print(f"refine {mode} panel_single gamma_max={gamma.max():.0f}: " +
          ", ".join(f"{k} {v:.2e}" for k, v in errs.items()))
    B.check(errs, mode, refine=True, label="refined panel_single")
