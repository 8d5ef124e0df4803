"""Parity of the plain level-streaming path (FP64 and FP32) with the FP64 oracle.

Every case runs through the C ABI (enkf_ism_plan / enkf_obs_prep /
enkf_ism_analysis) on seeded synthetic inputs; the oracle receives exactly the
values the device sees (FP32 inputs are rounded first).  The bars are per result
(tests/bars.py): relative Frobenius error <= 1e-10 for FP64 on every result; for FP32
<= 1e-5 on Z and X_A and <= 1e-4 on M and the increment dX_B M without refinement
(the part of Z in range(V) is damped by 1/gamma), <= 1e-5 on every result with one
refinement step.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from tests.bars import bars, check
from tests.util import host, rel, rounded, to_dev, vec_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1302_3876_gb300 import enkf  # noqa: E402

TOL = {enkf.ENKF_FP64: 1e-10, enkf.ENKF_FP32: 1e-5, enkf.ENKF_PANEL_FP32: 1e-5}
NP = {enkf.ENKF_FP64: np.float64, enkf.ENKF_FP32: np.float32, enkf.ENKF_PANEL_FP32: np.float32}
TT = {enkf.ENKF_FP64: torch.float64, enkf.ENKF_FP32: torch.float32, enkf.ENKF_PANEL_FP32: torch.float32}
MODES = [enkf.ENKF_FP64, enkf.ENKF_FP32, enkf.ENKF_PANEL_FP32]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    enkf.load(build_if_missing=True)


def random_problem(seed, nobs, nens, nstate=None, spread=1.0):
    nstate = nobs if nstate is None else nstate
    s = synth.uniform(seed, 1, nstate, 0.5, 2.0) * spread
    dXB = synth.normal_matrix(seed, 2, nstate, nens, row_scale=s)
    V = synth.normal_matrix(seed, 5, nobs, nens, std=1.0 / math.sqrt(max(nens - 1, 1)),
                            row_scale=synth.uniform(seed, 6, nobs, 0.5, 2.0))
    r = synth.uniform(seed, 3, nobs, 0.5, 1.5)
    D = synth.normal_matrix(seed, 4, nobs, nens)
    XB = dXB + synth.normal_matrix(seed, 7, nstate, 1, mean=1.0)[0][None, :]
    return r, V, D, dXB, XB


def run_device(mode, r, V, D, dXB=None, XB=None, ld_pad=0, info=True, flags=0, alias=False, panel_b=0):
    dt = NP[mode]
    nens, nobs = V.shape
    nstate = dXB.shape[1] if dXB is not None else 1
    plan = enkf.Plan(nstate, nobs, nens, mode, flags=flags, panel_b=panel_b)
    tV = to_dev(V, dt, nobs + ld_pad)
    tD = to_dev(D, dt, nobs + ld_pad)
    tr = vec_dev(r, dt)
    tZ = to_dev(np.zeros((nens, nobs)), dt, nobs + ld_pad)
    tM = torch.zeros(nens * nens, dtype=TT[mode], device="cuda") if nens >= 2 else None
    out = {}
    kw = {}
    if dXB is not None:
        tdX = to_dev(dXB, dt, nstate + ld_pad)
        tXB = to_dev(XB, dt, nstate + ld_pad)
        tXA = tXB if alias else to_dev(np.zeros_like(XB), dt, nstate + ld_pad)
        kw = dict(dXB=tdX, XB=tXB, XA=tXA)
    inf = plan.analysis(tr, tV, tD, Z=tZ, M=tM, info=info, **kw)
    torch.cuda.synchronize()
    out["Z"] = host(tZ)
    if tM is not None:
        out["M"] = host(tM).reshape(nens, nens).T     # column-major nens x nens -> M[m, e]
    if dXB is not None:
        out["XA"] = host(kw["XA"])
    out["info"] = inf
    plan.close()
    return out


def oracle_of(mode, r, V, D, dXB=None, XB=None):
    dt = NP[mode]
    r64, V64, D64 = rounded(r, dt), rounded(V, dt), rounded(D, dt)
    Z, gamma = oracle.ism_solve_refined(r64, V64, D64, return_gamma=True)
    out = {"Z": Z, "gamma": gamma}
    if V.shape[0] >= 2:
        out["M"] = oracle.vtz(V64, Z)
    if dXB is not None:
        dX64, XB64 = rounded(dXB, dt), rounded(XB, dt)
        out["XA"] = oracle.analysis_update(XB64, dX64, out["M"])
    return out


def errors(dev, ref, XB=None):
    """Relative errors of every result the device returned."""
    e = {"Z": rel(dev["Z"], ref["Z"])}
    if "M" in dev and "M" in ref:
        e["M"] = rel(dev["M"], ref["M"])
    if "XA" in dev and "XA" in ref:
        e["XA"] = rel(dev["XA"], ref["XA"])
        e["increment"] = rel(dev["XA"] - XB, ref["XA"] - XB)
    return e


CASES = [(1, 1), (2, 2), (3, 2), (31, 3), (33, 17), (127, 5), (129, 16), (1000, 32), (4099, 64), (20000, 48)]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("nobs,nens", CASES)
def test_solve_and_analysis_random(mode, nobs, nens):
    nstate = 3 * nobs + 5
    r, V, D, dXB, XB = random_problem(7000 + nobs + 13 * nens, nobs, nens, nstate)
    want_xa = nens >= 2
    dev = run_device(mode, r, V, D, dXB if want_xa else None, XB if want_xa else None)
    ref = oracle_of(mode, r, V, D, dXB if want_xa else None, XB if want_xa else None)
    XB64 = rounded(XB, NP[mode]) if want_xa else None
    errs = errors(dev, ref, XB64)
    print(f"mode {mode} nobs={nobs} nens={nens} gamma_max={ref['gamma'].max():.0f}: " +
          ", ".join(f"{k} {v:.2e}" for k, v in errs.items()))
    check(errs, mode, label=f"mode {mode} ({nobs}, {nens})")
    inf = dev["info"]
    assert inf.status == 0
    assert inf.gamma_min == pytest.approx(ref["gamma"].min(), rel=10 * TOL[mode])
    assert inf.gamma_max == pytest.approx(ref["gamma"].max(), rel=10 * TOL[mode])


@pytest.mark.parametrize("mode", MODES)
def test_padded_and_unaligned_leading_dimensions(mode):
    """ld > rows (padded, vector path) and an odd ld (scalar path) give the same result."""
    nobs, nens = 777, 9
    r, V, D, dXB, XB = random_problem(11, nobs, nens, 2000)
    ref = oracle_of(mode, r, V, D, dXB, XB)
    for pad in (0, 32, 3):
        dev = run_device(mode, r, V, D, dXB, XB, ld_pad=pad)
        check(errors(dev, ref, rounded(XB, NP[mode])), mode, label=f"pad {pad}")


@pytest.mark.parametrize("mode", [enkf.ENKF_FP64, enkf.ENKF_FP32])
def test_xa_aliases_xb(mode):
    nobs, nens = 500, 12
    r, V, D, dXB, XB = random_problem(12, nobs, nens, 1500)
    ref = oracle_of(mode, r, V, D, dXB, XB)
    dev = run_device(mode, r, V, D, dXB, XB, alias=True)
    check(errors(dev, ref, rounded(XB, NP[mode])), mode, label="alias")


@pytest.mark.parametrize("nens,xb_pad,alias", [(40, 0, False), (100, 4, False), (128, 0, False), (128, 0, True),
                                                (128, 1, False), (160, 0, False), (256, 4, False)])
def test_xa_update_paths(nens, xb_pad, alias):
    """X_A = X_B + dX_B M on the tensor-core update, every way the epilogue gets X_B: streamed
    by TMA into shared memory (Nens <= 128 and a 16-byte aligned X_B; two epilogue halves for
    Nens > 32), loaded from global memory (Nens > 128, or an X_B stride of an odd number of
    floats), and X_A written over X_B.  nstate is a multiple of 4 (TMA-aligned) and leaves a
    ragged last tile of 68 state rows."""
    mode = enkf.ENKF_FP32
    nobs, nstate = 700, 128 * 37 + 68
    r, V, D, dXB, XB = random_problem(13000 + nens + 7 * xb_pad, nobs, nens, nstate)
    ref = oracle_of(mode, r, V, D, dXB, XB)
    plan = enkf.Plan(nstate, nobs, nens, mode)
    tV, tD, tr = to_dev(V, np.float32), to_dev(D, np.float32), vec_dev(r, np.float32)
    tdX = to_dev(dXB, np.float32)
    tXB = to_dev(XB, np.float32, nstate + xb_pad)
    tXA = tXB if alias else to_dev(np.zeros_like(XB), np.float32, nstate + 8)
    tM = torch.zeros(nens * nens, dtype=torch.float32, device="cuda")
    inf = plan.analysis(tr, tV, tD, dXB=tdX, XB=tXB, XA=tXA, M=tM, info=True)
    torch.cuda.synchronize()
    plan.close()
    assert inf.status == 0
    XB64 = rounded(XB, np.float32)
    check({"XA": rel(host(tXA), ref["XA"]), "increment": rel(host(tXA) - XB64, ref["XA"] - XB64),
           "M": rel(host(tM).reshape(nens, nens).T, ref["M"])}, mode, label=f"xa paths {nens}")


@pytest.mark.parametrize("panel_b", [1, 5, 8, 16, 32])
def test_panel_widths(panel_b):
    """The panel form regroups the levels; every width (ragged last panel included)
    reaches the same result as the level-by-level oracle."""
    nobs, nens = 9000, 45
    r, V, D, dXB, XB = random_problem(31 + panel_b, nobs, nens, 20000)
    ref = oracle_of(enkf.ENKF_PANEL_FP32, r, V, D, dXB, XB)
    dev = run_device(enkf.ENKF_PANEL_FP32, r, V, D, dXB, XB, panel_b=panel_b)
    assert dev["info"].panel_b == panel_b
    check(errors(dev, ref, rounded(XB, np.float32)), enkf.ENKF_PANEL_FP32, label=f"b={panel_b}")
    assert dev["info"].gamma_max == pytest.approx(ref["gamma"].max(), rel=1e-4)


def test_zero_deviations():
    """V = 0: gamma_k = 1 and Z = R^-1 D exactly; M = 0 and X_A = X_B."""
    nobs, nens = 300, 8
    r, V, D, dXB, XB = random_problem(13, nobs, nens, 600)
    V[:] = 0.0
    dev = run_device(enkf.ENKF_FP64, r, V, D, dXB, XB)
    np.testing.assert_array_equal(dev["Z"], D / r[None, :])
    assert dev["info"].gamma_min == 1.0 and dev["info"].gamma_max == 1.0
    np.testing.assert_array_equal(dev["M"], 0.0)
    np.testing.assert_array_equal(dev["XA"], XB)


def test_deterministic_bitwise():
    nobs, nens = 50000, 40
    r, V, D, dXB, XB = random_problem(14, nobs, nens, 80000)
    a = run_device(enkf.ENKF_FP32, r, V, D, dXB, XB)
    b = run_device(enkf.ENKF_FP32, r, V, D, dXB, XB)
    for k in ("Z", "M", "XA"):
        np.testing.assert_array_equal(a[k], b[k])


@pytest.mark.parametrize("mode", [enkf.ENKF_FP64, enkf.ENKF_FP32])
def test_lorenz_small_full_pipeline(mode):
    """Lorenz-96 Nstate=40, Nens=20, every 2nd variable observed, R = 0.01 I:
    obs-space prep on the device (centering, H, 1/sqrt(Nens-1), D = Y - H X_B), then the analysis."""
    d = synth.lorenz_small_draws()
    dt = NP[mode]
    truth = oracle.l96_rk4(d["truth0"], F=d["F"], dt=0.01, nsteps=1000)[0]
    XB = rounded(truth[None, :] + d["ens_noise"], dt)
    Y = rounded((truth[::2] + d["obs_noise"])[None, :] + d["pert"], dt)
    r = np.full(d["nobs"], d["r"])
    # oracle
    _, dXB_o = oracle.ensemble_deviations(XB)
    V_o = oracle.observe_deviations(dXB_o, d["nobs"], 2)
    D_o = oracle.innovations(Y, XB, 2)
    ref = oracle.analysis(r, V_o, D_o, XB, dXB_o)
    # device
    plan = enkf.Plan(d["nstate"], d["nobs"], d["nens"], mode)
    tXB = to_dev(XB, dt)
    tdX = to_dev(np.zeros_like(XB), dt)
    tY = to_dev(Y, dt)
    tV = to_dev(np.zeros((d["nens"], d["nobs"])), dt)
    tD = to_dev(np.zeros((d["nens"], d["nobs"])), dt)
    plan.obs_prep(2, 1, tXB, tdX, tV, Y=tY, D=tD)
    tXA = to_dev(np.zeros_like(XB), dt)
    tZ = to_dev(np.zeros((d["nens"], d["nobs"])), dt)
    plan.analysis(vec_dev(r, dt), tV, tD, dXB=tdX, XB=tXB, XA=tXA, Z=tZ, info=True)
    torch.cuda.synchronize()
    tol = TOL[mode]
    assert rel(host(tdX), dXB_o) <= tol
    assert rel(host(tV), V_o) <= tol
    assert rel(host(tD), D_o) <= tol
    check({"Z": rel(host(tZ), ref["Z"]), "XA": rel(host(tXA), ref["XA"]),
           "increment": rel(host(tXA) - XB, ref["XA"] - XB)}, mode, label="lorenz_small")
    plan.close()


# ---------------------------------------------------------------------------
# Error paths: statuses, never a fault
# ---------------------------------------------------------------------------

def test_nonpositive_variance_is_a_numeric_error():
    nobs, nens = 100, 4
    r, V, D, _, _ = random_problem(15, nobs, nens)
    r[37] = 0.0
    with pytest.raises(enkf.EnkfError) as e:
        run_device(enkf.ENKF_FP64, r, V, D)
    assert e.value.status == enkf.ENKF_ERR_NUMERIC


def test_nan_innovation_is_a_numeric_error():
    nobs, nens = 100, 4
    r, V, D, _, _ = random_problem(16, nobs, nens)
    D[2, 5] = np.nan
    with pytest.raises(enkf.EnkfError) as e:
        run_device(enkf.ENKF_FP32, r, V, D)
    assert e.value.status == enkf.ENKF_ERR_NUMERIC


def test_bounded_barrier_wait_expires_with_a_status():
    """One CTA never arrives (test flag); the others' bounded wait returns ENKF_ERR_TIMEOUT."""
    nobs, nens = 200000, 8
    r, V, D, _, _ = random_problem(17, nobs, nens)
    with pytest.raises(enkf.EnkfError) as e:
        run_device(enkf.ENKF_FP32, r, V, D, flags=enkf.ENKF_FLAG_TEST_TIMEOUT)
    assert e.value.status == enkf.ENKF_ERR_TIMEOUT
    # the context is still usable afterwards
    dev = run_device(enkf.ENKF_FP32, r, V, D)
    assert dev["info"].status == 0


def test_argument_errors():
    plan = enkf.Plan(100, 50, 4, enkf.ENKF_FP32)
    r = torch.ones(50, device="cuda")
    V = torch.zeros(4, 50, device="cuda")
    D = torch.zeros(4, 50, device="cuda")
    small = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(enkf.EnkfError) as e:
        enkf.enkf_ism_analysis(plan.handle, r, V, D, small)
    assert e.value.status == enkf.ENKF_ERR_WORKSPACE
    with pytest.raises(enkf.EnkfError) as e:
        enkf.enkf_ism_analysis(plan.handle, r, torch.zeros(4, 40, device="cuda"), D, plan.workspace)
    assert e.value.status == enkf.ENKF_ERR_SHAPE
    plan.close()
    plan1 = enkf.Plan(100, 50, 1, enkf.ENKF_FP32)
    with pytest.raises(enkf.EnkfError) as e:
        plan1.analysis(r, V[:1], D[:1], M=torch.zeros(1, device="cuda"))
    assert e.value.status == enkf.ENKF_ERR_SHAPE
    plan1.close()


# ---------------------------------------------------------------------------
# Full size: the large single analysis (Nstate=2^21, Nobs=2^19, Nens=128)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("mode", [enkf.ENKF_PANEL_FP32, enkf.ENKF_FP32, enkf.ENKF_FP64])
def test_large_single_full_size(mode):
    """The benchmark's workload, in the benchmark's launch configuration: V from
    the deviations on the device (every 4th row, 1/sqrt(Nens-1)), then the
    analysis; every output compared with the oracle run on the same values."""
    dt = NP[mode]
    w = synth.large_single(dtype=dt)
    nstate, nobs, nens = w["nstate"], w["nobs"], w["nens"]
    plan = enkf.Plan(nstate, nobs, nens, mode)
    tdX = torch.from_numpy(w["dXB"]).cuda()
    tD = torch.from_numpy(w["D"]).cuda()
    tr = torch.from_numpy(w["r"]).cuda()
    tV = torch.zeros(nens, nobs, dtype=TT[mode], device="cuda")
    plan.obs_prep(4, 0, None, tdX, tV)
    tXA = torch.empty_like(tdX)
    tZ = torch.empty(nens, nobs, dtype=TT[mode], device="cuda")
    tM = torch.empty(nens * nens, dtype=TT[mode], device="cuda")
    inf = plan.analysis(tr, tV, tD, dXB=tdX, XB=tdX, XA=tXA, Z=tZ, M=tM, info=True)
    assert inf.status == 0
    dX64 = w["dXB"].astype(np.float64)
    del w
    V_o = oracle.observe_deviations(dX64, nobs, 4)
    assert rel(host(tV), V_o) <= TOL[mode]
    r64 = host(tr)
    D64 = host(tD)
    Z, gamma = oracle.ism_solve_refined(r64, V_o, D64, return_gamma=True)
    assert rel(host(tZ), Z) <= TOL[mode]
    M = oracle.vtz(V_o, Z)
    XA = oracle.analysis_update(dX64, dX64, M)
    errs = {"Z": rel(host(tZ), Z), "M": rel(host(tM).reshape(nens, nens).T, M), "XA": rel(host(tXA), XA),
            "increment": rel(host(tXA) - dX64, XA - dX64)}
    print(f"large_single mode {mode}: " + ", ".join(f"{k} {v:.2e}" for k, v in errs.items()))
    check(errs, mode, label="large_single")
    plan.close()
