"""Parity of inflation (Sec. 3.1.1), partial localization (Sec. 3.1.2) and the
block-diagonal R path (Sec. 3.1) with the FP64 oracle, through the C ABI
(enkf_inflate_prep, enkf_localized_update, enkf_rblock_factor / whiten /
unwhiten with enkf_ism_analysis).

Tolerances (relative Frobenius norm): FP64 <= 1e-10; FP32 <= 1e-5 on X_A, Z and the
prep outputs.  The localized increment dX_A = X_A - X_B on its own is held to 2e-5 in
FP32: it is a sum over every observation of products formed with FP32 sums over the
members, so its rounding error grows with sqrt(Nobs) relative to the increment.  The
block-R analysis is held to the plain path's per-result bars (tests/bars.py): FP32 Z
and X_A 1e-5, M and the increment 1e-4 without refinement."""
import math

import numpy as np
import pytest

import oracle
from tests import bars as B
import synth
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


# ----------------------------------------------------------------------------------------------
# inflation fused into the prep
# ----------------------------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("nstate,stride,nens,alpha", [(40, 2, 20, 1.1), (1001, 3, 17, 1.0), (1001, 3, 17, 1.35),
                                                      (8192, 4, 64, 1.02), (37, 1, 2, 0.5)])
def test_inflate_prep_matches_oracle(prec, nstate, stride, nens, alpha):
    npt, _, tol, _ = DT[prec]
    nobs = (nstate - 1) // stride + 1
    seed = 500 + nstate + nens
    XB = rounded(synth.normal_matrix(seed, 1, nstate, nens, mean=8.0), npt)
    Y = rounded(synth.normal_matrix(seed, 2, nobs, nens, mean=8.0), npt)
    tXB = to_dev(XB, npt, nstate + 3)
    tdX = to_dev(np.zeros_like(XB), npt)
    tV = to_dev(np.zeros((nens, nobs)), npt, nobs + 5)
    tY = to_dev(Y, npt)
    tD = to_dev(np.zeros((nens, nobs)), npt)
    enkf.enkf_inflate_prep(stride, alpha, tXB, tV, dXB=tdX, Y=tY, D=tD)
    torch.cuda.synchronize()
    Xi = oracle.inflate(XB, alpha)
    _, dX = oracle.ensemble_deviations(Xi)
    V = oracle.observe_deviations(dX, nobs, stride)
    D = oracle.innovations(Y, Xi, stride)
    assert rel(host(tXB), Xi) <= tol
    assert rel(host(tdX), dX) <= tol
    assert rel(host(tV), V) <= tol
    assert rel(host(tD), D) <= tol
    # the mean is unchanged and the spread scales by alpha (Sec. 3.1.1)
    np.testing.assert_allclose(host(tXB).mean(0), XB.mean(0), rtol=0, atol=64 * np.finfo(npt).eps * 10)


def test_inflate_prep_alpha_one_equals_obs_prep():
    nstate, nobs, nens, stride = 2048, 1024, 32, 2
    XB = synth.normal_matrix(77, 1, nstate, nens, mean=8.0).astype(np.float32)
    Y = synth.normal_matrix(77, 2, nobs, nens, mean=8.0).astype(np.float32)
    plan = enkf.Plan(nstate, nobs, nens, enkf.ENKF_FP32)
    outs = []
    for fused in (False, True):
        tXB, tY = to_dev(XB, np.float32), to_dev(Y, np.float32)
        tdX = to_dev(np.zeros_like(XB), np.float32)
        tV, tD = to_dev(np.zeros((nens, nobs)), np.float32), to_dev(np.zeros((nens, nobs)), np.float32)
        if fused:
            enkf.enkf_inflate_prep(stride, 1.0, tXB, tV, dXB=tdX, Y=tY, D=tD)
        else:
            plan.obs_prep(stride, 1, tXB, tdX, tV, Y=tY, D=tD)
        torch.cuda.synchronize()
        outs.append([host(t) for t in (tXB, tdX, tV, tD)])
    plan.close()
    (xb0, dx0, v0, d0), (xb1, dx1, v1, d1) = outs
    np.testing.assert_array_equal(xb1, xb0)          # alpha = 1 leaves X_B as it was
    np.testing.assert_array_equal(d1, d0)            # D = Y - H X_B, one FP32 subtraction on both paths
    assert rel(dx1, dx0) <= 1e-6                     # FP32 compensated mean against the FP64 mean
    assert rel(v1, v0) <= 1e-6


# ----------------------------------------------------------------------------------------------
# partial localization
# ----------------------------------------------------------------------------------------------

def _loc_problem(seed, nstate, stride, nens, npt):
    nobs = (nstate - 1) // stride + 1
    dXB = synth.normal_matrix(seed, 1, nstate, nens, row_scale=synth.uniform(seed, 2, nstate, 0.5, 2.0))
    XB = rounded(dXB + synth.normal_matrix(seed, 3, nstate, 1, mean=8.0)[0][None, :], npt)
    dXB = rounded(dXB, npt)
    V = rounded(synth.normal_matrix(seed, 4, nobs, nens, std=1.0 / math.sqrt(nens - 1)), npt)
    Z = rounded(synth.normal_matrix(seed, 5, nobs, nens), npt)
    return XB, dXB, V, Z


LOC_CASES = [
    (40, 2, 20, 40.0, None),        # the small Lorenz-96 ensemble with the weights of Sec. 4.2
    (1000, 4, 17, 1000.0, None),    # ragged tiles and members
    (1000, 4, 17, 50.0, 30.5),      # cut-off band, wrap-around at both ends
    (513, 1, 2, 10.0, 5.0),         # two members, every variable observed
    (777, 3, 33, math.inf, None),   # delta = 1: the unlocalized update
    (300, 5, 8, 20.0, 0.0),         # radius 0: only the observed components move
    (130, 1, 64, 40.0, 64.0),       # band wider than the ring: dense visit with a cut-off
    # the band shapes that tests/test_localize_band.py checks on the CPU, on the kernel itself:
    # tile 0 and the partial last tile wrap around the ring
    (97, 3, 12, 20.0, 31.9),
    (64, 1, 9, 8.0, 15.9),
]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("nstate,stride,nens,length,radius", LOC_CASES)
def test_localized_update_matches_oracle(prec, nstate, stride, nens, length, radius):
    npt, _, tol, _ = DT[prec]
    XB, dXB, V, Z = _loc_problem(900 + nstate + nens, nstate, stride, nens, npt)
    tXB, tdX = to_dev(XB, npt, nstate + 7), to_dev(dXB, npt)
    tV, tZ = to_dev(V, npt, V.shape[1] + 2), to_dev(Z, npt)
    tXA = to_dev(np.zeros_like(XB), npt)
    enkf.enkf_localized_update(stride, length, radius, tdX, tV, tZ, tXB, tXA)
    torch.cuda.synchronize()
    want = oracle.localized_update(XB, dXB, V, Z, stride, length, radius)
    got = host(tXA)
    assert rel(got, want) <= tol
    assert rel(got - XB, want - XB) <= (tol if prec == "fp64" else 2e-5)
    if length == math.inf and radius is None:
        # the unlocalized SMEnKF update X_B + dX_B M (Sec. 3.1) of the same inputs
        plain = oracle.analysis_update(XB, dXB, oracle.vtz(V, Z))
        assert rel(got, plain) <= tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_localized_update_in_place(prec):
    npt, _, tol, _ = DT[prec]
    nstate, stride, nens = 2000, 2, 40
    XB, dXB, V, Z = _loc_problem(31, nstate, stride, nens, npt)
    tXB, tdX, tV, tZ = to_dev(XB, npt), to_dev(dXB, npt), to_dev(V, npt), to_dev(Z, npt)
    enkf.enkf_localized_update(stride, 100.0, 250.0, tdX, tV, tZ, tXB, tXB)
    torch.cuda.synchronize()
    assert rel(host(tXB), oracle.localized_update(XB, dXB, V, Z, stride, 100.0, 250.0)) <= tol


@pytest.mark.parametrize("prec,radius", [("fp32", None), ("fp32", 64.0), ("fp64", None)])
def test_localized_update_lorenz_cycle_size(prec, radius):
    """Nstate 4096, every 2nd variable observed (Nobs 2048), 256 members: the size of the Lorenz-96
    cycle, with the paper's weights exp(-d / Nstate) (Sec. 4.2) or a 64-point cut-off."""
    npt, _, tol, _ = DT[prec]
    nstate, stride, nens = 4096, 2, 256
    XB, dXB, V, Z = _loc_problem(4096, nstate, stride, nens, npt)
    tXB, tdX, tV, tZ = to_dev(XB, npt), to_dev(dXB, npt), to_dev(V, npt), to_dev(Z, npt)
    tXA = torch.empty_like(tXB)
    enkf.enkf_localized_update(stride, float(nstate), radius, tdX, tV, tZ, tXB, tXA)
    torch.cuda.synchronize()
    want = oracle.localized_update(XB, dXB, V, Z, stride, float(nstate), radius)
    got = host(tXA)
    assert rel(got, want) <= tol
    assert rel(got - XB, want - XB) <= (tol if prec == "fp64" else 2e-5)


def test_localized_update_rejects_bad_arguments():
    XB, dXB, V, Z = _loc_problem(5, 64, 2, 8, np.float32)
    tXB, tdX, tV, tZ = (to_dev(a, np.float32) for a in (XB, dXB, V, Z))
    with pytest.raises(enkf.EnkfError) as e:
        enkf.enkf_localized_update(2, 0.0, None, tdX, tV, tZ, tXB, tXB)
    assert e.value.status == enkf.ENKF_ERR_ARG
    with pytest.raises(enkf.EnkfError) as e:                 # X_A on top of Z
        enkf.enkf_localized_update(2, 10.0, None, tdX, tV, tZ, tXB, tZ)
    assert e.value.status in (enkf.ENKF_ERR_ARG, enkf.ENKF_ERR_SHAPE)
    big = to_dev(np.zeros((257, 64)), np.float32)
    with pytest.raises(enkf.EnkfError) as e:
        enkf.enkf_localized_update(2, 10.0, None, big, to_dev(np.zeros((257, 32)), np.float32),
                                   to_dev(np.zeros((257, 32)), np.float32), big, to_dev(np.zeros((257, 64)),
                                                                                          np.float32))
    assert e.value.status == enkf.ENKF_ERR_SHAPE


# ----------------------------------------------------------------------------------------------
# block-diagonal R
# ----------------------------------------------------------------------------------------------

def _spd_blocks(seed, nblk, bs):
    A = synth.normal_matrix(seed, 1, nblk * bs, bs).reshape(bs, nblk, bs).transpose(1, 0, 2)
    d = synth.uniform(seed, 2, nblk * bs, 0.5, 1.5).reshape(nblk, bs)
    R = np.einsum("bij,bkj->bik", A, A) / bs
    R[:, np.arange(bs), np.arange(bs)] += d
    return R


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("nobs,bs,nens", [(100, 4, 8), (1000, 7, 32), (5000, 32, 64), (33, 1, 5), (4099, 16, 17)])
def test_block_diagonal_r_analysis_matches_oracle(prec, nobs, bs, nens):
    npt, tt, tol, mode = DT[prec]
    nstate = 2 * nobs + 3
    seed = 1300 + nobs + bs
    nblk = (nobs + bs - 1) // bs
    Rblk = _spd_blocks(seed, nblk, bs)
    dXB = rounded(synth.normal_matrix(seed, 3, nstate, nens), npt)
    XB = rounded(dXB + 1.0, npt)
    V = rounded(synth.normal_matrix(seed, 4, nobs, nens, std=1.0 / math.sqrt(nens - 1)), npt)
    D = rounded(synth.normal_matrix(seed, 5, nobs, nens), npt)
    tR = torch.from_numpy(Rblk.transpose(0, 2, 1).copy()).cuda()       # column-major blocks
    tL = torch.empty_like(tR)
    tV, tD = to_dev(V, npt), to_dev(D, npt)
    enkf.enkf_rblock_factor(nobs, bs, tR, tL)
    enkf.enkf_rblock_whiten(bs, tL, tV, tD)
    plan = enkf.Plan(nstate, nobs, nens, mode)
    tZ = to_dev(np.zeros((nens, nobs)), npt)
    tM = torch.zeros(nens * nens, dtype=tt, device="cuda")
    tdX, tXB = to_dev(dXB, npt), to_dev(XB, npt)
    tXA = torch.empty_like(tXB)
    inf = plan.analysis(torch.ones(nobs, dtype=tt, device="cuda"), tV, tD, dXB=tdX, XB=tXB, XA=tXA, Z=tZ, M=tM,
                        info=True)
    enkf.enkf_rblock_unwhiten(bs, tL, tZ)
    torch.cuda.synchronize()
    plan.close()
    Z, gamma = oracle.ism_solve_blockdiag(Rblk, V, D, return_gamma=True)
    M = oracle.vtz(V, Z)
    XA = oracle.analysis_update(XB, dXB, M)
    assert inf.status == 0
    assert inf.gamma_max == pytest.approx(gamma.max(), rel=10 * tol)
    B.check({"Z": rel(host(tZ), Z), "M": rel(host(tM).reshape(nens, nens).T, M), "XA": rel(host(tXA), XA),
             "increment": rel(host(tXA) - XB, XA - XB)}, mode, label=f"block-R {prec} ({nobs}, {bs}, {nens})")


def test_block_diagonal_r_not_positive_definite_is_reported():
    nobs, bs, nens = 64, 8, 4
    Rblk = _spd_blocks(3, nobs // bs, bs)
    Rblk[2] = -np.eye(bs)
    V = synth.normal_matrix(4, 1, nobs, nens, std=0.5).astype(np.float32)
    D = synth.normal_matrix(4, 2, nobs, nens).astype(np.float32)
    tR = torch.from_numpy(Rblk.transpose(0, 2, 1).copy()).cuda()
    tL = torch.empty_like(tR)
    tV, tD = to_dev(V, np.float32), to_dev(D, np.float32)
    enkf.enkf_rblock_factor(nobs, bs, tR, tL)
    enkf.enkf_rblock_whiten(bs, tL, tV, tD)
    assert torch.isnan(tV[:, 2 * bs:3 * bs]).all()
    plan = enkf.Plan(nobs, nobs, nens, enkf.ENKF_FP32)
    with pytest.raises(enkf.EnkfError) as e:
        plan.analysis(torch.ones(nobs, device="cuda"), tV, tD, Z=to_dev(np.zeros((nens, nobs)), np.float32),
                      info=True)
    assert e.value.status == enkf.ENKF_ERR_NUMERIC
    plan.close()


# ----------------------------------------------------------------------------------------------
# the Lorenz-96 cycle with inflation and partial localization
# ----------------------------------------------------------------------------------------------

def test_inflated_localized_cycles_match_oracle_cycles():
    """Three cycles of RK4 forecast, inflated prep, ISM solve and localized update on the device
    (FP32 ensemble, FP64 truth) against the same cycles composed from the oracle in FP64 on the
    same draws: within 2e-4 relative after three cycles (FP32 arithmetic on a chaotic system).
    The weights are the paper's exp(-d / Nstate) (Sec. 4.2).  Partial localization leaves
    (R + V V^T)^{-1} unlocalized, and with correlation lengths short against the state (16 to 64
    points here, with or without a cut-off) the cycle of the oracle itself diverges within two to
    four cycles, so those settings make no parity case."""
    from paper_1302_3876_gb300 import cycle as C
    nstate, nens, stride, r, seed = 128, 16, 2, 0.25, 99
    alpha, length, radius = 1.05, float(nstate), None
    cyc = C.LorenzCycle(nstate, nens, stride, r, seed=seed, spinup=300, inflation=alpha, loc_length=length,
                        loc_radius=radius)
    X = cyc.X.double().cpu().numpy()
    truth = cyc.truth.cpu().numpy()[0]
    nobs = nstate // stride
    for c in range(3):
        cyc.forecast("rk4")
        cyc.analysis()
        X = oracle.l96_rk4(X, 8.0, 0.01, 5)
        truth = oracle.l96_rk4(truth, 8.0, 0.01, 5)[0]
        d = synth.lorenz_cycle_draws(c, nstate, nens, stride, r, seed)
        y32 = truth[::stride].astype(np.float32) + d["obs_noise"].astype(np.float32)
        Y = (y32[None, :] + d["pert"].astype(np.float32)).astype(np.float64)
        X = oracle.inflate(X, alpha)
        _, dX = oracle.ensemble_deviations(X)
        V = oracle.observe_deviations(dX, nobs, stride)
        D = oracle.innovations(Y, X, stride)
        Z = oracle.ism_solve(np.full(nobs, r), V, D)
        X = oracle.localized_update(X, dX, V, Z, stride, length, radius)
    np.testing.assert_array_equal(cyc.truth.cpu().numpy()[0], truth)
    assert rel(cyc.X.double().cpu().numpy(), X) <= 2e-4
    rm, _, _ = cyc.run(20, "rk4")
    assert math.isfinite(rm)
    cyc.close()
