"""Pins of the oracle's inflation (Sec. 3.1.1), partial localization (Sec. 3.1.2)
and block-diagonal R (Sec. 3.1) routines against what the paper and the
mathematics fix: the alpha^2 covariance law, the unlocalized analysis as the
delta = 1 case, the diagonal (radius 0) and single-observation cases, the
periodic shift symmetry of the Lorenz-96 weights (Sec. 4.2), the component
formula against the matrix form, and the textbook dense solve of R + V V^T.
CPU only."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
import synth


def _problem(seed, nstate, nobs, nens):
    dXB = synth.normal_matrix(seed, 1, nstate, nens, row_scale=synth.uniform(seed, 2, nstate, 0.5, 2.0))
    XB = dXB + 3.0
    V = synth.normal_matrix(seed, 3, nobs, nens, std=1.0 / math.sqrt(nens - 1))
    Z = synth.normal_matrix(seed, 4, nobs, nens)
    return XB, dXB, V, Z


# ----------------------------------------------------------------------------------------------
# inflation
# ----------------------------------------------------------------------------------------------

def test_inflation_keeps_the_mean_and_scales_the_covariance_by_alpha_squared():
    X = synth.normal_matrix(11, 1, 30, 9, mean=2.0)           # (nens, nstate)
    for alpha in (0.5, 1.07, 2.0):
        Y = oracle.inflate(X, alpha)
        np.testing.assert_allclose(Y.mean(0), X.mean(0), rtol=0, atol=1e-13)
        np.testing.assert_allclose(np.cov(Y.T), alpha * alpha * np.cov(X.T), rtol=1e-12, atol=1e-13)


def test_inflation_special_factors():
    X = synth.normal_matrix(12, 1, 17, 5)
    np.testing.assert_allclose(oracle.inflate(X, 1.0), X, rtol=0, atol=1e-15)
    np.testing.assert_allclose(oracle.inflate(X, 0.0), np.broadcast_to(X.mean(0), X.shape), rtol=0, atol=1e-15)
    # two members (rows) of a two-component state: component 0 holds 1 and 3 (mean 2, half-spread 1),
    # component 1 holds -2 and 4 (mean 1, half-spread 3); alpha = 3 gives m -+ 3 a
    X2 = np.array([[1.0, -2.0], [3.0, 4.0]])
    np.testing.assert_allclose(oracle.inflate(X2, 3.0), [[-1.0, -8.0], [5.0, 10.0]], rtol=0, atol=1e-14)


# ----------------------------------------------------------------------------------------------
# partial localization
# ----------------------------------------------------------------------------------------------

@pytest.mark.parametrize("radius", [None, 0.0, 3.0, 7.5])
@pytest.mark.parametrize("stride", [1, 2, 3])
def test_component_formula_equals_matrix_form(stride, radius):
    nstate, nens = 23, 5
    nobs = (nstate - 1) // stride + 1
    XB, dXB, V, Z = _problem(21 + stride, nstate, nobs, nens)
    dX = oracle.localized_increment_literal(dXB, V, Z, stride, nstate, radius)
    XA = oracle.localized_update(XB, dXB, V, Z, stride, nstate, radius)
    np.testing.assert_allclose(XA - XB, dX, rtol=1e-12, atol=1e-13)


def test_unit_weights_give_the_unlocalized_analysis():
    """delta = 1 everywhere (infinite correlation length, no cut-off): Delta o (S V^T) Z = S V^T Z =
    dX_B M with M = V^T Z / sqrt(Nens - 1) (the SMEnKF update of Sec. 3.1)."""
    nstate, nobs, nens = 64, 16, 8
    XB, dXB, V, Z = _problem(31, nstate, nobs, nens)
    XA = oracle.localized_update(XB, dXB, V, Z, 4, math.inf, None)
    want = oracle.analysis_update(XB, dXB, oracle.vtz(V, Z))
    np.testing.assert_allclose(XA, want, rtol=1e-12, atol=1e-12)


def test_radius_zero_keeps_only_the_observed_component():
    """stride 1 and radius 0: delta_ij = [i == j], so dX[i, l] = (S V^T)[i, i] Z[i, l]."""
    nstate = nobs = 19
    nens = 6
    XB, dXB, V, Z = _problem(41, nstate, nobs, nens)
    XA = oracle.localized_update(XB, dXB, V, Z, 1, 5.0, 0.0)
    S = dXB / math.sqrt(nens - 1)                                    # (nens, nstate)
    diag = np.einsum("ki,ki->i", S, V)                                # (S V^T)[i, i]
    np.testing.assert_allclose(XA - XB, diag[None, :] * Z, rtol=1e-12, atol=1e-14)
    # stride 2, radius 0: unobserved (odd) components get no increment
    nobs2 = 10
    XB2, dXB2, V2, Z2 = _problem(42, 20, nobs2, nens)
    XA2 = oracle.localized_update(XB2, dXB2, V2, Z2, 2, 5.0, 0.0)
    np.testing.assert_array_equal((XA2 - XB2)[:, 1::2], 0.0)


def test_single_observation_is_the_paper_single_datum_localization():
    """One observation y_1 at state index 0: dX_{1} = Delta_hat S V^T Z_{1}, Delta_hat = diag of
    exp(-d(i, 0) / length), d the periodic distance (Sec. 3.1.2 and the weights of Sec. 4.2)."""
    nstate, nens = 40, 7
    XB, dXB, V, Z = _problem(51, nstate, 1, nens)
    length = float(nstate)
    XA = oracle.localized_update(XB, dXB, V, Z, 1, length, None)
    i = np.arange(nstate)
    dist = np.minimum(i, nstate - i)                                  # d(i, 0) on the ring
    w = np.exp(-dist / length)
    S = dXB / math.sqrt(nens - 1)
    sv = S.T @ V[:, 0]                                                # (S V^T)[:, 0]
    np.testing.assert_allclose((XA - XB), (w * sv)[None, :] * Z[:, :1], rtol=1e-12, atol=1e-14)
    # the two neighbours across the wrap-around get the same weight as the direct neighbours
    assert dist[1] == dist[nstate - 1] == 1


@pytest.mark.parametrize("radius", [None, 4.0])
def test_periodic_shift_symmetry(radius):
    """Rolling the state by s*stride and the observations by s rolls the increment by s*stride (the
    weights depend only on the periodic distance, Sec. 4.2)."""
    nstate, stride, nens = 30, 3, 5
    nobs = nstate // stride
    XB, dXB, V, Z = _problem(61, nstate, nobs, nens)
    dX = oracle.localized_update(XB, dXB, V, Z, stride, 9.0, radius) - XB
    s = 4
    XBr, dXBr = np.roll(XB, s * stride, axis=1), np.roll(dXB, s * stride, axis=1)
    Vr, Zr = np.roll(V, s, axis=1), np.roll(Z, s, axis=1)
    dXr = oracle.localized_update(XBr, dXBr, Vr, Zr, stride, 9.0, radius) - XBr
    np.testing.assert_allclose(dXr, np.roll(dX, s * stride, axis=1), rtol=1e-12, atol=1e-13)


def test_cut_off_zeroes_far_components():
    nstate, stride, nens = 48, 4, 5
    nobs = nstate // stride
    XB, dXB, V, Z = _problem(71, nstate, nobs, nens)
    # only observation 0 carries information
    Z[:, 1:] = 0.0
    dX = oracle.localized_update(XB, dXB, V, Z, stride, 10.0, 5.0) - XB
    i = np.arange(nstate)
    dist = np.minimum(i, nstate - i)
    assert np.all(dX[:, dist > 5] == 0.0)
    assert np.all(np.abs(dX[:, dist <= 5]) > 0.0)


# ----------------------------------------------------------------------------------------------
# block-diagonal R
# ----------------------------------------------------------------------------------------------

def _spd_blocks(seed, nblk, bs):
    out = np.zeros((nblk, bs, bs))
    for b in range(nblk):
        A = synth.normal_matrix(seed, 100 + b, bs, bs)
        out[b] = A @ A.T / bs + np.diag(synth.uniform(seed, 300 + b, bs, 0.5, 1.5))
    return out


def _dense_R(Rblk, nobs):
    nblk, bs, _ = Rblk.shape
    R = np.zeros((nobs, nobs))
    for b in range(nblk):
        r0 = b * bs
        m = min(bs, nobs - r0)
        R[r0:r0 + m, r0:r0 + m] = Rblk[b, :m, :m]
    return R


@pytest.mark.parametrize("nobs,bs,nens", [(24, 4, 5), (37, 8, 9), (50, 1, 6), (31, 31, 4), (40, 7, 12)])
def test_block_diagonal_solve_equals_dense_cholesky(nobs, bs, nens):
    nblk = (nobs + bs - 1) // bs
    Rblk = _spd_blocks(81 + nobs, nblk, bs)
    V = synth.normal_matrix(82, 1, nobs, nens, std=1.0 / math.sqrt(nens - 1))
    D = synth.normal_matrix(82, 2, nobs, nens)
    Z, gamma = oracle.ism_solve_blockdiag(Rblk, V, D, return_gamma=True)
    R = _dense_R(Rblk, nobs)
    W = R + V.T @ V
    want = sla.cho_solve(sla.cho_factor(W), D.T).T
    np.testing.assert_allclose(Z, want, rtol=1e-11, atol=1e-12)
    assert np.all(gamma >= 1.0)


def test_block_size_one_is_the_diagonal_step1():
    nobs, nens = 33, 7
    r = synth.uniform(91, 1, nobs, 0.5, 1.5)
    V = synth.normal_matrix(91, 2, nobs, nens)
    D = synth.normal_matrix(91, 3, nobs, nens)
    U1, Z1 = oracle.ism_step1_blockdiag(r.reshape(nobs, 1, 1), V, D)
    U0, Z0 = oracle.ism_step1(r, V, D)
    np.testing.assert_allclose(U1, U0, rtol=1e-15, atol=0)
    np.testing.assert_allclose(Z1, Z0, rtol=1e-15, atol=0)


def test_block_diagonal_woodbury():
    """Z = R^-1 D - R^-1 V (I + V^T R^-1 V)^-1 V^T R^-1 D (eq. SWM) with R^-1 applied by blocks."""
    nobs, bs, nens = 45, 6, 8
    nblk = (nobs + bs - 1) // bs
    Rblk = _spd_blocks(95, nblk, bs)
    V = synth.normal_matrix(96, 1, nobs, nens, std=0.5)
    D = synth.normal_matrix(96, 2, nobs, nens)
    Ri = np.linalg.inv(_dense_R(Rblk, nobs))
    RiV, RiD = Ri @ V.T, Ri @ D.T
    want = RiD - RiV @ np.linalg.solve(np.eye(nens) + V @ RiV, V @ RiD)
    np.testing.assert_allclose(oracle.ism_solve_blockdiag(Rblk, V, D), want.T, rtol=1e-11, atol=1e-12)


def test_block_not_positive_definite_is_rejected():
    Rblk = _spd_blocks(97, 3, 4)
    Rblk[1] = -np.eye(4)
    V = synth.normal_matrix(98, 1, 12, 3)
    D = synth.normal_matrix(98, 2, 12, 3)
    with pytest.raises(FloatingPointError, match="block 1"):
        oracle.ism_step1_blockdiag(Rblk, V, D)


# ----------------------------------------------------------------------------------------------
# pivoting (Sec. 3.4)
# ----------------------------------------------------------------------------------------------

def _piv_problem(seed, nobs, nens):
    r = synth.uniform(seed, 1, nobs, 0.5, 1.5)
    V = synth.normal_matrix(seed, 2, nobs, nens, std=1.0 / math.sqrt(nens - 1),
                            row_scale=synth.uniform(seed, 5, nobs, 0.2, 3.0))
    D = synth.normal_matrix(seed, 3, nobs, nens)
    return r, V, D


@pytest.mark.parametrize("nobs,nens", [(30, 4), (64, 9), (200, 16), (17, 17)])
def test_pivoted_solve_equals_dense_cholesky_and_the_unpivoted_solve(nobs, nens):
    r, V, D = _piv_problem(401 + nobs, nobs, nens)
    Z, gamma, perm = oracle.ism_solve_pivot(r, V, D)
    W = np.diag(r) + V.T @ V
    want = sla.cho_solve(sla.cho_factor(W), D.T).T
    np.testing.assert_allclose(Z, want, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(Z, oracle.ism_solve(r, V, D), rtol=1e-11, atol=1e-12)
    assert sorted(perm.tolist()) == list(range(nens))
    assert np.all(gamma >= 1.0)


@pytest.mark.parametrize("nobs,nens", [(12, 3), (20, 5), (9, 6)])
def test_pivot_is_the_largest_gamma_among_the_remaining_columns(nobs, nens):
    """Brute force of eq. EnKSM:gamma-value: at level k the candidate gamma of column i is
    1 + v_i^T W^{-1} v_i with W = R + sum of v v^T over the columns already used (dense solve)."""
    r, V, D = _piv_problem(433 + nobs, nobs, nens)
    _, gamma, perm = oracle.ism_solve_pivot(r, V, D)
    used = []
    for k in range(nens):
        W = np.diag(r) + sum((np.outer(V[p], V[p]) for p in used), np.zeros((nobs, nobs)))
        cand = {i: 1.0 + V[i] @ np.linalg.solve(W, V[i]) for i in range(nens) if i not in used}
        best = max(cand, key=lambda i: (abs(cand[i]), -i))
        assert perm[k] == best
        assert gamma[k] == pytest.approx(cand[best], rel=1e-12)
        used.append(best)
    assert perm.tolist() != list(range(nens))    # these inputs do reorder the columns


@pytest.mark.parametrize("nobs,nens", [(40, 7), (100, 12)])
def test_pivoted_long_operation_count_is_seven_halves(nobs, nens):
    """Sec. 3.4: T_SMF^PIV = 3 (N^2 Nobs + N Nobs) + Nobs per candidate = (7/2)(N^2 Nobs + N Nobs)."""
    r, V, D = _piv_problem(461, nobs, nens)
    _, _, _, ops = oracle.ism_solve_pivot(r, V, D, count_longops=True)
    assert ops == 7 * (nens * nens * nobs + nens * nobs) // 2
