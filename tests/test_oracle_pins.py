"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a textbook
dense solve, a closed form, an invariant the paper proves, a brute-force
evaluation of the paper's recursive definition, or the worked example of
Sec. 3.1.  The cases are chosen so that a dropped term, a wrong sign or index,
or a transposed operand in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def random_problem(seed, nobs, nens, nrhs=None, spread=1.0):
    """Random (r, V, D) with V of spread s_j/sqrt(nens-1) per row, r in [0.5, 1.5]."""
    nrhs = nens if nrhs is None else nrhs
    s = synth.uniform(seed, 1, nobs, 0.5, 2.0) * spread
    V = synth.normal_matrix(seed, 2, nobs, nens, std=1.0 / math.sqrt(max(nens - 1, 1)), row_scale=s)
    r = synth.uniform(seed, 3, nobs, 0.5, 1.5)
    D = synth.normal_matrix(seed, 4, nobs, nrhs)
    return r, V, D


def dense_W(r, V):
    Vm = V.T                       # nobs x nens
    return np.diag(r) + Vm @ Vm.T


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# ---------------------------------------------------------------------------
# The solve Z = (R + V V^T)^{-1} D
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("nobs,nens", [(1, 1), (2, 3), (7, 5), (33, 16), (64, 31), (200, 8)])
def test_solve_matches_dense_cholesky(nobs, nens):
    """Theorem 3 (Sec. 3.3): Z is the unique solution; the paper's Cholesky EnKF
    (Sec. 4.1, DPOTRF) computes the same Z.  Textbook Cholesky on tiny inputs."""
    r, V, D = random_problem(1000 + nobs * 7 + nens, nobs, nens)
    Z = oracle.ism_solve(r, V, D)
    W = dense_W(r, V)
    Zc = sla.cho_solve(sla.cho_factor(W), D.T).T
    assert rel(Z, Zc) < 1e-12


def test_solve_matches_woodbury_closed_form():
    """Eq. (SWM) applied once to R + V V^T (ensemble-space form, cf. eq.
    SVD:solution-linear-system): Z = R^-1 D - R^-1 V (I + V^T R^-1 V)^-1 V^T R^-1 D."""
    nobs, nens = 3000, 48
    r, V, D = random_problem(77, nobs, nens)
    Z = oracle.ism_solve(r, V, D)
    Vm, Dm = V.T, D.T
    RiV, RiD = Vm / r[:, None], Dm / r[:, None]
    G = np.eye(nens) + Vm.T @ RiV
    Zw = RiD - RiV @ np.linalg.solve(G, Vm.T @ RiD)
    assert rel(Z, Zw.T) < 1e-11


def test_single_member_sherman_morrison():
    """Nens = 1: one application of eq. (SWM), eqs. (EnKSM:solution-sherman-morrison)
    and (EnKMS:z-columns) with W^(0) = R: z = f - g (v^T f)/(1 + v^T g), f = R^-1 d,
    g = R^-1 v.  Several right-hand sides share the same v."""
    nobs = 257
    r, V, D = random_problem(5, nobs, 1, nrhs=4)
    Z, gamma = oracle.ism_solve(r, V, D, return_gamma=True)
    v = V[0]
    g = v / r
    for i in range(4):
        f = D[i] / r
        z = f - g * (v @ f) / (1.0 + v @ g)
        assert rel(Z[i], z) < 1e-14
    assert gamma[0] == pytest.approx(1.0 + v @ g, rel=1e-14)


def _recursive_S(x, k, r, Vm):
    """The recursive Sherman-Morrison formula S(x, k) = W^(k)^-1 x of Sec. 3
    (eq. EnKSM:recursive-solution), evaluated literally: exponential cost."""
    if k == 0:
        return x / r
    vk = Vm[:, k - 1]
    f = _recursive_S(x, k - 1, r, Vm)
    g = _recursive_S(vk, k - 1, r, Vm)
    return f - g * (vk @ f) / (1.0 + vk @ g)


@pytest.mark.parametrize("nens", [1, 2, 3, 5, 7])
def test_matches_brute_force_recursion(nens):
    """The iteration of Sec. 3.1 removes the repeated solves of the recursion
    (Fig. sherman-full) but must give the same values."""
    nobs = 19
    r, V, D = random_problem(300 + nens, nobs, nens)
    Z = oracle.ism_solve(r, V, D)
    Vm = V.T
    for i in range(nens):
        zi = _recursive_S(D[i], nens, r, Vm)
        assert rel(Z[i], zi) < 1e-13


def test_zero_deviations_give_R_inverse_D():
    """V = 0: every gamma_k = 1 and Z = R^-1 D (Step 1 alone)."""
    nobs, nens = 50, 6
    r, V, D = random_problem(9, nobs, nens)
    V[:] = 0.0
    Z, gamma = oracle.ism_solve(r, V, D, return_gamma=True)
    assert np.array_equal(gamma, np.ones(nens))
    np.testing.assert_array_equal(Z, D / r[None, :])


def test_orthogonal_columns_closed_form():
    """R = sigma^2 I and mutually orthogonal v_i: W^-1 = sigma^-2 (I - sum_i v_i v_i^T /
    (sigma^2 + |v_i|^2)), an exact closed form."""
    nobs, nens, sigma2 = 40, 5, 0.7
    Q, _ = np.linalg.qr(synth.normal_matrix(11, 1, nobs, nens).T)
    scales = np.array([0.3, 1.0, 2.5, 0.01, 7.0])
    Vm = Q * scales[None, :]
    V = np.ascontiguousarray(Vm.T)
    r = np.full(nobs, sigma2)
    D = synth.normal_matrix(11, 2, nobs, 3)
    Z = oracle.ism_solve(r, V, D)
    Winv = (np.eye(nobs) - sum(np.outer(Vm[:, i], Vm[:, i]) / (sigma2 + scales[i] ** 2)
                               for i in range(nens))) / sigma2
    assert rel(Z, (Winv @ D.T).T) < 1e-13


def test_gamma_values_and_theorem2():
    """Theorem 2 (Sec. 3.3): gamma_k = 1 + v_k^T W^(k-1)^-1 v_k > 1, with
    W^(k-1) = R + sum_{i<k} v_i v_i^T formed densely."""
    nobs, nens = 30, 9
    r, V, D = random_problem(21, nobs, nens)
    _, gamma = oracle.ism_solve(r, V, D, return_gamma=True)
    Vm = V.T
    for k in range(nens):
        Wk = np.diag(r) + Vm[:, :k] @ Vm[:, :k].T
        expect = 1.0 + Vm[:, k] @ np.linalg.solve(Wk, Vm[:, k])
        assert gamma[k] == pytest.approx(expect, rel=1e-12)
        assert gamma[k] > 1.0


def test_permutation_invariance():
    """W = R + sum_i v_i v_i^T does not depend on the order of the columns of V, so
    neither does Z (the premise of the pivoting of Sec. 3.4)."""
    nobs, nens = 60, 12
    r, V, D = random_problem(31, nobs, nens)
    Z = oracle.ism_solve(r, V, D)
    perm = np.array([5, 0, 11, 3, 2, 9, 1, 8, 10, 4, 7, 6])
    Zp = oracle.ism_solve(r, np.ascontiguousarray(V[perm]), D)
    assert rel(Zp, Z) < 1e-13


def test_residual_small_at_moderate_size():
    """Backward stability check: |(R + V V^T) Z - D| is at rounding level, with the
    product formed by numpy independently of the oracle."""
    nobs, nens = 20000, 64
    r, V, D = random_problem(41, nobs, nens)
    Z = oracle.ism_solve(r, V, D)
    Vm, Zm, Dm = V.T, Z.T, D.T
    Res = Dm - (r[:, None] * Zm + Vm @ (Vm.T @ Zm))
    denom = np.abs(r).max() * np.linalg.norm(Zm) + np.linalg.norm(Vm) ** 2 * np.linalg.norm(Zm) + np.linalg.norm(Dm)
    assert np.linalg.norm(Res) / denom < 4 * nens * np.finfo(float).eps
    # the oracle's own residual routine agrees with the numpy product on a
    # trial Z that is not the solution (residual of order one)
    Zt = Z + synth.normal_matrix(42, 1, nobs, nens)
    Rt = Dm - (r[:, None] * Zt.T + Vm @ (Vm.T @ Zt.T))
    Ro = oracle.residual(r, V, D, Zt)
    assert rel(Ro, Rt.T) < 1e-13


def test_long_operation_count():
    """Sec. 3.2: T_step1 = 2 Nobs Nens, T_step2 = 3 Nens^2 Nobs + Nens Nobs,
    T_SMF = 3 (Nens^2 Nobs + Nens Nobs) long operations."""
    for nobs, nens in [(10, 1), (37, 4), (100, 13)]:
        r, V, D = random_problem(51, nobs, nens)
        _, ops = oracle.ism_solve(r, V, D, count_longops=True)
        assert ops == 3 * (nens * nens * nobs + nens * nobs)


def _parse_worked_example():
    facts = []
    with open(os.path.join(GOLDEN, "worked_example_nens3.txt")) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                facts.append(line.split())
    return facts


def _state_after_levels(V, U0, Z0, k):
    """(U, Z) after levels 1..k of Step 2.  At levels m <= k a column u_i with
    i > k is updated by the same rule as a column of Z, so the oracle's Step 2
    run on the first k columns of V with [u_{k+1..Nens}, Z] as right-hand sides
    performs exactly those levels."""
    nens = V.shape[0]
    if k == 0:
        return U0.copy(), Z0.copy()
    Vk = np.array(V[:k], copy=True)
    Uk = np.array(U0[:k], copy=True)
    rhs = np.array(np.vstack([U0[k:], Z0]), copy=True)
    oracle.ism_levels(Vk, Uk, rhs)
    return np.vstack([Uk, rhs[: nens - k]]), rhs[nens - k:]


def test_worked_example_nens3():
    """The Nens = 3 derivation of Sec. 3.1: which columns each level updates and
    what the iterates equal at the end (golden fixture, read as text)."""
    facts = _parse_worked_example()
    nobs, nens = 11, 3
    r, V, D = random_problem(61, nobs, nens)
    Vm = V.T
    U0, Z0 = oracle.ism_step1(r, V, D)
    np.testing.assert_array_equal(U0, V / r[None, :])        # level 0
    np.testing.assert_array_equal(Z0, D / r[None, :])

    def W(m):
        return np.diag(r) + Vm[:, :m] @ Vm[:, :m].T

    prevU, prevZ = U0, Z0
    for k in range(1, nens + 1):
        U, Z = _state_after_levels(V, U0, Z0, k)
        changed = [f"u{i + 1}" for i in range(nens) if not np.array_equal(U[i], prevU[i])]
        changed += [f"z{i + 1}" for i in range(nens) if not np.array_equal(Z[i], prevZ[i])]
        expect = next(f for f in facts if f[0] == "level" and int(f[1]) == k)[3:]
        assert changed == expect, (k, changed, expect)
        prevU, prevZ = U, Z
    # the full run agrees with the level-by-level one
    assert rel(oracle.ism_solve(r, V, D), prevZ) < 1e-15
    n_final = 0
    for f in facts:
        if f[:2] == ["final", "U"]:
            i, m = int(f[2]), int(f[5])
            assert rel(prevU[i - 1], np.linalg.solve(W(m), Vm[:, i - 1])) < 1e-13
            n_final += 1
        elif f[:2] == ["final", "Z"]:
            m = int(f[4])
            assert rel(prevZ, np.linalg.solve(W(m), D.T).T) < 1e-13
            n_final += 1
    assert n_final == 4


# ---------------------------------------------------------------------------
# Analysis assembly and observation space
# ---------------------------------------------------------------------------

def test_observation_space_matches_sample_covariance():
    """S S^T is the ensemble covariance (eq. EnKSM:covariance-matrix), so
    V V^T = H P_B H^T with P_B from numpy's unbiased sample covariance."""
    nstate, nens, stride = 30, 9, 3
    XB = synth.normal_matrix(71, 1, nstate, nens, mean=2.0)
    xbar, dXB = oracle.ensemble_deviations(XB)
    np.testing.assert_allclose(xbar, XB.mean(axis=0), rtol=1e-14)
    np.testing.assert_allclose(dXB.sum(axis=0), 0.0, atol=1e-13)
    nobs = nstate // stride
    V = oracle.observe_deviations(dXB, nobs, stride)
    PB = np.cov(XB.T, ddof=1)                   # nstate x nstate
    HPH = PB[::stride, ::stride][:nobs, :nobs]
    np.testing.assert_allclose(V.T @ V, HPH, rtol=1e-12, atol=1e-13)


def test_M_matches_ensemble_space_form():
    """M = V^T Z / sqrt(Nens-1) = (I + V^T R^-1 V)^-1 V^T R^-1 D / sqrt(Nens-1)."""
    nobs, nens = 500, 10
    r, V, D = random_problem(81, nobs, nens)
    Z = oracle.ism_solve(r, V, D)
    M = oracle.vtz(V, Z)
    Vm, Dm = V.T, D.T
    G = np.eye(nens) + Vm.T @ (Vm / r[:, None])
    Mw = np.linalg.solve(G, Vm.T @ (Dm / r[:, None])) / math.sqrt(nens - 1)
    assert rel(M, Mw) < 1e-12


def test_full_analysis_matches_textbook_enkf():
    """Eqs. (EnKF:ensemble-analysis) and (EnKF:kalman-gain) on a small Lorenz-96
    ensemble: X_A = X_B + K (Y - H X_B), K = P_B H^T (H P_B H^T + R)^-1, dense."""
    d = synth.lorenz_small_draws()
    nstate, nens, nobs, stride, rv = d["nstate"], d["nens"], d["nobs"], d["obs_stride"], d["r"]
    truth = oracle.l96_rk4(d["truth0"], F=d["F"], dt=0.01, nsteps=1000)[0]
    XB = truth[None, :] + d["ens_noise"]
    y = truth[::stride] + d["obs_noise"]
    Y = y[None, :] + d["pert"]
    xbar, dXB = oracle.ensemble_deviations(XB)
    V = oracle.observe_deviations(dXB, nobs, stride)
    D = oracle.innovations(Y, XB, stride)
    r = np.full(nobs, rv)
    out = oracle.analysis(r, V, D, XB, dXB)
    H = np.zeros((nobs, nstate))
    H[np.arange(nobs), np.arange(nobs) * stride] = 1.0
    PB = np.cov(XB.T, ddof=1)
    K = PB @ H.T @ np.linalg.inv(H @ PB @ H.T + np.diag(r))
    XA = XB.T + K @ (Y.T - H @ XB.T)
    assert rel(out["XA"], XA.T) < 1e-12
    # the analysis mean equals the Kalman update of the mean (linearity)
    xa_mean = xbar + K @ (Y.mean(axis=0) - H @ xbar)
    np.testing.assert_allclose(out["XA"].mean(axis=0), xa_mean, rtol=1e-12, atol=1e-12)


def test_xa_update_alias_and_zero_M():
    """X_A = X_B + dX_B M: zero M returns X_B exactly; one unit column of M adds one
    deviation column."""
    nstate, nens = 17, 4
    XB = synth.normal_matrix(91, 1, nstate, nens)
    dXB = synth.normal_matrix(91, 2, nstate, nens)
    np.testing.assert_array_equal(oracle.analysis_update(XB, dXB, np.zeros((nens, nens))), XB)
    M = np.zeros((nens, nens))
    M[2, 1] = 1.0
    XA = oracle.analysis_update(XB, dXB, M)
    np.testing.assert_array_equal(XA[1], XB[1] + dXB[2])
    np.testing.assert_array_equal(XA[0], XB[0])


# ---------------------------------------------------------------------------
# Lorenz-96 and RK4 (Sec. 4.2)
# ---------------------------------------------------------------------------

def test_l96_fixed_point():
    """x_i = F for all i is an equilibrium of eq. (eqn:Lorenz96)."""
    x = np.full(40, 8.0)
    np.testing.assert_array_equal(oracle.l96_rhs(x, 8.0), np.zeros(40))
    np.testing.assert_array_equal(oracle.l96_rk4(x, 8.0, 0.01, 10)[0], x)


def test_l96_energy_identity():
    """The advection term of eq. (eqn:Lorenz96) conserves energy: sum_i x_i
    (x_{i+1} - x_{i-2}) x_{i-1} = 0 for periodic indices, so
    sum_i x_i dx_i/dt = -|x|^2 + F sum_i x_i.  A wrong index breaks it."""
    for n in (5, 6, 40, 101):
        x = synth.normal_matrix(100 + n, 1, n, 1)[0] * 3.0 + 1.0
        dx = oracle.l96_rhs(x, 8.0)
        assert x @ dx == pytest.approx(-(x @ x) + 8.0 * x.sum(), rel=1e-12, abs=1e-10)
        # and the forcing/damping part: rhs at F=0 of a constant vector is -x
        c = np.full(n, 2.5)
        np.testing.assert_allclose(oracle.l96_rhs(c, 0.0), -c)


def test_l96_explicit_wraparound_cases():
    """The paper writes the periodic cases i = 1 and i = Nstate explicitly; check
    them on a vector of distinct integers (exact arithmetic)."""
    n = 7
    x = np.arange(1.0, n + 1.0) ** 2
    dx = oracle.l96_rhs(x, 8.0)
    # i = 1 (1-based): (x_2 - x_{N-1}) x_N - x_1 + F
    assert dx[0] == (x[1] - x[n - 2]) * x[n - 1] - x[0] + 8.0
    # i = N: (x_1 - x_{N-2}) x_{N-1} - x_N + F
    assert dx[n - 1] == (x[0] - x[n - 3]) * x[n - 2] - x[n - 1] + 8.0


def test_rk4_fourth_order_convergence():
    """Classical RK4 has global error O(dt^4): halving dt divides the error by ~16
    (a wrong stage coefficient drops the order)."""
    from scipy.integrate import solve_ivp
    n = 12
    x0 = 8.0 + synth.normal_matrix(7, 1, n, 1)[0]
    T = 0.4

    def f(t, x):
        return oracle.l96_rhs(x, 8.0)

    ref = solve_ivp(f, (0, T), x0, method="DOP853", rtol=1e-13, atol=1e-13).y[:, -1]
    errs = []
    for dt in (0.04, 0.02, 0.01):
        xt = oracle.l96_rk4(x0, 8.0, dt, int(round(T / dt)))[0]
        errs.append(np.linalg.norm(xt - ref))
    ratio1, ratio2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 12.0 < ratio1 < 20.0 and 12.0 < ratio2 < 20.0, errs


def test_vtz_is_accurate_under_cancellation():
    """M = V^T Z / sqrt(N - 1) (Sec. 3.1) where the sums cancel: Z made almost orthogonal to the
    columns of V, as the solve makes the part of Z in range(V) small.  The oracle's entries
    must match exact rational arithmetic (fractions.Fraction on the same FP64 values)
    within the Dot2 error bound of Ogita, Rump and Oishi, |res - exact| <= u |exact| +
    gamma_{n-1}^2 sum |v_j z_j| (gamma_n = n u / (1 - n u)), plus one rounding for the
    scaling by 1/sqrt(N - 1); the plain FP64 sum misses by far more than that bound."""
    from fractions import Fraction
    nobs, nens, nrhs = 3000, 4, 3
    V = synth.normal_matrix(811, 1, nobs, nens)
    Z = synth.normal_matrix(811, 2, nobs, nrhs)
    # remove the range(V) part of Z in FP64 (leaves a residue of rounding size)
    Q, _ = np.linalg.qr(V.T)
    Z = Z - (Z @ Q) @ Q.T
    M = oracle.vtz(V, Z)
    plain_worst = 0.0
    for k in range(nens):
        for i in range(nrhs):
            exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(V[k], Z[i]))
            scale = 1.0 / math.sqrt(nens - 1)
            want = float(exact) * scale
            u = 2.0 ** -53
            gam = (nobs - 1) * u / (1 - (nobs - 1) * u)
            bound = (3 * u * abs(float(exact)) + gam ** 2 * float(np.sum(np.abs(V[k] * Z[i])))) * scale
            assert abs(M[k, i] - want) <= bound, (k, i, M[k, i], want, bound)
            plain = float(np.sum(V[k] * Z[i])) * scale
            plain_worst = max(plain_worst, abs(plain - want) / bound)
    assert plain_worst > 100.0        # the case really cancels: the plain sum misses by > 100 bounds


def test_refined_solve_gives_the_m_of_the_exact_solution():
    """M = V^T Z / sqrt(N - 1) with Z the solution of (R + V V^T) Z = D (Sec. 3.1), at gamma ~ 1e6.
    Exact rational arithmetic on the same FP64 inputs gives V^T Z = (I + V^T R^-1 V)^-1 V^T R^-1 D
    (the ensemble-space form of the Woodbury identity, eq. SWM).  Any Z stored in FP64 carries
    a rounding of ~u |Z| that the damping of range(V) does not shrink, so V^T Z can be no
    closer than ~u gamma_max: the refined oracle must be within that bound, and the plain
    solve (one pass of Step 2, whose rounding accumulates over the levels) is not."""
    from fractions import Fraction

    def exact_vtz(r, V, D):
        nens, nobs = V.shape
        rf = [Fraction(float(x)) for x in r]
        Vf = [[Fraction(float(x)) for x in row] for row in V]
        Df = [[Fraction(float(x)) for x in row] for row in D]
        A = [[(1 if k == m else 0) + sum(Vf[k][j] * Vf[m][j] / rf[j] for j in range(nobs)) for m in range(nens)]
             for k in range(nens)]
        B = [[sum(Vf[k][j] * Df[i][j] / rf[j] for j in range(nobs)) for i in range(D.shape[0])] for k in range(nens)]
        for c in range(nens):                       # Gauss-Jordan, exact (A is SPD: no pivoting needed)
            for rr in range(nens):
                if rr != c:
                    f = A[rr][c] / A[c][c]
                    A[rr] = [a - f * b for a, b in zip(A[rr], A[c])]
                    B[rr] = [a - f * b for a, b in zip(B[rr], B[c])]
        return np.array([[float(B[k][i] / A[k][k]) for i in range(D.shape[0])] for k in range(nens)])

    u = 2.0 ** -53
    for seed in (1, 2, 3):
        nobs, nens, nrhs = 300, 4, 3
        V = 58.0 * synth.normal_matrix(900 + seed, 1, nobs, nens)
        D = synth.normal_matrix(900 + seed, 2, nobs, nrhs)
        r = synth.uniform(900 + seed, 3, nobs, 0.5, 1.5)
        want = exact_vtz(r, V, D) / math.sqrt(nens - 1)
        err = lambda M: np.linalg.norm(M - want) / np.linalg.norm(want)
        Zr, gamma = oracle.ism_solve_refined(r, V, D, return_gamma=True)
        bound = u * gamma.max()
        assert 5e5 < gamma.min() and gamma.max() < 5e6, gamma
        assert err(oracle.vtz(V, Zr)) <= bound, (seed, err(oracle.vtz(V, Zr)), bound)
        assert err(oracle.vtz(V, oracle.ism_solve(r, V, D))) > bound     # the plain solve misses it
        ref = oracle.analysis(r, V, D, np.zeros((nens, 5)), np.zeros((nens, 5)))
        assert np.array_equal(ref["M"], oracle.vtz(V, Zr))
