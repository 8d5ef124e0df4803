"""Two identities of the level recurrence that the GPU paths use in place of literal sums,
checked on the CPU in FP64.

Step 2 of Sec. 3.1 (eqs. SM-step-2-h/Z/u) applies level k to a column x as x <- x - h_k c_k,
with c_k = v_k^T x^(k-1) and h_k = u_k^(k-1) / gamma_k.  Two consequences:

1. V^T Z from the recurrence's own coefficients.  For k < m, v_k^T Z^(m) = v_k^T Z^(m-1) -
   (v_k^T h_m) c_m, and v_k^T Z^(k) = c_k / gamma_k, so
       V^T Z = (I - triu(Q, 1)) diag(1 / gamma) C,   Q_km = v_k^T u_m^(m-1)  (the final U columns).
   The library forms M = V^T Z / sqrt(N - 1) this way, and in the refinement P = V^T Z1 and
   V^T delta from the solve's and the correction's coefficients.
2. The levels of one panel P applied with stored factors.  Within P, c = (I + L)^-1 a with
   a = V_P^T x and L_ml = v_m^T h_l (l < m in P), so the panel maps x to
       x - U_fin,P diag(1 / gamma_P) (I + L)^-1 V_P^T x.
   The refinement's correction sweep applies the solve's operator to the residual this way,
   from the final U columns and diag(1/gamma)(I + L)^-1 kept by the solve.

The transcription of the levels below is anchored to the oracle (same Z and gamma); the
identities are then held to the oracle's solve of other right-hand sides and to the closed
ensemble-space form V^T Z = (I + V R^-1 V^T)^-1 V R^-1 D^T (eq. SWM).  Dropping the diagonal
of Q from triu, the 1/gamma scaling, or the (I + L)^-1 fails them by orders of magnitude.
"""
import numpy as np
import pytest

import oracle
import synth

SEED = 7711
NOBS, NENS, NRHS = 300, 13, 5


def _problem(seed=SEED, nobs=NOBS, nens=NENS, nrhs=NRHS):
    s = synth.uniform(seed, 1, nobs, 0.5, 2.0)
    V = synth.normal_matrix(seed, 2, nobs, nens, std=1.0 / np.sqrt(nens - 1), row_scale=s)
    r = synth.uniform(seed, 3, nobs, 0.5, 1.5)
    D = synth.normal_matrix(seed, 4, nobs, nrhs)
    return r, V, D


def _levels(r, V, D):
    """Step 1 and Step 2 in the paper's order, recording the per-level coefficients c_k of the
    columns of D (C[k, i] = v_k^T z_i^(k-1)), the final U columns u_k^(k-1) and gamma."""
    n = V.shape[0]
    U = V / r
    Z = D / r
    C = np.zeros((n, D.shape[0]))
    gamma = np.zeros(n)
    ufin = np.zeros_like(U)
    for k in range(n):
        gamma[k] = 1.0 + V[k] @ U[k]
        ufin[k] = U[k]
        h = U[k] / gamma[k]
        C[k] = Z @ V[k]
        Z = Z - np.outer(C[k], h)
        U[k + 1:] = U[k + 1:] - np.outer(U[k + 1:] @ V[k], h)
    return Z, gamma, C, ufin


def _closed_vtz(r, V, D):
    """V^T Z = (I + V R^-1 V^T)^-1 V R^-1 D^T (rows = members, columns = right-hand sides)."""
    VR = V / r
    return np.linalg.solve(np.eye(V.shape[0]) + VR @ V.T, VR @ D.T)


def _identity(Q, gamma, C):
    return (np.eye(len(gamma)) - np.triu(Q, 1)) @ (C / gamma[:, None])


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_transcription_matches_the_oracle():
    r, V, D = _problem()
    Z, gamma, _, _ = _levels(r, V, D)
    Zo, go = oracle.ism_solve(r, V, D, return_gamma=True)
    assert _rel(Z, Zo) <= 1e-13
    np.testing.assert_allclose(gamma, go, rtol=1e-14)


def test_vtz_from_the_level_coefficients():
    r, V, D = _problem()
    _, gamma, C, ufin = _levels(r, V, D)
    Q = V @ ufin.T                                   # Q[k, m] = v_k^T u_m^(m-1)
    want = _closed_vtz(r, V, D)
    assert _rel(_identity(Q, gamma, C), want) <= 1e-12
    # and the literal sums of the oracle's Z (M = V^T Z / sqrt(N - 1))
    Zo = oracle.ism_solve(r, V, D)
    assert _rel(_identity(Q, gamma, C) / np.sqrt(NENS - 1), oracle.vtz(V, Zo)) <= 1e-12
    # the forms a slip would give are far off
    assert _rel((np.eye(NENS) - np.triu(Q, 0)) @ (C / gamma[:, None]), want) > 1e-3
    assert _rel((np.eye(NENS) - np.triu(Q, 1)) @ C, want) > 1e-3


@pytest.mark.parametrize("b", [1, 4, 7, 13])
def test_panel_sweep_with_stored_factors_applies_the_solve(b):
    r, V, D = _problem()
    _, gamma, _, ufin = _levels(r, V, D)
    Q = V @ ufin.T
    E = synth.normal_matrix(SEED, 9, NOBS, 3)        # other right-hand sides (a residual)
    X = E / r                                        # Step 1 of the residual
    Cd = np.zeros((NENS, E.shape[0]))
    for k0 in range(0, NENS, b):
        P = slice(k0, min(k0 + b, NENS))
        bp = P.stop - P.start
        # the solve's stored factors of the panel: W = diag(1/gamma_P) (I + L)^-1, L_ml = v_m^T h_l
        L = np.tril(V[P] @ (ufin[P] / gamma[P, None]).T, -1)
        W = np.diag(1.0 / gamma[P]) @ np.linalg.inv(np.eye(bp) + L)
        a = V[P] @ X.T                               # the panel's dots
        Cd[P] = np.linalg.solve(np.eye(bp) + L, a)   # the per-level coefficients c = (I + L)^-1 a
        X = X + (ufin[P].T @ (-W @ a)).T
    assert _rel(X, oracle.ism_solve(r, V, E)) <= 1e-12
    # V^T delta from the sweep's own coefficients, by the identity of the previous test
    assert _rel(_identity(Q, gamma, Cd), _closed_vtz(r, V, E)) <= 1e-12
    if b > 1:
        # without (I + L)^-1 the panel's levels would not see each other's updates
        Xs = E / r
        for k0 in range(0, NENS, b):
            P = slice(k0, min(k0 + b, NENS))
            Xs = Xs - (ufin[P].T @ ((V[P] @ Xs.T) / gamma[P, None])).T
        assert _rel(Xs, oracle.ism_solve(r, V, E)) > 1e-4
