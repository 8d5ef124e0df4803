"""Plain FP64 CPU oracle of the iterative Sherman-Morrison EnKF analysis.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this package.  It shares no code with
the CUDA library (``paper_1302_3876_gb300``) and never imports it.

The arithmetic lives in ``ism_oracle.c`` (compiled here with the host C
compiler, ``-O2 -fno-fast-math -ffp-contract=off``) and in ``surrogate.py``
(numpy, FP64).  This module only marshals numpy arrays.

Array convention: a column-major matrix with ``rows`` rows, ``cols`` columns and
leading dimension ``ld`` is a C-contiguous numpy array of shape ``(cols, ld)``;
entry (j, c) is ``a[c, j]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_DIR = os.path.join(_HERE, "_lib")
_LIB_PATH = os.path.join(_LIB_DIR, "libism_oracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile ism_oracle.c into oracle/_lib/libism_oracle.so (no-op when up to date)."""
    src = os.path.join(_HERE, "ism_oracle.c")
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src):
        return _LIB_PATH
    os.makedirs(_LIB_DIR, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math", "-ffp-contract=off",
                    "-o", tmp, src, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p
            sig = {
                "oracle_ensemble_deviations": ([i64, i32, vp, i64, vp, vp, i64], None),
                "oracle_observe_deviations": ([i64, i32, i32, vp, i64, vp, i64], None),
                "oracle_innovations": ([i64, i32, i32, vp, i64, vp, i64, vp, i64], None),
                "oracle_ism_step1": ([i64, i32, i32, vp, vp, i64, vp, i64, vp, i64, vp, i64, vp], None),
                "oracle_ism_step2": ([i64, i32, i32, vp, i64, vp, i64, vp, i64, vp, vp], ctypes.c_int),
                "oracle_ism_solve": ([i64, i32, i32, vp, vp, i64, vp, i64, vp, i64, vp, i64, vp, vp],
                                     ctypes.c_int),
                "oracle_vtz": ([i64, i32, i32, vp, i64, vp, i64, vp], None),
                "oracle_analysis_update": ([i64, i32, i32, vp, i64, vp, i64, vp, vp, i64], None),
                "oracle_residual": ([i64, i32, i32, vp, vp, i64, vp, i64, vp, i64, vp, i64], ctypes.c_int),
                "oracle_l96_rhs": ([i64, vp, dbl, vp], None),
                "oracle_l96_rk4": ([i64, i32, vp, i64, dbl, dbl, i32], ctypes.c_int),
                "oracle_inflate": ([i64, i32, dbl, vp, i64], None),
                "oracle_ism_step2_pivot": ([i64, i32, i32, vp, i64, vp, i64, vp, i64, vp, vp, vp], ctypes.c_int),
                "oracle_localized_increment_literal": ([i64, i64, i32, i32, i32, dbl, dbl, vp, i64, vp, i64, vp,
                                                        i64, vp, i64], None),
                "oracle_localized_update": ([i64, i64, i32, i32, i32, dbl, dbl, vp, i64, vp, i64, vp, i64, vp,
                                             i64, vp, i64], ctypes.c_int),
                "oracle_ism_step1_blockdiag": ([i64, i32, i32, i32, vp, vp, i64, vp, i64, vp, i64, vp, i64],
                                               ctypes.c_int),
            }
            for name, (args, res) in sig.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _f64(a, name):
    a = np.asarray(a)
    if a.dtype != np.float64 or not a.flags.c_contiguous:
        raise TypeError(f"{name} must be a C-contiguous float64 array")
    return a


def _mat(a, name, cols, rows):
    a = _f64(a, name)
    if a.ndim != 2 or a.shape[0] < cols or a.shape[1] < rows:
        raise ValueError(f"{name}: shape {a.shape} cannot hold {rows}x{cols}")
    return a, a.shape[1]


# ---------------------------------------------------------------------------
# Observation space (Sec. 2, Sec. 3)
# ---------------------------------------------------------------------------

def ensemble_deviations(XB, nstate=None):
    """Ensemble mean and deviations of X_B (eq. ensemble-background-mean)."""
    XB = _f64(XB, "XB")
    nens, ldb = XB.shape
    nstate = ldb if nstate is None else nstate
    xbar = np.empty(nstate)
    dXB = np.zeros((nens, ldb))
    _load().oracle_ensemble_deviations(nstate, nens, _p(XB), ldb, _p(xbar), _p(dXB), ldb)
    return xbar, dXB


def observe_deviations(dXB, nobs, stride):
    """V = H dX_B / sqrt(Nens-1), H = rows 0, stride, ... (eq. EnKSM:member-observations)."""
    dXB = _f64(dXB, "dXB")
    nens, ldx = dXB.shape
    if (nobs - 1) * stride >= ldx:
        raise ValueError("observation rows exceed the state")
    V = np.zeros((nens, nobs))
    _load().oracle_observe_deviations(nobs, nens, stride, _p(dXB), ldx, _p(V), nobs)
    return V


def innovations(Y, XB, stride):
    """D = Y - H X_B (eq. EnKSM:system-rhs)."""
    Y, XB = _f64(Y, "Y"), _f64(XB, "XB")
    nens, nobs = Y.shape
    D = np.zeros((nens, nobs))
    _load().oracle_innovations(nobs, nens, stride, _p(Y), nobs, _p(XB), XB.shape[1], _p(D), nobs)
    return D


# ---------------------------------------------------------------------------
# Iterative Sherman-Morrison formula (Sec. 3.1)
# ---------------------------------------------------------------------------

def ism_solve(r, V, D, nobs=None, return_gamma=False, count_longops=False):
    """Z = S_*(R, V, D): Step 1 (eq. SM-step-1) then Step 2 (eqs. SM-step-2-*).

    ``V`` has shape (nens, ldv), ``D`` shape (nrhs, ldd); ``r`` holds the nobs
    variances.  Returns Z with shape (nrhs, nobs), plus gamma_1..gamma_Nens and
    the long-operation count when asked.
    """
    r = _f64(r, "r")
    nobs = r.shape[0] if nobs is None else nobs
    V, ldv = _mat(V, "V", V.shape[0], nobs)
    D, ldd = _mat(D, "D", D.shape[0], nobs)
    nens, nrhs = V.shape[0], D.shape[0]
    U = np.zeros((nens, max(nobs, 1)))
    Z = np.zeros((nrhs, max(nobs, 1)))
    gamma = np.zeros(max(nens, 1))
    ops = ctypes.c_int64(0)
    st = _load().oracle_ism_solve(nobs, nens, nrhs, _p(r), _p(V), ldv, _p(D), ldd, _p(U), U.shape[1],
                                  _p(Z), Z.shape[1], _p(gamma), ctypes.byref(ops))
    if st != 0:
        raise FloatingPointError(f"iterative Sherman-Morrison stopped at level {st}")
    Z = Z[:, :nobs]
    out = [Z]
    if return_gamma:
        out.append(gamma[:nens])
    if count_longops:
        out.append(int(ops.value))
    return out[0] if len(out) == 1 else tuple(out)


def ism_step1(r, V, D):
    """Step 1 only: (U^(0), Z^(0)) = (R^{-1} V, R^{-1} D)."""
    r = _f64(r, "r")
    nobs = r.shape[0]
    V, ldv = _mat(V, "V", V.shape[0], nobs)
    D, ldd = _mat(D, "D", D.shape[0], nobs)
    U = np.zeros((V.shape[0], nobs))
    Z = np.zeros((D.shape[0], nobs))
    _load().oracle_ism_step1(nobs, V.shape[0], D.shape[0], _p(r), _p(V), ldv, _p(D), ldd, _p(U), nobs,
                             _p(Z), nobs, None)
    return U, Z


def ism_levels(V, U, Z, nobs=None):
    """Step 2 in place on U and Z (given Step 1's output); returns gamma."""
    V, U, Z = _f64(V, "V"), _f64(U, "U"), _f64(Z, "Z")
    nobs = U.shape[1] if nobs is None else nobs
    gamma = np.zeros(max(V.shape[0], 1))
    st = _load().oracle_ism_step2(nobs, V.shape[0], Z.shape[0], _p(V), V.shape[1], _p(U), U.shape[1],
                                  _p(Z), Z.shape[1], _p(gamma), None)
    if st != 0:
        raise FloatingPointError(f"iterative Sherman-Morrison stopped at level {st}")
    return gamma[:V.shape[0]]


def ism_solve_pivot(r, V, D, count_longops=False):
    """Z = S_*(R, V, D) with the pivoting of Sec. 3.4: Step 1, then Step 2 choosing at each level
    the remaining column with the largest |gamma|.  Returns (Z, gamma in level order, perm[, longops]),
    perm[k] = the original column index used at level k."""
    U, Z = ism_step1(r, V, D)
    V = _f64(np.ascontiguousarray(V[:, :r.shape[0]]), "V")
    nobs = r.shape[0]
    nens, nrhs = V.shape[0], Z.shape[0]
    gamma = np.zeros(max(nens, 1))
    perm = np.zeros(max(nens, 1), dtype=np.int32)
    ops = ctypes.c_int64(nobs * (nens + nrhs))            # Step 1: one division per entry of U and Z
    st = _load().oracle_ism_step2_pivot(nobs, nens, nrhs, _p(V), nobs, _p(U), nobs, _p(Z), nobs, _p(gamma),
                                        ctypes.c_void_p(perm.ctypes.data), ctypes.byref(ops))
    if st != 0:
        raise FloatingPointError(f"iterative Sherman-Morrison stopped at level {st}")
    out = (Z, gamma[:nens], perm[:nens])
    return out + (int(ops.value),) if count_longops else out


def vtz(V, Z, nobs=None):
    """M = V^T Z / sqrt(Nens-1), returned as a numpy (nens, nrhs) array (row = member m)."""
    V, Z = _f64(V, "V"), _f64(Z, "Z")
    nobs = V.shape[1] if nobs is None else nobs
    nens, nrhs = V.shape[0], Z.shape[0]
    M = np.zeros((nrhs, nens))      # column-major nens x nrhs
    _load().oracle_vtz(nobs, nens, nrhs, _p(V), V.shape[1], _p(Z), Z.shape[1], _p(M))
    return M.T.copy()


def analysis_update(XB, dXB, M, nstate=None):
    """X_A = X_B + dX_B M (SMEnKF analysis, Sec. 3.1).  M is (nens, nrhs)."""
    XB, dXB = _f64(XB, "XB"), _f64(dXB, "dXB")
    M = np.ascontiguousarray(np.asarray(M, dtype=np.float64).T)   # column-major nens x nrhs
    nens = dXB.shape[0]
    nrhs = M.shape[0]
    nstate = XB.shape[1] if nstate is None else nstate
    XA = np.zeros((nrhs, nstate))
    _load().oracle_analysis_update(nstate, nens, nrhs, _p(XB), XB.shape[1], _p(dXB), dXB.shape[1], _p(M),
                                   _p(XA), nstate)
    return XA


def residual(r, V, D, Z):
    """D - (R + V V^T) Z (eq. EnKSM:system-to-solve-V)."""
    r, V, D, Z = _f64(r, "r"), _f64(V, "V"), _f64(D, "D"), _f64(Z, "Z")
    nobs = r.shape[0]
    Res = np.zeros((Z.shape[0], nobs))
    _load().oracle_residual(nobs, V.shape[0], Z.shape[0], _p(r), _p(V), V.shape[1], _p(D), D.shape[1],
                            _p(Z), Z.shape[1], _p(Res), nobs)
    return Res


def ism_solve_refined(r, V, D, return_gamma=False):
    """Z with (R + V V^T) Z = D (Sec. 3.1) to FP64 accuracy in every direction.

    The ISM solve (Step 1, Step 2), then one step of classical iterative refinement with
    the residual of eq. EnKSM:system-to-solve-V: Z <- Z + S_*(R, V, D - (R + V V^T) Z).
    The solve's own rounding leaves in Z an error of ~1e-16 of |Z| in every direction,
    while the part of Z in range(V) is damped by 1/gamma_k (gamma ~ 8000 at the large
    workloads), so V^T Z computed from it is off by ~1e-10.  The correction's error in
    range(V) is damped by the same factor, which brings V^T Z to ~1e-13.  gamma is that
    of the first solve.
    """
    Z, gamma = ism_solve(r, V, D, return_gamma=True)
    Z = Z + ism_solve(r, V, residual(r, V, D, Z))
    return (Z, gamma) if return_gamma else Z


def analysis(r, V, D, XB, dXB, refine=True):
    """Full SMEnKF analysis: Z = S_*(R,V,D), M = V^T Z/sqrt(Nens-1), X_A = X_B + dX_B M.

    refine=True takes Z from ism_solve_refined (the reference for results whose error
    the damping in range(V) magnifies: M, X_A and the increment); refine=False is the
    paper's sequence of steps as written (one solve).
    """
    Z, gamma = ism_solve_refined(r, V, D, return_gamma=True) if refine else ism_solve(r, V, D, return_gamma=True)
    M = vtz(V, Z)
    XA = analysis_update(XB, dXB, M)
    return {"Z": Z, "gamma": gamma, "M": M, "XA": XA}


# ---------------------------------------------------------------------------
# Inflation, partial localization, block-diagonal R (Sec. 3.1.1, 3.1.2, 3.1)
# ---------------------------------------------------------------------------

def inflate(X, alpha):
    """x_i <- xbar + alpha (x_i - xbar) for every member (Sec. 3.1.1); returns a new array."""
    X = np.array(_f64(X, "X"), copy=True)
    _load().oracle_inflate(X.shape[1], X.shape[0], float(alpha), _p(X), X.shape[1])
    return X


def _loc_args(length, radius):
    return float(length), (-1.0 if radius is None else float(radius))


def localized_increment_literal(dXB, V, Z, stride, length, radius=None):
    """dX[i,l] = sum_k S[i,k] sum_j delta_ij V[j,k] Z[j,l] (eq. localized-correction-component),
    as printed; tiny inputs only.  radius None = no cut-off.  Returns dX with shape (nrhs, nstate)."""
    dXB, V, Z = _f64(dXB, "dXB"), _f64(V, "V"), _f64(Z, "Z")
    nens, nstate = dXB.shape
    nobs, nrhs = V.shape[1], Z.shape[0]
    if (nobs - 1) * stride >= nstate:
        raise ValueError("observation rows exceed the state")
    L, rad = _loc_args(length, radius)
    dX = np.zeros((nrhs, nstate))
    _load().oracle_localized_increment_literal(nstate, nobs, nens, nrhs, stride, L, rad, _p(dXB), nstate, _p(V),
                                               nobs, _p(Z), Z.shape[1], _p(dX), nstate)
    return dX


def localized_update(XB, dXB, V, Z, stride, length, radius=None):
    """X_A = X_B + (Delta o (S V^T)) Z (Sec. 3.1.2, matrix form).  Returns X_A (nrhs, nstate)."""
    XB, dXB, V, Z = _f64(XB, "XB"), _f64(dXB, "dXB"), _f64(V, "V"), _f64(Z, "Z")
    nens, nstate = dXB.shape
    nobs, nrhs = V.shape[1], Z.shape[0]
    if (nobs - 1) * stride >= nstate:
        raise ValueError("observation rows exceed the state")
    L, rad = _loc_args(length, radius)
    XA = np.zeros((nrhs, nstate))
    st = _load().oracle_localized_update(nstate, nobs, nens, nrhs, stride, L, rad, _p(dXB), nstate, _p(V), nobs,
                                         _p(Z), Z.shape[1], _p(XB), XB.shape[1], _p(XA), nstate)
    if st != 0:
        raise MemoryError("oracle_localized_update failed")
    return XA


def ism_step1_blockdiag(Rblk, V, D):
    """Step 1 with block-diagonal R (Sec. 3.1): (U^(0), Z^(0)) = (R^{-1} V, R^{-1} D), R = diag(R_b).
    Rblk has shape (nblk, bs, bs) (symmetric blocks; the last may be used in its leading part)."""
    Rblk = np.ascontiguousarray(np.asarray(Rblk, dtype=np.float64))
    V, D = _f64(V, "V"), _f64(D, "D")
    nobs = V.shape[1]
    nblk, bs, _ = Rblk.shape
    if nblk != (nobs + bs - 1) // bs:
        raise ValueError("block count does not cover nobs")
    # (nblk, bs, bs) C-order = column-major blocks of a symmetric matrix either way
    U = np.zeros((V.shape[0], nobs))
    Z = np.zeros((D.shape[0], nobs))
    st = _load().oracle_ism_step1_blockdiag(nobs, V.shape[0], D.shape[0], bs, _p(Rblk), _p(V), V.shape[1], _p(D),
                                            D.shape[1], _p(U), nobs, _p(Z), nobs)
    if st != 0:
        raise FloatingPointError(f"block {-st - 1} of R is not positive definite")
    return U, Z


def ism_solve_blockdiag(Rblk, V, D, return_gamma=False):
    """Z = (R + V V^T)^{-1} D for block-diagonal R: the block Step 1, then Step 2 unchanged."""
    U, Z = ism_step1_blockdiag(Rblk, V, D)
    gamma = ism_levels(V, U, Z)
    return (Z, gamma) if return_gamma else Z


# ---------------------------------------------------------------------------
# Lorenz-96 (Sec. 4.2, eq. eqn:Lorenz96)
# ---------------------------------------------------------------------------

def l96_rhs(x, F=8.0):
    x = np.ascontiguousarray(x, dtype=np.float64)
    dx = np.empty_like(x)
    _load().oracle_l96_rhs(x.shape[0], _p(x), F, _p(dx))
    return dx


def l96_rk4(X, F=8.0, dt=0.01, nsteps=1):
    """RK4 on every column of X (shape (nens, ld), nstate = ld); returns a new array."""
    X = np.array(X, dtype=np.float64, copy=True, order="C")
    if X.ndim == 1:
        X = X[None, :]
    st = _load().oracle_l96_rk4(X.shape[1], X.shape[0], _p(X), X.shape[1], F, dt, nsteps)
    if st != 0:
        raise MemoryError("oracle_l96_rk4 failed")
    return X
