"""Thin Python binding of libenkf_ism (C ABI in include/enkf_ism.h).

Argument marshalling only: every step of the analysis runs in the library's
CUDA kernels.  Functions carry the C names.  Array arguments are CUDA torch
tensors laid out column-major: a matrix with ``rows`` rows and ``cols`` columns
is a tensor of shape ``(cols, rows)`` (or a ``[:, :rows]`` view of a padded
``(cols, ld)`` tensor) whose leading dimension is ``tensor.stride(0)``.

There is no fallback: if the shared library is missing or fails to load, every
call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

ENKF_OK = 0
ENKF_ERR_ARG = 1
ENKF_ERR_SHAPE = 2
ENKF_ERR_CUDA = 3
ENKF_ERR_NUMERIC = 4
ENKF_ERR_TIMEOUT = 5
ENKF_ERR_UNSUPPORTED = 6
ENKF_ERR_WORKSPACE = 7

ENKF_FP64 = 0
ENKF_FP32 = 1
ENKF_PANEL_BF16 = 2
ENKF_PANEL_FP16 = 3
ENKF_PANEL_FP32 = 4
ENKF_PANEL_BF16X3 = 5

ENKF_FLAG_REFINE = 0x1
ENKF_FLAG_NO_CHECKS = 0x2
ENKF_FLAG_TEST_TIMEOUT = 0x4

ENKF_FORECAST_RK4 = 0
ENKF_FORECAST_SURROGATE = 1

ENKF_PROFILE_PHASES = 8
PROFILE_PHASE_NAMES = ("obs_prep", "ism_solve", "gram_upper", "assemble_M", "xa_update", "refine", "panel_kernel",
                       "correction_kernel")


class EnkfError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{status_name(status)}: {message}")
        self.status = status


class enkf_ism_problem(ctypes.Structure):
    _fields_ = [("nobs", ctypes.c_int64), ("nens", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("r", ctypes.c_int64), ("V", ctypes.c_int64), ("D", ctypes.c_int64),
                ("ldv", ctypes.c_int64), ("ldd", ctypes.c_int64), ("Z", ctypes.c_int64), ("ldz", ctypes.c_int64),
                ("M", ctypes.c_int64)]


class enkf_ism_info(ctypes.Structure):
    _fields_ = [("gamma_min", ctypes.c_double), ("gamma_max", ctypes.c_double), ("panel_b", ctypes.c_int32),
                ("grid_ctas", ctypes.c_int32), ("status", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("refine_resid", ctypes.c_double)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = False):
    """Load libenkf_ism.so (raises if it is missing and building is not requested)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB_PATH
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"libenkf_ism.so not built ({path}); run paper_1302_3876_gb300.build.build()")
            _build.build()
        lib = ctypes.CDLL(path)
        i64, i32, u32, vp, sz = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_size_t
        lib.enkf_ism_plan.argtypes = [ctypes.POINTER(vp), i64, i64, i32, i32, i32, u32, ctypes.POINTER(sz)]
        lib.enkf_ism_plan.restype = ctypes.c_int
        lib.enkf_ism_plan_destroy.argtypes = [vp]
        lib.enkf_ism_plan_destroy.restype = None
        lib.enkf_obs_prep.argtypes = [vp, i32, i32, vp, i64, vp, i64, vp, i64, vp, i64, vp, i64, vp]
        lib.enkf_obs_prep.restype = ctypes.c_int
        lib.enkf_ism_analysis.argtypes = [vp, vp, vp, i64, vp, i64, vp, i64, vp, i64, vp, i64, vp, i64, vp, vp, sz,
                                          vp, ctypes.POINTER(enkf_ism_info)]
        lib.enkf_ism_analysis.restype = ctypes.c_int
        lib.enkf_ism_gamma.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_double)]
        lib.enkf_ism_gamma.restype = ctypes.c_int
        lib.enkf_ism_profile.argtypes = [vp, i32]
        lib.enkf_ism_profile.restype = ctypes.c_int
        lib.enkf_ism_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i32)]
        lib.enkf_ism_profile_read.restype = ctypes.c_int
        dbl = ctypes.c_double
        lib.enkf_forecast.argtypes = [vp, i64, i64, i32, i32, dbl, dbl, i32, i32, vp, vp, sz, vp]
        lib.enkf_forecast.restype = ctypes.c_int
        lib.enkf_forecast_workspace.argtypes = [i64, i32, i32, ctypes.POINTER(sz)]
        lib.enkf_forecast_workspace.restype = ctypes.c_int
        lib.enkf_ism_solve_noalloc.argtypes = [i64, i32, i32, vp, vp, i64, vp, i64, vp, i64, vp,
                                               ctypes.POINTER(i32)]
        lib.enkf_ism_solve_noalloc.restype = ctypes.c_int
        lib.enkf_inflate_prep.argtypes = [i64, i64, i32, i32, i32, dbl, vp, i64, vp, i64, vp, i64, vp, i64, vp, i64,
                                          vp]
        lib.enkf_inflate_prep.restype = ctypes.c_int
        lib.enkf_localized_update.argtypes = [i64, i64, i32, i32, i32, dbl, dbl, vp, i64, vp, i64, vp, i64, vp, i64,
                                              vp, i64, vp]
        lib.enkf_localized_update.restype = ctypes.c_int
        lib.enkf_rblock_factor.argtypes = [i64, i32, vp, vp, vp]
        lib.enkf_rblock_factor.restype = ctypes.c_int
        lib.enkf_rblock_whiten.argtypes = [i64, i32, i32, i32, vp, vp, i64, vp, i64, vp]
        lib.enkf_rblock_whiten.restype = ctypes.c_int
        lib.enkf_rblock_unwhiten.argtypes = [i64, i32, i32, i32, vp, vp, i64, vp]
        lib.enkf_rblock_unwhiten.restype = ctypes.c_int
        lib.enkf_rows_workspace.argtypes = [i64, i32, ctypes.POINTER(sz)]
        lib.enkf_rows_workspace.restype = ctypes.c_int
        lib.enkf_rows_level.argtypes = [i32, i64, i32, i32, vp, vp, i64, vp, i64, vp, i64, vp, i64, vp, vp, vp, vp,
                                        vp, sz, vp]
        lib.enkf_rows_level.restype = ctypes.c_int
        lib.enkf_rows_gram.argtypes = [i32, i64, i32, vp, i64, vp, i64, vp, vp, sz, vp]
        lib.enkf_rows_gram.restype = ctypes.c_int
        lib.enkf_rows_assemble.argtypes = [i32, i32, vp, vp, vp, vp, vp]
        lib.enkf_rows_assemble.restype = ctypes.c_int
        lib.enkf_rows_xa.argtypes = [i32, i64, i32, vp, i64, vp, i64, vp, vp, i64, vp]
        lib.enkf_rows_xa.restype = ctypes.c_int
        lib.enkf_rows_status.argtypes = [vp, vp, ctypes.POINTER(i32)]
        lib.enkf_rows_status.restype = ctypes.c_int
        lib.enkf_ism_pivot_workspace.argtypes = [i64, i32, i32, ctypes.POINTER(sz)]
        lib.enkf_ism_pivot_workspace.restype = ctypes.c_int
        lib.enkf_ism_solve_pivot.argtypes = [i64, i32, i32, vp, vp, i64, vp, i64, vp, i64, vp, vp, vp, vp, sz, vp,
                                             ctypes.POINTER(i32)]
        lib.enkf_ism_solve_pivot.restype = ctypes.c_int
        lib.enkf_ism_batch_plan.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(enkf_ism_problem), i32, u32,
                                            ctypes.POINTER(sz)]
        lib.enkf_ism_batch_plan.restype = ctypes.c_int
        lib.enkf_ism_batch_plan_destroy.argtypes = [vp]
        lib.enkf_ism_batch_plan_destroy.restype = None
        lib.enkf_ism_batch_autotune.argtypes = [vp, vp, vp, vp, sz, vp, ctypes.c_char_p, ctypes.POINTER(i32)]
        lib.enkf_ism_batch_autotune.restype = ctypes.c_int
        lib.enkf_ism_batch.argtypes = [vp, vp, vp, vp, sz, vp, ctypes.POINTER(i32)]
        lib.enkf_ism_batch.restype = ctypes.c_int
        lib.enkf_surrogate_sizes.argtypes = [i64, i32, ctypes.POINTER(i64), ctypes.POINTER(sz), ctypes.POINTER(sz)]
        lib.enkf_surrogate_sizes.restype = ctypes.c_int
        lib.enkf_surrogate_pack.argtypes = [vp, vp, vp]
        lib.enkf_surrogate_pack.restype = ctypes.c_int
        lib.enkf_surrogate_train_step.argtypes = [vp, vp, vp, i32, ctypes.c_float, vp, vp, vp, i64, i32, vp, sz, vp,
                                                  vp, vp]
        lib.enkf_surrogate_train_step.restype = ctypes.c_int
        lib.enkf_fma_peak_launch.argtypes = [i32, i32, i32, vp, vp, ctypes.POINTER(dbl)]
        lib.enkf_fma_peak_launch.restype = ctypes.c_int
        lib.enkf_status_string.argtypes = [ctypes.c_int]
        lib.enkf_status_string.restype = ctypes.c_char_p
        lib.enkf_last_error.argtypes = []
        lib.enkf_last_error.restype = ctypes.c_char_p
        _lib = lib
        return lib


def status_name(status: int) -> str:
    try:
        return load().enkf_status_string(status).decode()
    except Exception:  # noqa: BLE001 - used while formatting another error
        return f"status {status}"


def _check(status: int):
    if status != ENKF_OK:
        raise EnkfError(status, load().enkf_last_error().decode())


def _mat(t, name):
    """(pointer, ld) of a column-major matrix tensor of shape (cols, rows)."""
    if t is None:
        return None, 0
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dim() == 1:
        return ctypes.c_void_p(t.data_ptr()), max(t.shape[0], 1)
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError(f"{name} must be a 2-D tensor with unit row stride (shape (cols, rows))")
    return ctypes.c_void_p(t.data_ptr()), int(t.stride(0)) if t.shape[0] > 1 else int(max(t.stride(0), t.shape[1]))


def _ptr(t, name):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def enkf_ism_plan(nstate: int, nobs: int, nens: int, mode: int, panel_b: int = 0, flags: int = 0):
    """Returns (plan handle, workspace bytes)."""
    lib = load()
    h = ctypes.c_void_p()
    ws = ctypes.c_size_t()
    _check(lib.enkf_ism_plan(ctypes.byref(h), nstate, nobs, nens, mode, panel_b, flags, ctypes.byref(ws)))
    return h, ws.value


def enkf_ism_plan_destroy(plan) -> None:
    load().enkf_ism_plan_destroy(plan)


def enkf_obs_prep(plan, obs_stride: int, center: int, XB, dXB, V, Y=None, D=None, stream=None) -> None:
    pXB, ldb = _mat(XB, "XB")
    pdX, ldx = _mat(dXB, "dXB")
    pY, ldy = _mat(Y, "Y")
    pV, ldv = _mat(V, "V")
    pD, ldd = _mat(D, "D")
    _check(load().enkf_obs_prep(plan, obs_stride, center, pXB, ldb, pdX, ldx, pY, ldy, pV, ldv, pD, ldd,
                                _stream(stream)))


def enkf_ism_analysis(plan, r, V, D, workspace, dXB=None, XB=None, XA=None, Z=None, M=None, stream=None,
                      info: bool = False):
    """One analysis.  Returns an enkf_ism_info when ``info`` (the call then synchronises)."""
    pV, ldv = _mat(V, "V")
    pD, ldd = _mat(D, "D")
    pdX, ldx = _mat(dXB, "dXB")
    pXB, ldb = _mat(XB, "XB")
    pXA, lda = _mat(XA, "XA")
    pZ, ldz = _mat(Z, "Z")
    inf = enkf_ism_info() if info else None
    ws_bytes = workspace.numel() * workspace.element_size()
    st = load().enkf_ism_analysis(plan, _ptr(r, "r"), pV, ldv, pD, ldd, pdX, ldx, pXB, ldb, pXA, lda, pZ, ldz,
                                  _ptr(M, "M"), _ptr(workspace, "workspace"), ws_bytes, _stream(stream),
                                  ctypes.byref(inf) if inf is not None else None)
    _check(st)
    return inf


def enkf_forecast_workspace(nstate: int, nens: int, method: int) -> int:
    b = ctypes.c_size_t()
    _check(load().enkf_forecast_workspace(nstate, nens, method, ctypes.byref(b)))
    return b.value


def enkf_forecast(X, F: float, dt: float, nsteps: int, method: int = ENKF_FORECAST_RK4, weights=None,
                  workspace=None, stream=None) -> None:
    """Forecast in place; X is a CUDA tensor (nens, nstate) float64 or float32."""
    import torch
    pX, ld = _mat(X, "X")
    nens, nstate = X.shape
    precision = ENKF_FP64 if X.dtype == torch.float64 else ENKF_FP32
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check(load().enkf_forecast(pX, ld, nstate, nens, precision, F, dt, nsteps, method, _ptr(weights, "weights"),
                                _ptr(workspace, "workspace"), ws_bytes, _stream(stream)))


def enkf_ism_solve_noalloc(r, V, D, Z, stream=None, sync: bool = True) -> int:
    """Solve Z = (R + V V^T)^{-1} D without a workspace (scratch in the library's static
    device array).  For callers that cannot allocate device memory.  Returns the
    device status word when ``sync`` (the call then synchronises), else 0."""
    import torch
    pV, ldv = _mat(V, "V")
    pD, ldd = _mat(D, "D")
    pZ, ldz = _mat(Z, "Z")
    nens, nobs = V.shape
    precision = ENKF_FP64 if V.dtype == torch.float64 else ENKF_FP32
    st = ctypes.c_int32(0)
    _check(load().enkf_ism_solve_noalloc(nobs, nens, precision, _ptr(r, "r"), pV, ldv, pD, ldd, pZ, ldz,
                                         _stream(stream), ctypes.byref(st) if sync else None))
    return st.value


def _precision(t):
    import torch
    return ENKF_FP64 if t.dtype == torch.float64 else ENKF_FP32


def enkf_inflate_prep(obs_stride: int, alpha: float, XB, V, dXB=None, Y=None, D=None, stream=None) -> None:
    """Inflation x <- xbar + alpha (x - xbar) of XB in place, fused with the centering prep
    (dXB, V, and D when Y is given).  Sizes come from the tensors: XB (nens, nstate), V (nens, nobs)."""
    pXB, ldb = _mat(XB, "XB")
    pdX, ldx = _mat(dXB, "dXB")
    pY, ldy = _mat(Y, "Y")
    pV, ldv = _mat(V, "V")
    pD, ldd = _mat(D, "D")
    nens, nstate = XB.shape
    nobs = V.shape[1]
    _check(load().enkf_inflate_prep(nstate, nobs, nens, _precision(XB), obs_stride, float(alpha), pXB, ldb, pdX,
                                    ldx, pY, ldy, pV, ldv, pD, ldd, _stream(stream)))


def enkf_localized_update(obs_stride: int, length: float, radius, dXB, V, Z, XB, XA, stream=None) -> None:
    """X_A = X_B + (Delta o (S V^T)) Z (partial localization); radius None = no cut-off.
    dXB, XB, XA: (nens, nstate); V, Z: (nens, nobs).  XA may be XB."""
    pdX, ldx = _mat(dXB, "dXB")
    pV, ldv = _mat(V, "V")
    pZ, ldz = _mat(Z, "Z")
    pXB, ldb = _mat(XB, "XB")
    pXA, lda = _mat(XA, "XA")
    nens, nstate = dXB.shape
    nobs = V.shape[1]
    rad = -1.0 if radius is None else float(radius)
    _check(load().enkf_localized_update(nstate, nobs, nens, _precision(dXB), obs_stride, float(length), rad, pdX, ldx,
                                        pV, ldv, pZ, ldz, pXB, ldb, pXA, lda, _stream(stream)))


def enkf_rblock_factor(nobs: int, bs: int, Rblk, Lblk, stream=None) -> None:
    """Lblk <- block Cholesky factors of Rblk (CUDA float64 tensors of nblk * bs * bs entries)."""
    _check(load().enkf_rblock_factor(nobs, bs, _ptr(Rblk, "Rblk"), _ptr(Lblk, "Lblk"), _stream(stream)))


def enkf_rblock_whiten(bs: int, Lblk, V, D=None, stream=None) -> None:
    """V <- L^{-1} V, D <- L^{-1} D in place (V, D: (nens, nobs))."""
    pV, ldv = _mat(V, "V")
    pD, ldd = _mat(D, "D")
    nens, nobs = V.shape
    _check(load().enkf_rblock_whiten(nobs, nens, _precision(V), bs, _ptr(Lblk, "Lblk"), pV, ldv, pD, ldd,
                                     _stream(stream)))


def enkf_rblock_unwhiten(bs: int, Lblk, Z, stream=None) -> None:
    """Z <- L^{-T} Z in place (Z: (ncols, nobs))."""
    pZ, ldz = _mat(Z, "Z")
    ncols, nobs = Z.shape
    _check(load().enkf_rblock_unwhiten(nobs, ncols, _precision(Z), bs, _ptr(Lblk, "Lblk"), pZ, ldz, _stream(stream)))


def enkf_rows_workspace(nobs: int, nens: int) -> int:
    b = ctypes.c_size_t()
    _check(load().enkf_rows_workspace(nobs, nens, ctypes.byref(b)))
    return b.value


def enkf_rows_level(k: int, r, V, D, U, Z, coef, C, gamma, part, workspace, stream=None) -> None:
    """Level k of Step 2 on a block of rows (k = -1: Step 1); V, D, U, Z: (nens, nobs) tensors,
    r: (nobs,), coef / part: (2 nens,) float64, C: (nens, nens) float64, gamma: (nens,) float64."""
    pV, ldv = _mat(V, "V")
    pD, ldd = _mat(D, "D")
    pU, ldu = _mat(U, "U")
    pZ, ldz = _mat(Z, "Z")
    nens, nobs = V.shape[0], V.shape[1]
    _check(load().enkf_rows_level(_precision(V), nobs, nens, k, _ptr(r, "r"), pV, ldv, pD, ldd, pU, ldu, pZ, ldz,
                                  _ptr(coef, "coef"), _ptr(C, "C"), _ptr(gamma, "gamma"), _ptr(part, "part"),
                                  _ptr(workspace, "workspace"), workspace.numel() * workspace.element_size(),
                                  _stream(stream)))


def enkf_rows_gram(V, U, Q, workspace, stream=None) -> None:
    """The block's partial Q[k][m] = v_k^T u_m (k < m) into Q ((nens, nens) float64, row-major [k][m])."""
    pV, ldv = _mat(V, "V")
    pU, ldu = _mat(U, "U")
    nens, nobs = V.shape[0], V.shape[1]
    _check(load().enkf_rows_gram(_precision(V), nobs, nens, pV, ldv, pU, ldu, _ptr(Q, "Q"), _ptr(workspace, "workspace"),
                                 workspace.numel() * workspace.element_size(), _stream(stream)))


def enkf_rows_assemble(Q, C, gamma, M, stream=None) -> None:
    """M = (I - triu(Q,1)) diag(1/gamma) C / sqrt(N - 1); M: (nens * nens,) of the storage precision."""
    nens = gamma.shape[0]
    _check(load().enkf_rows_assemble(_precision(M), nens, _ptr(Q, "Q"), _ptr(C, "C"), _ptr(gamma, "gamma"),
                                     _ptr(M, "M"), _stream(stream)))


def enkf_rows_xa(XB, dXB, M, XA, stream=None) -> None:
    """X_A = X_B + dX_B M on a block of state rows (XB, dXB, XA: (nens, nstate_block))."""
    pXB, ldb = _mat(XB, "XB")
    pdX, ldx = _mat(dXB, "dXB")
    pXA, lda = _mat(XA, "XA")
    nens, nstate = dXB.shape[0], dXB.shape[1]
    _check(load().enkf_rows_xa(_precision(dXB), nstate, nens, pXB, ldb, pdX, ldx, _ptr(M, "M"), pXA, lda,
                               _stream(stream)))


def enkf_rows_status(workspace, stream=None) -> int:
    st = ctypes.c_int32(0)
    _check(load().enkf_rows_status(_ptr(workspace, "workspace"), _stream(stream), ctypes.byref(st)))
    return st.value


def enkf_ism_pivot_workspace(nobs: int, nens: int, precision: int) -> int:
    b = ctypes.c_size_t()
    _check(load().enkf_ism_pivot_workspace(nobs, nens, precision, ctypes.byref(b)))
    return b.value


def enkf_ism_solve_pivot(r, V, D, Z, workspace, M=None, perm=None, gamma=None, stream=None, sync: bool = True) -> int:
    """Solve with the pivoting of Sec. 3.4.  V, D, Z: (nens, nobs); M: nens*nens (nullable); perm: int32 (nens);
    gamma: float64 (nens).  Returns the device status word when ``sync``."""
    pV, ldv = _mat(V, "V")
    pD, ldd = _mat(D, "D")
    pZ, ldz = _mat(Z, "Z")
    nens, nobs = V.shape
    st = ctypes.c_int32(0)
    _check(load().enkf_ism_solve_pivot(nobs, nens, _precision(V), _ptr(r, "r"), pV, ldv, pD, ldd, pZ, ldz,
                                       _ptr(M, "M"), _ptr(perm, "perm"), _ptr(gamma, "gamma"),
                                       _ptr(workspace, "workspace"), workspace.numel() * workspace.element_size(),
                                       _stream(stream), ctypes.byref(st) if sync else None))
    return st.value


def enkf_ism_batch_plan(problems, mode: int = ENKF_FP32, flags: int = 0):
    """problems: sequence of dicts with keys nobs, nens, r, V, D, ldv, ldd, Z, ldz, M (float offsets).
    Returns (batch plan handle, workspace bytes)."""
    arr = (enkf_ism_problem * max(len(problems), 1))()
    for i, p in enumerate(problems):
        arr[i] = enkf_ism_problem(nobs=p["nobs"], nens=p["nens"], reserved=0, r=p["r"], V=p["V"], D=p["D"],
                                  ldv=p["ldv"], ldd=p["ldd"], Z=p.get("Z", -1), ldz=p.get("ldz", p["nobs"]),
                                  M=p.get("M", -1))
    h = ctypes.c_void_p()
    ws = ctypes.c_size_t()
    _check(load().enkf_ism_batch_plan(ctypes.byref(h), len(problems), arr, mode, flags, ctypes.byref(ws)))
    return h, ws.value


def enkf_ism_batch_plan_destroy(plan) -> None:
    load().enkf_ism_batch_plan_destroy(plan)


def enkf_ism_batch_autotune(plan, base_in, base_out, workspace, stream=None, cache_path=None):
    """Returns the 16 per-class panel widths chosen."""
    w = (ctypes.c_int32 * 16)()
    _check(load().enkf_ism_batch_autotune(plan, _ptr(base_in, "base_in"), _ptr(base_out, "base_out"),
                                          _ptr(workspace, "workspace"), workspace.numel() * workspace.element_size(),
                                          _stream(stream), cache_path.encode() if cache_path else None, w))
    return list(w)


def enkf_ism_batch(plan, base_in, base_out, workspace, stream=None, sync: bool = False) -> int:
    st = ctypes.c_int32(0)
    _check(load().enkf_ism_batch(plan, _ptr(base_in, "base_in"), _ptr(base_out, "base_out"),
                                 _ptr(workspace, "workspace"), workspace.numel() * workspace.element_size(),
                                 _stream(stream), ctypes.byref(st) if sync else None))
    return st.value


def enkf_surrogate_sizes(nstate: int, nbatch: int):
    """(number of parameters, packed bytes, training workspace bytes)."""
    n = ctypes.c_int64()
    pb = ctypes.c_size_t()
    tw = ctypes.c_size_t()
    _check(load().enkf_surrogate_sizes(nstate, nbatch, ctypes.byref(n), ctypes.byref(pb), ctypes.byref(tw)))
    return n.value, pb.value, tw.value


def enkf_surrogate_pack(master, packed, stream=None) -> None:
    _check(load().enkf_surrogate_pack(_ptr(master, "master"), _ptr(packed, "packed"), _stream(stream)))


def enkf_surrogate_train_step(master, adam_m, adam_v, step, lr, packed, X, target, workspace, sq_err, grad=None,
                              stream=None) -> None:
    """X, target: CUDA float32 (nbatch, nstate) contiguous."""
    nbatch, nstate = X.shape
    _check(load().enkf_surrogate_train_step(_ptr(master, "master"), _ptr(adam_m, "adam_m"), _ptr(adam_v, "adam_v"),
                                            step, lr, _ptr(packed, "packed"), _ptr(X, "X"), _ptr(target, "target"),
                                            nstate, nbatch, _ptr(workspace, "workspace"),
                                            workspace.numel() * workspace.element_size(), _ptr(sq_err, "sq_err"),
                                            _ptr(grad, "grad"), _stream(stream)))


def enkf_ism_gamma(plan, workspace, nens: int):
    """The level denominators gamma_k of the plan's last analysis (list of nens floats)."""
    g = (ctypes.c_double * nens)()
    _check(load().enkf_ism_gamma(plan, _ptr(workspace, "workspace"), g))
    return list(g)


def enkf_ism_profile(plan, enable: bool) -> None:
    _check(load().enkf_ism_profile(plan, 1 if enable else 0))


def enkf_ism_profile_read(plan):
    """{phase name: (total ms, launches)} of the phases recorded since the last read."""
    ms = (ctypes.c_double * ENKF_PROFILE_PHASES)()
    cnt = (ctypes.c_int32 * ENKF_PROFILE_PHASES)()
    _check(load().enkf_ism_profile_read(plan, ms, cnt))
    return {PROFILE_PHASE_NAMES[i]: (ms[i], cnt[i]) for i in range(ENKF_PROFILE_PHASES) if cnt[i]}


def enkf_fma_peak_launch(precision: int, iters: int, ctas_per_sm: int, sink, stream=None) -> float:
    """Launch the CUDA-core FMA microbenchmark; returns the launch's flop count (time it with events)."""
    fl = ctypes.c_double(0.0)
    _check(load().enkf_fma_peak_launch(precision, iters, ctas_per_sm, _ptr(sink, "sink"), _stream(stream),
                                       ctypes.byref(fl)))
    return fl.value


def enkf_status_string(status: int) -> str:
    return load().enkf_status_string(status).decode()


def enkf_last_error() -> str:
    return load().enkf_last_error().decode()


class Plan:
    """Owns a plan handle and its device workspace (allocated by torch)."""

    def __init__(self, nstate, nobs, nens, mode, panel_b=0, flags=0, device=None):
        import torch
        self.handle, self.workspace_bytes = enkf_ism_plan(nstate, nobs, nens, mode, panel_b, flags)
        dev = torch.device("cuda") if device is None else torch.device(device)
        # 256-byte alignment: torch's caching allocator returns 512-byte aligned blocks
        self.workspace = torch.empty(max(self.workspace_bytes, 256), dtype=torch.uint8, device=dev)
        self.nstate, self.nobs, self.nens, self.mode = nstate, nobs, nens, mode

    def close(self):
        if self.handle is not None:
            enkf_ism_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def analysis(self, r, V, D, **kw):
        return enkf_ism_analysis(self.handle, r, V, D, self.workspace, **kw)

    def gamma(self):
        return enkf_ism_gamma(self.handle, self.workspace, self.nens)

    def obs_prep(self, obs_stride, center, XB, dXB, V, Y=None, D=None, stream=None):
        enkf_obs_prep(self.handle, obs_stride, center, XB, dXB, V, Y, D, stream)
