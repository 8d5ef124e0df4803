"""Host-side argument checks of the C ABI, run on the CPU: the analysis plan, the
no-allocation solve, and the entry points beside the analysis (inflation, partial
localization, block-diagonal R, pivoted solve, the row-sharded analysis).  Every call here is
rejected by the library's validation before it touches the GPU, so placeholder device
addresses (never dereferenced) stand in for arrays.  Also the workspace sizing of the pivoted
solve and of the row-sharded analysis."""
import ctypes
import math

import pytest

from paper_1302_3876_gb300 import build as libbuild
from paper_1302_3876_gb300 import enkf

FP64, FP32 = enkf.ENKF_FP64, enkf.ENKF_FP32
ARG, SHAPE, WS = enkf.ENKF_ERR_ARG, enkf.ENKF_ERR_SHAPE, enkf.ENKF_ERR_WORKSPACE

# 256-byte aligned placeholder addresses, far apart (no overlap unless a test wants one)
A0, A1, A2, A3, A4, A5 = (ctypes.c_void_p(0x100000000 * (k + 1)) for k in range(6))


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return enkf.load()


def _err(lib):
    return lib.enkf_last_error().decode()


def _loc(lib, nstate=64, nobs=32, nens=8, prec=FP32, stride=2, length=10.0, radius=-1.0, dXB=A0, ldx=None, V=A1,
         ldv=None, Z=A2, ldz=None, XB=A3, ldb=None, XA=A4, lda=None):
    return lib.enkf_localized_update(nstate, nobs, nens, prec, stride, length, radius, dXB, ldx or nstate, V,
                                     ldv or nobs, Z, ldz or nobs, XB, ldb or nstate, XA, lda or nstate, None)


def test_localized_update_rejects_bad_arguments(lib):
    assert _loc(lib, nens=257) == SHAPE and "nens" in _err(lib)
    assert _loc(lib, nens=1) == SHAPE
    assert _loc(lib, prec=7) == ARG
    assert _loc(lib, length=0.0) == ARG
    assert _loc(lib, length=-3.0) == ARG
    assert _loc(lib, radius=math.nan) == ARG
    assert _loc(lib, nobs=40) == SHAPE                      # (nobs - 1) * stride >= nstate
    assert _loc(lib, lda=63) == SHAPE
    assert _loc(lib, ldv=31) == SHAPE
    assert _loc(lib, dXB=None) == ARG
    assert _loc(lib, XA=ctypes.c_void_p(0x100000002)) == ARG   # not aligned to 4 bytes
    assert _loc(lib, XA=A1) == ARG and "overlaps" in _err(lib)  # X_A on top of V
    assert _loc(lib, XA=A2) == ARG                              # X_A on top of Z
    assert _loc(lib, XA=A3, lda=100) == ARG                     # X_B's memory with another ld


def _infl(lib, nstate=64, nobs=16, nens=8, prec=FP32, stride=4, alpha=1.1, XB=A0, dXB=A1, Y=A2, V=A3, D=A4,
          ldb=None):
    return lib.enkf_inflate_prep(nstate, nobs, nens, prec, stride, alpha, XB, ldb or nstate, dXB, nstate, Y, nobs, V,
                                 nobs, D, nobs, None)


def test_inflate_prep_rejects_bad_arguments(lib):
    assert _infl(lib, alpha=-0.5) == ARG
    assert _infl(lib, alpha=math.inf) == ARG
    assert _infl(lib, nens=1) == SHAPE
    assert _infl(lib, prec=3) == ARG
    assert _infl(lib, XB=None) == ARG
    assert _infl(lib, D=None) == ARG                            # Y given without D
    assert _infl(lib, nobs=17) == SHAPE                         # observed rows beyond the state
    assert _infl(lib, ldb=10) == SHAPE


def test_rblock_entry_points_reject_bad_arguments(lib):
    assert lib.enkf_rblock_factor(100, 33, A0, A1, None) == SHAPE
    assert lib.enkf_rblock_factor(100, 0, A0, A1, None) == SHAPE
    assert lib.enkf_rblock_factor(0, 4, A0, A1, None) == SHAPE
    assert lib.enkf_rblock_factor(100, 4, None, A1, None) == ARG
    assert lib.enkf_rblock_factor(100, 4, A0, A0, None) == ARG and "overlap" in _err(lib)
    assert lib.enkf_rblock_factor(100, 4, A0, ctypes.c_void_p(0x200000004), None) == ARG
    assert lib.enkf_rblock_whiten(100, 8, 9, 4, A0, A1, 100, A2, 100, None) == ARG
    assert lib.enkf_rblock_whiten(100, 0, FP32, 4, A0, A1, 100, A2, 100, None) == SHAPE
    assert lib.enkf_rblock_whiten(100, 8, FP32, 4, A0, A1, 99, A2, 100, None) == SHAPE
    assert lib.enkf_rblock_whiten(100, 8, FP64, 4, A0, ctypes.c_void_p(0x200000004), 100, A2, 100, None) == ARG
    assert lib.enkf_rblock_whiten(100, 8, FP32, 64, A0, A1, 100, A2, 100, None) == SHAPE
    assert lib.enkf_rblock_unwhiten(100, 0, FP32, 4, A0, A1, 100, None) == SHAPE
    assert lib.enkf_rblock_unwhiten(100, 8, FP32, 4, None, A1, 100, None) == ARG
    assert lib.enkf_rblock_unwhiten(100, 8, FP32, 4, A0, A1, 50, None) == SHAPE


def _ws(lib, nobs, nens, prec):
    b = ctypes.c_size_t()
    st = lib.enkf_ism_pivot_workspace(nobs, nens, prec, ctypes.byref(b))
    return st, b.value


def test_pivot_workspace_sizes(lib):
    assert _ws(lib, 1000, 257, FP32)[0] == SHAPE
    assert _ws(lib, 0, 8, FP32)[0] == SHAPE
    assert _ws(lib, 1000, 8, 4)[0] == ARG
    st, b1 = _ws(lib, 1000, 32, FP32)
    assert st == 0 and b1 % 256 == 0
    # grows with the rows and the members; FP64 storage of U needs more
    assert _ws(lib, 100000, 32, FP32)[1] > b1
    assert _ws(lib, 1000, 64, FP32)[1] > b1
    assert _ws(lib, 1000, 32, FP64)[1] > b1
    # at least U (nobs x nens, ld padded to 32 rows) and the nens x nens factor arrays
    nobs, nens = 12345, 100
    assert _ws(lib, nobs, nens, FP32)[1] >= 4 * ((nobs + 31) // 32 * 32) * nens + 3 * 8 * nens * nens


def _piv(lib, nobs=1000, nens=8, prec=FP32, Z=A3, M=A4, ws=A5, ws_bytes=None, ldz=None):
    if ws_bytes is None:
        ws_bytes = _ws(lib, nobs, min(nens, 256), FP32 if prec not in (FP32, FP64) else prec)[1]
    st = ctypes.c_int32(0)
    return lib.enkf_ism_solve_pivot(nobs, nens, prec, A0, A1, nobs, A2, nobs, Z, ldz or nobs, M, None, None, ws,
                                    ws_bytes, None, ctypes.byref(st))


def test_pivoted_solve_rejects_bad_arguments(lib):
    assert _piv(lib, nens=257) == SHAPE
    assert _piv(lib, nens=1) == SHAPE                           # M needs nens >= 2
    assert _piv(lib, prec=2) == ARG
    assert _piv(lib, Z=None) == ARG
    assert _piv(lib, ldz=999) == SHAPE
    assert _piv(lib, Z=A1) == ARG and "overlaps" in _err(lib)   # Z on top of V
    assert _piv(lib, ws_bytes=1024) == WS
    assert _piv(lib, ws=ctypes.c_void_p(0x600000010)) == WS     # not 256-byte aligned
    assert _piv(lib, M=ctypes.c_void_p(0x500000002)) == ARG


# ---------------------------------------------------------------------------
# Row-sharded entry points (enkf_rows_*): sizing and the host-side checks.


def _rows_ws(lib, nobs, nens):
    b = ctypes.c_size_t(0)
    st = lib.enkf_rows_workspace(nobs, nens, ctypes.byref(b))
    return st, b.value


def test_rows_workspace_sizes(lib):
    st, small = _rows_ws(lib, 1000, 16)
    assert st == enkf.ENKF_OK and small > 0
    # per-CTA partial dots (2N per 1024-row block) and the Gram's row-slice partials grow with
    # the rows and the members
    assert _rows_ws(lib, 100000, 16)[1] > small
    assert _rows_ws(lib, 1000, 64)[1] > small
    assert _rows_ws(lib, 0, 16)[0] == SHAPE
    assert _rows_ws(lib, 1000, 0)[0] == SHAPE
    assert _rows_ws(lib, 1000, 1025)[0] == SHAPE
    assert lib.enkf_rows_workspace(1000, 16, None) == ARG


def _rows_level(lib, k=0, nobs=1000, nens=16, prec=FP32, r=A0, V=A1, ldv=None, D=A2, ldd=None, U=A3, ldu=None,
                Z=A4, ldz=None, coef=A5, C=A0, gamma=A1, part=A2, ws=A3, wsb=None):
    if wsb is None:
        wsb = _rows_ws(lib, nobs, nens)[1]
    return lib.enkf_rows_level(prec, nobs, nens, k, r, V, ldv or nobs, D, ldd or nobs, U, ldu or nobs, Z,
                               ldz or nobs, coef, C, gamma, part, ws, wsb, None)


def test_rows_level_rejects_bad_arguments(lib):
    assert _rows_level(lib, prec=7) == ARG
    assert _rows_level(lib, nens=0) == SHAPE
    assert _rows_level(lib, k=-2) == ARG
    assert _rows_level(lib, k=16) == ARG and "out of" in _err(lib)
    assert _rows_level(lib, V=None) == ARG
    assert _rows_level(lib, ws=None) == ARG
    assert _rows_level(lib, k=3, part=None) == ARG              # the next level's dots are wanted
    assert _rows_level(lib, k=-1, r=None) == ARG                # Step 1 needs r and D
    assert _rows_level(lib, k=-1, D=None) == ARG
    assert _rows_level(lib, k=0, coef=None) == ARG              # a level needs the reduced dots
    assert _rows_level(lib, k=0, gamma=None) == ARG
    assert _rows_level(lib, ldu=999) == SHAPE
    assert _rows_level(lib, k=-1, ldd=999) == SHAPE
    assert _rows_level(lib, wsb=64) == WS


def test_rows_gram_assemble_xa_reject_bad_arguments(lib):
    wsb = _rows_ws(lib, 1000, 16)[1]
    assert lib.enkf_rows_gram(FP32, 1000, 16, A0, 1000, A1, 999, A2, A3, wsb, None) == SHAPE
    assert lib.enkf_rows_gram(FP32, 1000, 16, A0, 1000, A1, 1000, None, A3, wsb, None) == ARG
    assert lib.enkf_rows_gram(FP32, 1000, 16, A0, 1000, A1, 1000, A2, A3, 8, None) == WS
    assert lib.enkf_rows_assemble(FP32, 1, A0, A1, A2, A3, None) == SHAPE     # M needs two members
    assert lib.enkf_rows_assemble(FP64, 16, A0, None, A2, A3, None) == ARG
    assert lib.enkf_rows_xa(FP32, 0, 16, A0, 1, A1, 1, A2, A3, 1, None) == SHAPE
    assert lib.enkf_rows_xa(FP32, 500, 16, A0, 500, A1, 499, A2, A3, 500, None) == SHAPE
    assert lib.enkf_rows_xa(FP32, 500, 16, A0, 500, None, 500, A2, A3, 500, None) == ARG
    st = ctypes.c_int32(0)
    assert lib.enkf_rows_status(None, None, ctypes.byref(st)) == ARG
    assert lib.enkf_rows_status(A0, None, None) == ARG


# ---------------------------------------------------------------------------
# The analysis plan: sizes, modes, widths and flags rejected before the device is touched.


def test_plan_rejects_bad_sizes_widths_and_flags(lib):
    h, ws = ctypes.c_void_p(), ctypes.c_size_t()

    def plan(nstate=100, nobs=50, nens=8, mode=FP32, panel_b=0, flags=0, out=True, wsp=True):
        return lib.enkf_ism_plan(ctypes.byref(h) if out else None, nstate, nobs, nens, mode, panel_b, flags,
                                 ctypes.byref(ws) if wsp else None)

    assert plan(out=False) == ARG
    assert plan(wsp=False) == ARG
    assert plan(nstate=0) == SHAPE and plan(nobs=0) == SHAPE and plan(nens=0) == SHAPE
    assert plan(nens=1025) == SHAPE
    assert plan(nobs=(1 << 40) + 1) == SHAPE
    assert plan(mode=17) == ARG
    # the single-problem panel width is at most 32 (the tensor-core kernel's shared-memory plan and
    # its one-warp factor); 64 is refused, for every panel mode
    for mode in (enkf.ENKF_PANEL_FP32, enkf.ENKF_PANEL_BF16, enkf.ENKF_PANEL_FP16, enkf.ENKF_PANEL_BF16X3):
        assert plan(mode=mode, panel_b=64) == ARG and "panel_b" in _err(lib)
        assert plan(mode=mode, panel_b=33) == ARG
        assert plan(mode=mode, panel_b=-1) == ARG
    assert plan(flags=0x100) == ARG and "flag" in _err(lib)


def test_noalloc_solve_rejects_bad_arguments(lib):
    def call(nobs=1000, nens=16, prec=FP32, r=A0, V=A1, ldv=None, D=A2, ldd=None, Z=A3, ldz=None):
        return lib.enkf_ism_solve_noalloc(nobs, nens, prec, r, V, ldv or nobs, D, ldd or nobs, Z, ldz or nobs,
                                          None, None)

    assert call(r=None) == ARG and call(Z=None) == ARG
    assert call(prec=enkf.ENKF_PANEL_FP32) == ARG            # the plain FP64 / FP32 solve only
    assert call(nobs=0) == SHAPE and call(nens=1025) == SHAPE
    assert call(ldz=999) == SHAPE and call(ldv=999) == SHAPE
    assert call(prec=FP64, D=ctypes.c_void_p(0x300000004)) == ARG and "aligned" in _err(lib)


# ---------------------------------------------------------------------------
# The forecast (RK4 and the surrogate), the surrogate's training entry points and the batch plan.

UNSUP = enkf.ENKF_ERR_UNSUPPORTED
RK4, SURR = enkf.ENKF_FORECAST_RK4, enkf.ENKF_FORECAST_SURROGATE


def test_forecast_workspace_sizes(lib):
    b = ctypes.c_size_t(7)
    assert lib.enkf_forecast_workspace(4096, 256, RK4, ctypes.byref(b)) == enkf.ENKF_OK and b.value == 0
    assert lib.enkf_forecast_workspace(4096, 256, SURR, ctypes.byref(b)) == enkf.ENKF_OK and b.value > 0
    small = b.value
    assert lib.enkf_forecast_workspace(4096, 512, SURR, ctypes.byref(b)) == enkf.ENKF_OK and b.value > small
    assert lib.enkf_forecast_workspace(4096, 256, 9, ctypes.byref(b)) == UNSUP
    assert lib.enkf_forecast_workspace(0, 256, RK4, ctypes.byref(b)) == SHAPE
    assert lib.enkf_forecast_workspace(4096, 256, RK4, None) == ARG


def test_forecast_rejects_bad_arguments(lib):
    def call(X=A0, ld=None, nstate=40, nens=20, prec=FP64, nsteps=5, method=RK4, weights=None, ws=None, wsb=0):
        return lib.enkf_forecast(X, ld or nstate, nstate, nens, prec, 8.0, 0.01, nsteps, method, weights, ws, wsb,
                                 None)

    assert call(X=None) == ARG
    assert call(prec=enkf.ENKF_PANEL_BF16) == ARG
    assert call(nstate=3) == SHAPE and call(ld=39) == SHAPE and call(nsteps=-1) == SHAPE
    assert call(X=ctypes.c_void_p(0x100000004)) == ARG           # FP64 state not 8-byte aligned
    assert call(nstate=6145) == SHAPE                             # the RK4 state lives in shared memory
    assert call(nsteps=0) == enkf.ENKF_OK                         # nothing to do, nothing launched
    assert call(method=SURR) == UNSUP                             # the surrogate runs on FP32 states
    assert call(method=SURR, prec=FP32) == ARG                    # no weights
    assert call(method=SURR, prec=FP32, weights=A1, ws=A2, wsb=16) == WS
    assert call(method=3, prec=FP32) == UNSUP


def test_surrogate_entry_points_reject_bad_arguments(lib):
    n, pb, wb = ctypes.c_int64(0), ctypes.c_size_t(0), ctypes.c_size_t(0)
    assert lib.enkf_surrogate_sizes(4096, 64, ctypes.byref(n), ctypes.byref(pb), ctypes.byref(wb)) == enkf.ENKF_OK
    assert n.value > 0 and pb.value > 0 and wb.value > 0
    assert lib.enkf_surrogate_sizes(4, 64, None, None, None) == SHAPE
    assert lib.enkf_surrogate_sizes(4096, 0, None, None, None) == SHAPE
    assert lib.enkf_surrogate_pack(None, A1, None) == ARG
    assert lib.enkf_surrogate_pack(A0, ctypes.c_void_p(0x200000010), None) == ARG   # packed not 256-byte aligned

    def train(master=A0, m=A1, v=A2, step=1, packed=A3, X=A4, target=A5, nstate=4096, nbatch=64, ws=A0,
              wsb=None, sq=A1):
        return lib.enkf_surrogate_train_step(master, m, v, step, 1e-3, packed, X, target, nstate, nbatch, ws,
                                             wb.value if wsb is None else wsb, sq, None, None)

    assert train(master=None) == ARG and train(sq=None) == ARG
    assert train(m=None) == ARG                                   # Adam's moments from step 1 on
    assert train(nstate=4) == SHAPE and train(nbatch=0) == SHAPE
    assert train(wsb=16) == WS and train(ws=None) == WS


def test_batch_plan_rejects_bad_problems(lib):
    P = enkf.enkf_ism_problem
    h, ws = ctypes.c_void_p(), ctypes.c_size_t()

    def plan(probs, mode=FP32, flags=0, n=None):
        arr = (P * max(1, len(probs)))(*probs)
        return lib.enkf_ism_batch_plan(ctypes.byref(h), len(probs) if n is None else n, arr, mode, flags,
                                       ctypes.byref(ws))

    def prob(nobs=100, nens=32, ldv=None, ldd=None, Z=0, ldz=None, r=0):
        return P(nobs=nobs, nens=nens, reserved=0, r=r, V=0, D=0, ldv=ldv or nobs, ldd=ldd or nobs, Z=Z,
                 ldz=ldz or nobs, M=-1)

    assert lib.enkf_ism_batch_plan(None, 0, None, FP32, 0, ctypes.byref(ws)) == ARG
    assert plan([prob()], n=-1) == SHAPE
    assert plan([prob()], mode=FP64) == UNSUP                     # the batched kernel is built for FP32
    assert plan([prob()], flags=enkf.ENKF_FLAG_REFINE) == ARG
    assert plan([prob(), prob(nens=30)]) == SHAPE and "problem 1" in _err(lib)   # nens a multiple of 4
    assert plan([prob(nens=132)]) == SHAPE
    assert plan([prob(nobs=0)]) == SHAPE
    assert plan([prob(ldd=99)]) == SHAPE
    assert plan([prob(ldz=99)]) == SHAPE
    assert plan([prob(r=-8)]) == ARG
