"""Row-sharded analysis over several ranks (one block of observation rows per rank).

Every rank holds the rows of r, V, D (and so of U and Z) of its block of observations and
a block of state rows of X_B, dX_B and X_A.  Step 1 is local; each level of Step 2 needs
the dots of v_k with every column over all rows (Sec. 3.1, eqs. SM-step-2-h/Z/u), so the
ranks exchange one vector of 2N partial dots per level, and one N x N Gram at the end for
M.  The arithmetic runs in the library's kernels (enkf_rows_*); this module only orders the
calls and hands the partial sums to the caller's collective.
"""
from __future__ import annotations

from . import enkf


def sharded_analysis(r, V, D, dXB, XB, XA, all_reduce, stream=None):
    """Z, M and X_A of the analysis whose observation rows are split over the ranks.

    r (nobs_b,), V and D (nens, nobs_b): this rank's observation rows; dXB, XB, XA
    (nens, nstate_b): this rank's state rows (XA is written).  all_reduce(t) must replace
    the float64 CUDA tensor t by its sum over the ranks (for example torch.distributed's
    all_reduce over NCCL, or a host round trip over gloo).  Returns a dict with this
    rank's Z and U rows, and M, gamma, C (the same on every rank).
    """
    import torch

    nens, nobs = V.shape
    dev = V.device
    ws = torch.empty(enkf.enkf_rows_workspace(nobs, nens), dtype=torch.uint8, device=dev)
    U = torch.empty(nens, nobs, dtype=V.dtype, device=dev)
    Z = torch.empty(nens, nobs, dtype=V.dtype, device=dev)
    part = torch.zeros(2 * nens, dtype=torch.float64, device=dev)
    coef = torch.empty_like(part)
    C = torch.zeros(nens, nens, dtype=torch.float64, device=dev)
    gamma = torch.zeros(nens, dtype=torch.float64, device=dev)
    enkf.enkf_rows_level(-1, r, V, D, U, Z, None, None, None, part, ws, stream)
    for k in range(nens):
        coef.copy_(part)
        all_reduce(coef)
        enkf.enkf_rows_level(k, r, V, D, U, Z, coef, C, gamma, part if k + 1 < nens else None, ws, stream)
    out = {"Z": Z, "U": U, "gamma": gamma, "C": C}
    if nens >= 2:
        Q = torch.zeros(nens, nens, dtype=torch.float64, device=dev)
        enkf.enkf_rows_gram(V, U, Q, ws, stream)
        all_reduce(Q)
        M = torch.empty(nens * nens, dtype=V.dtype, device=dev)
        enkf.enkf_rows_assemble(Q, C, gamma, M, stream)
        if XA is not None:
            enkf.enkf_rows_xa(XB, dXB, M, XA, stream)
        out["M"] = M
    st = enkf.enkf_rows_status(ws, stream)
    if st != enkf.ENKF_OK:
        raise enkf.EnkfError(st, "row-sharded analysis: device check failed")
    return out
