"""Shared helpers of the GPU tests (marshalling only; no arithmetic of the method)."""
import numpy as np


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def to_dev(a, dtype, ld=None):
    """numpy (cols, rows) column-major matrix -> CUDA tensor (cols, rows) view of a (cols, ld) buffer."""
    import torch
    a = np.asarray(a)
    cols, rows = a.shape
    ld = rows if ld is None else ld
    buf = np.zeros((cols, ld), dtype=dtype)
    buf[:, :rows] = a
    t = torch.from_numpy(buf).cuda()
    return t[:, :rows]


def vec_dev(v, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(v, dtype=dtype))).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def rounded(a, dtype):
    """The values the device sees for dtype, back in float64 (so the oracle solves the same problem)."""
    return np.ascontiguousarray(np.asarray(a, dtype=dtype).astype(np.float64))
