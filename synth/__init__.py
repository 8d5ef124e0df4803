"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module draws random numbers and lays them out; it holds none of the
filter's arithmetic (no observation operator, no scaling by 1/sqrt(Nens-1), no
solve).  The draws come from the counter-based SplitMix64 generator in
``prng.c`` (compiled on first use with the host C compiler), so every array is a
pure function of (seed, stream, index) and is identical on every machine and
thread count.

Workload recipes (seed = 13023876 + workload index):

* ``lorenz_small`` -- Lorenz-96 with Nstate=40, Nens=20, every 2nd variable
  observed (Nobs=20), R = 0.01 I: initial truth F + N(0,1) (to be spun up by the
  caller), ensemble noise N(0, 0.1^2), observation noise and perturbations
  N(0, 0.01).
* ``large_single`` -- Nstate x Nens deviations dX_B[i,e] = s_i N(0,1) with
  s_i ~ U[0.5, 2]; variances r_j ~ U[0.5, 1.5]; innovations D ~ N(0,1).
  Nstate = 2^21, Nobs = 2^19, Nens = 128 at full size.
* ``panel_single`` -- the same distributions at Nstate = 2^22, Nobs = 2^20,
  Nens = 256.
* ``batch_local`` -- independent problems with Nobs_i = round(exp(U[ln 16,
  ln 4096])), Nens_i uniform over {32, 64, 96, 128}, V_i[j,e] ~ N(0, s_j^2/(Nens_i-1))
  with s_j ~ U[0.5, 2], r ~ U[0.5, 1.5], D ~ N(0,1).
* ``lorenz_cycle`` -- Lorenz-96 with Nstate = 4096, Nens = 256, every 2nd
  variable observed, R = 0.25 I.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

SEED_BASE = 13023876
WORKLOADS = ("lorenz_small", "large_single", "panel_single", "batch_local", "lorenz_cycle", "next_rows")

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_DIR = os.path.join(_HERE, "_lib")
_LIB_PATH = os.path.join(_LIB_DIR, "libsynth.so")
_lib = None
_lock = threading.Lock()


def seed_for(workload: str) -> int:
    return SEED_BASE + WORKLOADS.index(workload)


def build(force: bool = False) -> str:
    """Compile prng.c into synth/_lib/libsynth.so (no-op when up to date)."""
    src = os.path.join(_HERE, "prng.c")
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
            u64, i64, dbl, vp = ctypes.c_uint64, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
            lib.synth_u64.argtypes = [u64, u64, u64, i64, vp]
            lib.synth_uniform.argtypes = [u64, u64, u64, i64, dbl, dbl, vp]
            lib.synth_normal_matrix.argtypes = [u64, u64, i64, i64, i64, dbl, dbl, vp, vp]
            lib.synth_normal_matrix_f32.argtypes = [u64, u64, i64, i64, i64, dbl, dbl, vp, vp]
            for f in (lib.synth_u64, lib.synth_uniform, lib.synth_normal_matrix, lib.synth_normal_matrix_f32):
                f.restype = None
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def uniform(seed: int, stream: int, n: int, lo: float, hi: float, offset: int = 0) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    _load().synth_uniform(seed, stream, offset, n, lo, hi, _ptr(out))
    return out


def u64(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    out = np.empty(n, dtype=np.uint64)
    _load().synth_u64(seed, stream, offset, n, _ptr(out))
    return out


def normal_matrix(seed: int, stream: int, rows: int, cols: int, ld: int | None = None,
                  mean: float = 0.0, std: float = 1.0, row_scale: np.ndarray | None = None,
                  dtype=np.float64) -> np.ndarray:
    """Column-major rows x cols normal matrix, returned as an (cols, ld) C array.

    The returned array ``a`` has shape (cols, ld); column c of the matrix is
    ``a[c, :rows]``.  Padding rows are zero.
    """
    ld = rows if ld is None else ld
    if ld < rows:
        raise ValueError("ld < rows")
    out = np.zeros((cols, ld), dtype=dtype)
    rs = None
    if row_scale is not None:
        rs = np.ascontiguousarray(row_scale, dtype=np.float64)
        if rs.shape[0] < rows:
            raise ValueError("row_scale too short")
    lib = _load()
    fn = lib.synth_normal_matrix if dtype == np.float64 else lib.synth_normal_matrix_f32
    if dtype not in (np.float64, np.float32):
        raise ValueError("dtype must be float64 or float32")
    fn(seed, stream, rows, cols, ld, mean, std, _ptr(rs), _ptr(out))
    return out


def pad_ld(rows: int, multiple: int = 32) -> int:
    """Leading dimension padded to a multiple of 32 elements (256-byte columns in FP64)."""
    return max(multiple, (rows + multiple - 1) // multiple * multiple)


# ---------------------------------------------------------------------------
# Workload recipes
# ---------------------------------------------------------------------------

def large_single(nstate: int = 1 << 21, nobs: int = 1 << 19, nens: int = 128, seed: int | None = None,
                 dtype=np.float64, ld_state: int | None = None, ld_obs: int | None = None):
    """Deviations, variances and innovations of the large single analysis.

    Returns a dict with ``dXB`` (shape (nens, ld_state)), ``r`` (nobs,),
    ``D`` (shape (nens, ld_obs)) and the per-variable spread ``s``.  The
    background is taken equal to the deviations (zero background mean).
    """
    seed = seed_for("large_single") if seed is None else seed
    s = uniform(seed, 1, nstate, 0.5, 2.0)
    dXB = normal_matrix(seed, 2, nstate, nens, ld_state, row_scale=s, dtype=dtype)
    r = uniform(seed, 3, nobs, 0.5, 1.5).astype(dtype)
    D = normal_matrix(seed, 4, nobs, nens, ld_obs, dtype=dtype)
    return {"s": s, "dXB": dXB, "r": r, "D": D, "nstate": nstate, "nobs": nobs, "nens": nens}


def panel_single(nstate: int = 1 << 22, nobs: int = 1 << 20, nens: int = 256, seed: int | None = None,
                 dtype=np.float32, ld_state: int | None = None, ld_obs: int | None = None):
    """Same distributions as ``large_single`` at the panel workload's sizes."""
    seed = seed_for("panel_single") if seed is None else seed
    return large_single(nstate, nobs, nens, seed, dtype, ld_state, ld_obs)


def lorenz_small_draws(nstate: int = 40, nens: int = 20, obs_stride: int = 2, r: float = 0.01,
                       forcing: float = 8.0, seed: int | None = None):
    """Raw draws of the small Lorenz-96 analysis (the truth still has to be spun up)."""
    seed = seed_for("lorenz_small") if seed is None else seed
    nobs = (nstate + obs_stride - 1) // obs_stride
    return {
        "truth0": normal_matrix(seed, 1, nstate, 1, mean=forcing)[0],
        "ens_noise": normal_matrix(seed, 2, nstate, nens, std=0.1),
        "obs_noise": normal_matrix(seed, 3, nobs, 1, std=float(np.sqrt(r)))[0],
        "pert": normal_matrix(seed, 4, nobs, nens, std=float(np.sqrt(r))),
        "nstate": nstate, "nobs": nobs, "nens": nens, "obs_stride": obs_stride, "r": r, "F": forcing,
    }


def lorenz_cycle_draws(cycle: int, nstate: int = 4096, nens: int = 256, obs_stride: int = 2,
                       r: float = 0.25, seed: int | None = None):
    """Per-cycle observation noise and perturbations of the Lorenz-96 cycling workload."""
    seed = seed_for("lorenz_cycle") if seed is None else seed
    nobs = (nstate + obs_stride - 1) // obs_stride
    return {
        "obs_noise": normal_matrix(seed, 1000 + 2 * cycle, nobs, 1, std=float(np.sqrt(r)))[0],
        "pert": normal_matrix(seed, 1001 + 2 * cycle, nobs, nens, std=float(np.sqrt(r))),
    }


def lorenz_cycle_init(nstate: int = 4096, nens: int = 256, forcing: float = 8.0, seed: int | None = None):
    """Initial truth F + N(0,1) and initial ensemble noise N(0,1) of the cycling workload."""
    seed = seed_for("lorenz_cycle") if seed is None else seed
    return {
        "truth0": normal_matrix(seed, 1, nstate, 1, mean=forcing)[0],
        "ens_noise": normal_matrix(seed, 2, nstate, nens, std=1.0),
    }


def batch_local_sizes(nprob: int = 8192, seed: int | None = None):
    """Problem sizes (nobs_i, nens_i) of the batched workload."""
    seed = seed_for("batch_local") if seed is None else seed
    u = uniform(seed, 1, nprob, np.log(16.0), np.log(4096.0))
    nobs = np.rint(np.exp(u)).astype(np.int64)
    pick = u64(seed, 2, nprob) % np.uint64(4)
    nens = (32 * (pick.astype(np.int64) + 1)).astype(np.int64)
    return nobs, nens


def batch_local_problem(i: int, nobs: int, nens: int, seed: int | None = None, dtype=np.float32):
    """Inputs of problem i of the batched workload: V (nens, nobs), D (nens, nobs), r (nobs,)."""
    seed = seed_for("batch_local") if seed is None else seed
    base = 16 + 8 * i
    s = uniform(seed, base + 0, nobs, 0.5, 2.0)
    V = normal_matrix(seed, base + 1, nobs, nens, std=1.0 / np.sqrt(nens - 1.0), row_scale=s, dtype=dtype)
    r = uniform(seed, base + 2, nobs, 0.5, 1.5).astype(dtype)
    D = normal_matrix(seed, base + 3, nobs, nens, dtype=dtype)
    return {"V": V, "D": D, "r": r}


def batch_local_packed(nprob: int = 8192, seed: int | None = None, nens_override=None, nobs_override=None):
    """Packs the inputs of the batched workload into one float32 buffer.

    Returns (base_in numpy float32, descriptors, out_floats, sizes): descriptor i
    holds float offsets of r_i, V_i (column-major, ld = nobs_i), D_i and of the
    outputs Z_i (column-major) and M_i (nens_i x nens_i) in an output buffer of
    out_floats floats.  Offsets are multiples of 4 floats."""
    seed = seed_for("batch_local") if seed is None else seed
    nobs, nens = batch_local_sizes(nprob, seed)
    if nens_override is not None:
        nens = np.asarray(nens_override, dtype=np.int64)
    if nobs_override is not None:
        nobs = np.asarray(nobs_override, dtype=np.int64)

    def up4(x):
        return (int(x) + 3) // 4 * 4

    descs, off_in, off_out = [], 0, 0
    for i in range(nprob):
        n, N = int(nobs[i]), int(nens[i])
        d = {"nobs": n, "nens": N, "ldv": n, "ldd": n, "ldz": n}
        d["r"] = off_in
        off_in += up4(n)
        d["V"] = off_in
        off_in += up4(n * N)
        d["D"] = off_in
        off_in += up4(n * N)
        d["Z"] = off_out
        off_out += up4(n * N)
        d["M"] = off_out
        off_out += up4(N * N)
        descs.append(d)
    base = np.zeros(off_in, dtype=np.float32)
    for i, d in enumerate(descs):
        n, N = d["nobs"], d["nens"]
        p = batch_local_problem(i, n, N, seed, dtype=np.float32)
        base[d["r"]:d["r"] + n] = p["r"]
        base[d["V"]:d["V"] + n * N] = p["V"].reshape(-1)
        base[d["D"]:d["D"] + n * N] = p["D"].reshape(-1)
    return base, descs, off_out
