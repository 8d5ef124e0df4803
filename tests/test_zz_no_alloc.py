"""enkf_ism_solve_noalloc: the solve for callers that cannot allocate device memory.

Such callers (for example a plugin whose host application already owns the GPU
memory through its own pool) cannot give enkf_ism_analysis a workspace.  The
no-allocation entry point keeps its scratch in the library's static device
array; these tests check, through the C ABI, that two calls in a row give the
same Z as the workspace entry point and as the FP64 oracle, within the
tolerance of the other parity tests (1e-10 FP64, 1e-5 FP32), that an
asynchronous call (no status word) gives the same Z once the stream is
synchronised, and that a device-side error comes back through the status word.
The file is collected last; one test also runs the file again in a fresh
Python process, so that it is known to pass alone as well as after the others.
"""
import math
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import synth
from tests.util import host, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1302_3876_gb300 import enkf  # noqa: E402

TOL = {torch.float64: 1e-10, torch.float32: 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    enkf.load(build_if_missing=True)


def problem(seed, nobs, nens, dt):
    s = synth.uniform(seed, 1, nobs, 0.5, 2.0)
    V = synth.normal_matrix(seed, 2, nobs, nens, std=1.0 / math.sqrt(nens - 1), row_scale=s)
    r = synth.uniform(seed, 3, nobs, 0.5, 1.5)
    D = synth.normal_matrix(seed, 4, nobs, nens)
    return (torch.from_numpy(r).cuda().to(dt), torch.from_numpy(V).cuda().to(dt),
            torch.from_numpy(D).cuda().to(dt))


def workspace_solve(r, V, D):
    nens, nobs = V.shape
    mode = enkf.ENKF_FP64 if V.dtype == torch.float64 else enkf.ENKF_FP32
    plan = enkf.Plan(nobs, nobs, nens, mode)
    Z = torch.empty_like(D)
    inf = plan.analysis(r, V, D, Z=Z, info=True)
    assert inf.status == 0
    plan.close()
    return host(Z)


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_noalloc_matches_workspace_entry_twice(dt):
    cases = [(20000, 48, 101), (777, 9, 102)]          # two different problems, one call after the other
    for nobs, nens, seed in cases:
        r, V, D = problem(seed, nobs, nens, dt)
        ref = workspace_solve(r, V, D)
        Z = torch.full_like(D, float("nan"))
        assert enkf.enkf_ism_solve_noalloc(r, V, D, Z) == 0
        torch.cuda.synchronize()
        assert rel(host(Z), ref) <= TOL[dt]
        assert rel(host(Z), oracle.ism_solve(host(r), host(V), host(D))) <= TOL[dt]
    # the same problem again: the scratch keeps the previous call's contents, the
    # result must not depend on them
    nobs, nens, seed = cases[0]
    r, V, D = problem(seed, nobs, nens, dt)
    ref = workspace_solve(r, V, D)
    Z1 = torch.empty_like(D)
    Z2 = torch.empty_like(D)
    assert enkf.enkf_ism_solve_noalloc(r, V, D, Z1) == 0
    assert enkf.enkf_ism_solve_noalloc(r, V, D, Z2) == 0
    assert rel(host(Z1), ref) <= TOL[dt]
    assert rel(host(Z2), ref) <= TOL[dt]


def test_noalloc_rejects_sizes_beyond_the_static_scratch():
    nobs, nens = 1 << 20, 64            # U alone would need 256 MiB in float
    r = torch.ones(nobs, device="cuda")
    V = torch.zeros(nens, nobs, device="cuda")
    D = torch.zeros(nens, nobs, device="cuda")
    Z = torch.empty_like(D)
    with pytest.raises(enkf.EnkfError) as e:
        enkf.enkf_ism_solve_noalloc(r, V, D, Z)
    assert e.value.status == enkf.ENKF_ERR_WORKSPACE
    assert "static array" in str(e.value)


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_noalloc_asynchronous_call(dt):
    """status NULL: the call returns at once; after a synchronise Z equals the oracle's."""
    nobs, nens = 5000, 24
    r, V, D = problem(103, nobs, nens, dt)
    Z = torch.full_like(D, float("nan"))
    assert enkf.enkf_ism_solve_noalloc(r, V, D, Z, sync=False) == 0
    torch.cuda.synchronize()
    assert rel(host(Z), oracle.ism_solve(host(r), host(V), host(D))) <= TOL[dt]


def test_noalloc_reports_a_numeric_error_through_the_status_word():
    """A NaN innovation latches ENKF_ERR_NUMERIC on the device; the status word brings it back,
    and the next call (valid data, same static array) succeeds."""
    nobs, nens = 1000, 8
    r, V, D = problem(104, nobs, nens, torch.float32)
    Dbad = D.clone()
    Dbad[3, 17] = float("nan")
    Z = torch.empty_like(D)
    with pytest.raises(enkf.EnkfError) as e:
        enkf.enkf_ism_solve_noalloc(r, V, Dbad, Z)
    assert e.value.status == enkf.ENKF_ERR_NUMERIC
    assert enkf.enkf_ism_solve_noalloc(r, V, D, Z) == 0
    assert rel(host(Z), oracle.ism_solve(host(r), host(V), host(D))) <= TOL[torch.float32]


def test_noalloc_file_passes_alone_in_a_fresh_process():
    if os.environ.get("ENKF_NOALLOC_CHILD"):
        pytest.skip("already the fresh process")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, ENKF_NOALLOC_CHILD="1")
    res = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
                          os.path.abspath(__file__)], cwd=root, env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stdout[-2000:] + res.stderr[-2000:]
