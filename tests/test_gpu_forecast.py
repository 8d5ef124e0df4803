"""Parity of the Lorenz-96 RK4 forecast kernel (enkf_forecast) with the oracle.

The FP64 kernel evaluates the same explicitly rounded operations in the same
order as the oracle, so the results are compared bit for bit.  The FP32 kernel is
compared within 1e-5 relative (a few steps of a chaotic system)."""
import numpy as np
import pytest

import oracle
import synth
from tests.util import host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1302_3876_gb300 import enkf  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    enkf.load(build_if_missing=True)


def ensemble(seed, nstate, nens, spread=1.0):
    return 8.0 + spread * synth.normal_matrix(seed, 1, nstate, nens)


@pytest.mark.parametrize("nstate,nens,nsteps", [(4, 1, 3), (5, 2, 7), (40, 20, 100), (101, 3, 50), (4096, 8, 5),
                                                 (6144, 2, 5)])
def test_rk4_fp64_bitwise(nstate, nens, nsteps):
    X0 = ensemble(nstate + nens, nstate, nens)
    ref = oracle.l96_rk4(X0, F=8.0, dt=0.01, nsteps=nsteps)
    t = torch.from_numpy(X0.copy()).cuda()
    enkf.enkf_forecast(t, 8.0, 0.01, nsteps)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(host(t), ref)


def test_rk4_fp64_padded_ld():
    nstate, nens, ld = 40, 5, 64
    X0 = ensemble(3, nstate, nens)
    buf = np.full((nens, ld), 123.0)
    buf[:, :nstate] = X0
    t = torch.from_numpy(buf).cuda()
    enkf.enkf_forecast(t[:, :nstate], 8.0, 0.01, 20)
    out = host(t)
    np.testing.assert_array_equal(out[:, :nstate], oracle.l96_rk4(X0, 8.0, 0.01, 20))
    np.testing.assert_array_equal(out[:, nstate:], 123.0)     # padding untouched


def test_rk4_fp32_close():
    nstate, nens = 4096, 16
    X0 = ensemble(5, nstate, nens).astype(np.float32).astype(np.float64)
    ref = oracle.l96_rk4(X0, 8.0, 0.01, 5)
    t = torch.from_numpy(X0.astype(np.float32)).cuda()
    enkf.enkf_forecast(t, 8.0, 0.01, 5)
    err = np.linalg.norm(host(t) - ref) / np.linalg.norm(ref)
    assert err <= 1e-5


def test_rk4_fixed_point_and_errors():
    t = torch.full((3, 40), 8.0, dtype=torch.float64, device="cuda")
    enkf.enkf_forecast(t, 8.0, 0.01, 10)
    assert torch.equal(t, torch.full_like(t, 8.0))
    with pytest.raises(enkf.EnkfError) as e:
        enkf.enkf_forecast(torch.zeros(2, 7000, dtype=torch.float64, device="cuda"), 8.0, 0.01, 1)
    assert e.value.status == enkf.ENKF_ERR_SHAPE
