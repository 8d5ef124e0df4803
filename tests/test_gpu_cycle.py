"""The EnKF cycle on Lorenz-96 (forecast + analysis repeated, Sec. 2 and Sec. 4.2)
through the C ABI, and the learned surrogate inside it.

1. Three RK4 cycles on the device (FP32 ensemble, FP64 truth) against the same
   cycles composed from the oracle in FP64, on the same draws: the ensemble after
   three cycles within 2e-4 relative (FP32 analysis on a chaotic system).
2. The surrogate, trained by the library's kernels on pairs the filter itself
   generates (training seed), replaces RK4 in the cycle on a held-out truth: the
   analysis RMSE must beat the filter without a forecast model (persistence), and
   the numbers against RK4 are reported."""
import math

import numpy as np
import pytest

import oracle
import synth
from tests.util import rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1302_3876_gb300 import cycle as C  # noqa: E402
from paper_1302_3876_gb300 import enkf  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    enkf.load(build_if_missing=True)


def test_rk4_cycles_match_oracle_cycles():
    nstate, nens, stride, r, seed = 128, 16, 2, 0.25, 99
    cyc = C.LorenzCycle(nstate, nens, stride, r, seed=seed, spinup=300)
    # oracle: same start (truth spun up by the bit-identical FP64 RK4, ensemble as the device holds it)
    X = cyc.X.double().cpu().numpy()
    truth = cyc.truth.cpu().numpy()[0]
    nobs = nstate // stride
    for c in range(3):
        cyc.forecast("rk4")
        cyc.analysis()
        X = oracle.l96_rk4(X, 8.0, 0.01, 5)
        truth = oracle.l96_rk4(truth, 8.0, 0.01, 5)[0]
        d = synth.lorenz_cycle_draws(c, nstate, nens, stride, r, seed)
        # observations formed in FP32 exactly as the cycle does on the device
        y32 = truth[::stride].astype(np.float32) + d["obs_noise"].astype(np.float32)
        Y = (y32[None, :] + d["pert"].astype(np.float32)).astype(np.float64)
        _, dX = oracle.ensemble_deviations(X)
        V = oracle.observe_deviations(dX, nobs, stride)
        D = oracle.innovations(Y, X, stride)
        X = oracle.analysis(np.full(nobs, r), V, D, X, dX)["XA"]
    np.testing.assert_array_equal(cyc.truth.cpu().numpy()[0], truth)
    assert rel(cyc.X.double().cpu().numpy(), X) <= 2e-4
    cyc.close()


def test_surrogate_in_the_cycle_beats_persistence():
    nstate, nens = 512, 32
    # training data from the RK4 filter itself (training seed)
    train = C.LorenzCycle(nstate, nens, seed=555, spinup=500)
    pairs = []
    train.run(40, "rk4", collect=pairs)
    xs = torch.cat([a for a, _ in pairs]).contiguous()
    ys = torch.cat([b for _, b in pairs]).contiguous()
    train.close()
    master, packed, log = C.train_surrogate(xs, ys, steps=800, batch=16, lr=2e-3)
    assert log[-1][1] < log[0][1] / 10.0, log
    results = {}
    for method in ("rk4", "surrogate", "persistence"):
        cyc = C.LorenzCycle(nstate, nens, seed=777, spinup=500)
        if method == "surrogate":
            cyc.set_surrogate(packed)
        results[method] = cyc.run(40, method)[:2]
        cyc.close()
    print("cycle RMSE / cycles/s:", {k: (round(v[0], 4), round(v[1], 1)) for k, v in results.items()})
    assert all(math.isfinite(v[0]) for v in results.values())
    assert results["surrogate"][0] < results["persistence"][0]
    assert results["rk4"][0] < results["persistence"][0]
