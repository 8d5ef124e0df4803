"""Parity of the surrogate kernels (enkf_forecast with ENKF_FORECAST_SURROGATE and
enkf_surrogate_train_step) with the FP64 oracle (oracle/surrogate.py).

The kernels store weights and activations in BF16 (unit roundoff 2^-9) and
accumulate in FP32.  Tolerances, stated per result: the increment x_next - x
within 3e-2 relative (BF16 activations through four layers), x_next within 1e-3;
the flat gradient within 5e-2 relative; the Adam update on the device's own
gradient within 1e-5 relative (FP32 arithmetic)."""
import numpy as np
import pytest

import oracle
import synth
from oracle import surrogate as S
from tests.util import rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1302_3876_gb300 import enkf  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    enkf.load(build_if_missing=True)


def device_params(seed):
    params = S.init_params(synth.normal_matrix(seed, 1, S.n_params(), 1)[0])
    # non-zero biases so every term is exercised
    for l, (W, b) in enumerate(params):
        b[:] = 0.05 * synth.normal_matrix(seed, 10 + l, b.size, 1)[0]
    flat = S.flatten(params).astype(np.float32)
    params = S.unflatten(flat.astype(np.float64))          # the values the device sees
    n, pbytes, _ = enkf.enkf_surrogate_sizes(128, 1)
    assert n == S.n_params()
    master = torch.from_numpy(flat).cuda()
    packed = torch.empty(pbytes, dtype=torch.uint8, device="cuda")
    enkf.enkf_surrogate_pack(master, packed)
    return params, master, packed


def lorenz_states(seed, nstate, nens):
    x = 8.0 + synth.normal_matrix(seed, 3, nstate, 1)[0][None, :] + 0.5 * synth.normal_matrix(seed, 4, nstate, nens)
    return x.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("nstate,nens", [(300, 3), (4096, 2), (128, 5), (40, 4)])
def test_forward_matches_oracle(nstate, nens):
    params, master, packed = device_params(11)
    x = lorenz_states(12 + nstate, nstate, nens)
    ref = S.forward(params, x)
    t = torch.from_numpy(x.astype(np.float32)).cuda()
    ws = torch.empty(enkf.enkf_forecast_workspace(nstate, nens, enkf.ENKF_FORECAST_SURROGATE), dtype=torch.uint8,
                     device="cuda")
    enkf.enkf_forecast(t, 8.0, 0.05, 1, method=enkf.ENKF_FORECAST_SURROGATE, weights=packed, workspace=ws)
    out = t.cpu().numpy().astype(np.float64)
    assert rel(out - x, ref - x) <= 3e-2
    assert rel(out, ref) <= 1e-3


def test_gradient_matches_oracle():
    params, master, packed = device_params(21)
    nstate, nb = 256, 3
    x = lorenz_states(22, nstate, nb)
    target = (x + 0.3 * synth.normal_matrix(23, 1, nstate, nb)).astype(np.float32).astype(np.float64)
    loss_ref, grads = S.loss_and_grads(params, x, target)
    gref = S.flatten(grads)
    _, _, tw = enkf.enkf_surrogate_sizes(nstate, nb)
    ws = torch.empty(tw, dtype=torch.uint8, device="cuda")
    tx = torch.from_numpy(x.astype(np.float32)).cuda()
    tt = torch.from_numpy(target.astype(np.float32)).cuda()
    sq = torch.zeros(1, device="cuda")
    g = torch.zeros(S.n_params(), device="cuda")
    enkf.enkf_surrogate_train_step(master, None, None, 0, 0.0, packed, tx, tt, ws, sq, grad=g)
    torch.cuda.synchronize()
    assert float(sq.item()) / x.size == pytest.approx(loss_ref, rel=3e-2)
    gd = g.cpu().numpy().astype(np.float64)
    assert rel(gd, gref) <= 5e-2
    # every layer's block individually
    off = 0
    for (ws_shape, bs_shape) in S.param_shapes():
        n = int(np.prod(ws_shape)) + int(np.prod(bs_shape))
        assert rel(gd[off:off + n], gref[off:off + n]) <= 8e-2
        off += n


def test_adam_step_matches_oracle_on_device_gradient():
    params, master, packed = device_params(31)
    nstate, nb = 256, 2
    x = lorenz_states(32, nstate, nb)
    target = x + 0.1
    _, _, tw = enkf.enkf_surrogate_sizes(nstate, nb)
    ws = torch.empty(tw, dtype=torch.uint8, device="cuda")
    tx = torch.from_numpy(x.astype(np.float32)).cuda()
    tt = torch.from_numpy(target.astype(np.float32)).cuda()
    sq = torch.zeros(1, device="cuda")
    g = torch.zeros(S.n_params(), device="cuda")
    m = torch.zeros_like(master)
    v = torch.zeros_like(master)
    before = master.clone()
    enkf.enkf_surrogate_train_step(master, m, v, 1, 1e-3, packed, tx, tt, ws, sq, grad=g)
    torch.cuda.synchronize()
    p_ref = S.unflatten(before.cpu().numpy().astype(np.float64))
    g_dev = S.unflatten(g.cpu().numpy().astype(np.float64))
    S.adam_step(p_ref, g_dev, {}, lr=1e-3)
    step_ref = S.flatten(p_ref) - before.cpu().numpy()
    step_dev = (master - before).cpu().numpy().astype(np.float64)
    assert rel(step_dev, step_ref) <= 1e-5


def test_training_reduces_the_loss_on_rk4_pairs():
    """A few hundred Adam steps on (x, RK4^5(x)) pairs must cut the MSE by 10x."""
    nstate, nb = 512, 8
    _, master, packed = device_params(41)
    _, _, tw = enkf.enkf_surrogate_sizes(nstate, nb)
    ws = torch.empty(tw, dtype=torch.uint8, device="cuda")
    m = torch.zeros_like(master)
    v = torch.zeros_like(master)
    sq = torch.zeros(1, device="cuda")
    # a pool of states on the attractor: spin up, then sample along a trajectory
    x0 = oracle.l96_rk4(8.0 + synth.normal_matrix(42, 1, nstate, 1)[0], 8.0, 0.01, 500)[0]
    pool = [x0]
    for _ in range(63):
        pool.append(oracle.l96_rk4(pool[-1], 8.0, 0.01, 7)[0])
    pool = np.array(pool).astype(np.float32)
    tgt_pool = torch.from_numpy(pool.copy()).cuda()
    enkf.enkf_forecast(tgt_pool, 8.0, 0.01, 5)       # targets: 5 RK4 steps on the device
    src_pool = torch.from_numpy(pool).cuda()
    losses = []
    for step in range(1, 401):
        idx = torch.tensor([(step * 7 + q * 11) % 64 for q in range(nb)], device="cuda")
        xb = src_pool[idx].contiguous()
        tb = tgt_pool[idx].contiguous()
        enkf.enkf_surrogate_train_step(master, m, v, step, 2e-3, packed, xb, tb, ws, sq)
        if step in (1, 400):
            torch.cuda.synchronize()
            losses.append(float(sq.item()) / xb.numel())
    assert losses[1] < losses[0] / 10.0, losses
