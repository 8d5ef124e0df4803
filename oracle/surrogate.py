"""FP64 oracle of the learned Lorenz-96 forecast surrogate.

TEST INFRASTRUCTURE ONLY (imported by tests/, the smoke check and the CPU
baseline of the benchmark; never by the CUDA library).

The surrogate replaces the model propagation of the forecast step (Sec. 2, eq.
forecast-step) between analyses: x_{t+T} ~ x_t + s_out * f(x_t) with f a 4-layer
periodic 1-D convolutional network over the state index (channels 1 -> 64 -> 64
-> 64 -> 1, kernel 5, circular padding 2, GELU-tanh between layers):

    z0[0, p] = (x[p] - shift) * scale_in
    y_l[o, p] = b_l[o] + sum_i sum_{t=0..4} W_l[o, i, t] z_{l-1}[i, (p + t - 2) mod P]
    z_l = gelu(y_l)  for l = 1, 2, 3;      x_next = x + s_out * y_4[0, :]

gelu(u) = 0.5 u (1 + tanh(sqrt(2/pi) (u + 0.044715 u^3))).  The loss of a batch
is the mean squared error over positions and members.  Adam (Kingma and Ba,
2015) with bias correction updates the parameters.

Everything here is plain numpy in float64 with explicit loops over the 5 taps;
a state batch is an array of shape (members, P).
"""
from __future__ import annotations

import math

import numpy as np

WIDTH = 64
KERNEL = 5
PAD = 2
SHIFT = 2.5
SCALE_IN = 0.25
SCALE_OUT = 1.0
CHANNELS = (1, WIDTH, WIDTH, WIDTH, 1)
GELU_C = math.sqrt(2.0 / math.pi)
GELU_A = 0.044715


def param_shapes():
    """[(W shape (out, in, 5), b shape (out,))] for the 4 layers."""
    return [((CHANNELS[l + 1], CHANNELS[l], KERNEL), (CHANNELS[l + 1],)) for l in range(4)]


def n_params():
    return sum(int(np.prod(w)) + int(np.prod(b)) for w, b in param_shapes())


def init_params(seed_values):
    """Parameters from a flat vector of standard normals (length n_params()):
    W ~ N(0, 1/(in*5)) * gain, b = 0 (He-like scaling for GELU layers; the last
    layer is scaled by 0.1 so the initial increment is small)."""
    params, off = [], 0
    for l, (ws, bs) in enumerate(param_shapes()):
        nw = int(np.prod(ws))
        fan_in = ws[1] * ws[2]
        gain = math.sqrt(2.0) if l < 3 else 0.1
        W = np.asarray(seed_values[off:off + nw], dtype=np.float64).reshape(ws) * gain / math.sqrt(fan_in)
        off += nw
        off += int(np.prod(bs))
        params.append([W, np.zeros(bs)])
    return params


def conv(z, W, b):
    """y[m, o, p] = b[o] + sum_i sum_t W[o, i, t] z[m, i, (p + t - 2) mod P]."""
    y = np.broadcast_to(b[None, :, None], (z.shape[0], W.shape[0], z.shape[2])).copy()
    for t in range(KERNEL):
        zs = np.roll(z, -(t - PAD), axis=2)          # zs[..., p] = z[..., (p + t - 2) mod P]
        y += np.einsum("oi,mip->mop", W[:, :, t], zs)
    return y


def conv_backward(z, W, gy):
    """Gradients of sum(gy * conv(z, W, b)) w.r.t. z, W and b."""
    gz = np.zeros_like(z)
    gW = np.zeros_like(W)
    for t in range(KERNEL):
        zs = np.roll(z, -(t - PAD), axis=2)
        gW[:, :, t] = np.einsum("mop,mip->oi", gy, zs)
        gzs = np.einsum("oi,mop->mip", W[:, :, t], gy)
        gz += np.roll(gzs, (t - PAD), axis=2)
    gb = gy.sum(axis=(0, 2))
    return gz, gW, gb


def gelu(u):
    return 0.5 * u * (1.0 + np.tanh(GELU_C * (u + GELU_A * u ** 3)))


def gelu_grad(u):
    k = GELU_C * (u + GELU_A * u ** 3)
    th = np.tanh(k)
    return 0.5 * (1.0 + th) + 0.5 * u * (1.0 - th * th) * GELU_C * (1.0 + 3.0 * GELU_A * u * u)


def forward(params, x, keep=False):
    """x: (members, P) -> x_next (members, P); with keep, also the layer inputs/pre-activations."""
    z = ((x - SHIFT) * SCALE_IN)[:, None, :]
    cache = []
    for l, (W, b) in enumerate(params):
        y = conv(z, W, b)
        cache.append((z, y))
        z = gelu(y) if l < 3 else y
    out = x + SCALE_OUT * z[:, 0, :]
    return (out, cache) if keep else out


def loss_and_grads(params, x, target):
    """MSE loss over all entries and its gradients (list of [gW, gb])."""
    out, cache = forward(params, x, keep=True)
    diff = out - target
    loss = float(np.mean(diff * diff))
    g = (2.0 / diff.size) * diff                     # dL/d out
    gy = (SCALE_OUT * g)[:, None, :]                 # dL/d y_4
    grads = [None] * 4
    for l in range(3, -1, -1):
        z, y = cache[l]
        if l < 3:
            gy = gy * gelu_grad(y)
        gz, gW, gb = conv_backward(z, params[l][0], gy)
        grads[l] = [gW, gb]
        gy = gz
    return loss, grads


def adam_step(params, grads, state, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step in place; state = {"t": int, "m": [...], "v": [...]} (created if empty)."""
    if not state:
        state["t"] = 0
        state["m"] = [[np.zeros_like(p) for p in layer] for layer in params]
        state["v"] = [[np.zeros_like(p) for p in layer] for layer in params]
    state["t"] += 1
    t = state["t"]
    for l in range(4):
        for q in range(2):
            m = state["m"][l][q] = beta1 * state["m"][l][q] + (1 - beta1) * grads[l][q]
            v = state["v"][l][q] = beta2 * state["v"][l][q] + (1 - beta2) * grads[l][q] ** 2
            mhat = m / (1 - beta1 ** t)
            vhat = v / (1 - beta2 ** t)
            params[l][q] = params[l][q] - lr * mhat / (np.sqrt(vhat) + eps)
    return params


def flatten(params):
    """Flat parameter vector in the order W1, b1, W2, b2, W3, b3, W4, b4 (W row-major (out, in, tap))."""
    return np.concatenate([np.concatenate([W.reshape(-1), b.reshape(-1)]) for W, b in params])


def unflatten(vec):
    params, off = [], 0
    for ws, bs in param_shapes():
        nw, nb = int(np.prod(ws)), int(np.prod(bs))
        params.append([np.asarray(vec[off:off + nw], dtype=np.float64).reshape(ws),
                       np.asarray(vec[off + nw:off + nw + nb], dtype=np.float64)])
        off += nw + nb
    return params


def rmse_time_mean(truth, means):
    """RMSE of Sec. 4.1: the time mean of the per-time root mean square error of the
    ensemble mean, (1/Nsteps) sum_t sqrt(|x_t^true - xbar_t|^2 / Nstate)."""
    truth, means = np.asarray(truth), np.asarray(means)
    return float(np.mean(np.sqrt(np.mean((truth - means) ** 2, axis=1))))
