"""EnKF assimilation cycle on Lorenz-96 through the C ABI (Sec. 2: forecast and
analysis steps repeated; Sec. 4.2: the Lorenz-96 experiment).

Each cycle: forecast every member (RK4 ``substeps`` steps, or one application
of the learned surrogate, or persistence), propagate the truth with RK4, draw
the observations y = H truth + noise and perturbations (host draws from
``synth``), then the analysis: enkf_obs_prep (deviations, V, D) and
enkf_ism_analysis, X_A written over X_B.  Optionally the prep inflates the
ensemble first (enkf_inflate_prep, Sec. 3.1.1) and the update is localized
(Z from enkf_ism_analysis, then enkf_localized_update, Sec. 3.1.2).  The RMSE is the time mean of the
per-cycle root mean square error of the ensemble mean (Sec. 4.1).

This module is orchestration only: the forecast, the prep and the analysis run
in the library's kernels; torch provides device memory.
"""
from __future__ import annotations

import math
import time

import numpy as np

import synth

from . import enkf


class LorenzCycle:
    def __init__(self, nstate=4096, nens=256, obs_stride=2, r=0.25, forcing=8.0, dt=0.01, substeps=5,
                 mode=enkf.ENKF_FP32, seed=None, device="cuda", spinup=1000, inflation=1.0, loc_length=None,
                 loc_radius=None):
        import torch
        self.torch = torch
        self.nstate, self.nens, self.stride, self.r, self.F, self.dt = nstate, nens, obs_stride, r, forcing, dt
        self.substeps = substeps
        self.nobs = (nstate + obs_stride - 1) // obs_stride
        self.seed = synth.seed_for("lorenz_cycle") if seed is None else seed
        self.dev = torch.device(device)
        init = synth.lorenz_cycle_init(nstate, nens, forcing, self.seed)
        truth = torch.from_numpy(init["truth0"][None, :].copy()).to(self.dev)          # FP64 truth
        enkf.enkf_forecast(truth, forcing, dt, spinup)
        self.truth = truth
        self.X = (truth.float() + torch.from_numpy(init["ens_noise"]).to(self.dev).float()).contiguous()
        self.dX = torch.empty_like(self.X)
        self.V = torch.empty(nens, self.nobs, device=self.dev)
        self.D = torch.empty(nens, self.nobs, device=self.dev)
        self.Y = torch.empty(nens, self.nobs, device=self.dev)
        self.rvec = torch.full((self.nobs,), r, device=self.dev)
        self.plan = enkf.Plan(nstate, self.nobs, nens, mode, device=self.dev)
        self.inflation, self.loc_length, self.loc_radius = float(inflation), loc_length, loc_radius
        self.Z = torch.empty(nens, self.nobs, device=self.dev, dtype=self.X.dtype) if loc_length else None
        self.cycle_index = 0
        self.sur_packed = None
        self.sur_ws = None

    def set_surrogate(self, packed):
        self.sur_packed = packed
        nbytes = enkf.enkf_forecast_workspace(self.nstate, self.nens, enkf.ENKF_FORECAST_SURROGATE)
        self.sur_ws = self.torch.empty(nbytes, dtype=self.torch.uint8, device=self.dev)

    def forecast(self, method):
        if method == "rk4":
            enkf.enkf_forecast(self.X, self.F, self.dt, self.substeps)
        elif method == "surrogate":
            enkf.enkf_forecast(self.X, self.F, self.dt, 1, method=enkf.ENKF_FORECAST_SURROGATE,
                               weights=self.sur_packed, workspace=self.sur_ws)
        elif method != "persistence":
            raise ValueError(method)
        enkf.enkf_forecast(self.truth, self.F, self.dt, self.substeps)

    def analysis(self):
        torch = self.torch
        draws = synth.lorenz_cycle_draws(self.cycle_index, self.nstate, self.nens, self.stride, self.r, self.seed)
        y = self.truth[0, ::self.stride].float() + torch.from_numpy(draws["obs_noise"]).to(self.dev).float()
        self.Y.copy_(y[None, :] + torch.from_numpy(draws["pert"]).to(self.dev).float())
        if self.inflation != 1.0:
            enkf.enkf_inflate_prep(self.stride, self.inflation, self.X, self.V, dXB=self.dX, Y=self.Y, D=self.D)
        else:
            self.plan.obs_prep(self.stride, 1, self.X, self.dX, self.V, Y=self.Y, D=self.D)
        if self.Z is not None:
            self.plan.analysis(self.rvec, self.V, self.D, Z=self.Z)
            enkf.enkf_localized_update(self.stride, self.loc_length, self.loc_radius, self.dX, self.V, self.Z,
                                       self.X, self.X)
        else:
            self.plan.analysis(self.rvec, self.V, self.D, dXB=self.dX, XB=self.X, XA=self.X)
        self.cycle_index += 1

    def rmse(self):
        """Root mean square error of the ensemble mean against the truth (one time)."""
        return float(self.torch.sqrt(self.torch.mean((self.X.double().mean(0) - self.truth[0]) ** 2)).item())

    def run(self, ncycles, method="rk4", collect=None):
        """Runs ncycles; returns (time-mean analysis RMSE, cycles/s, per-cycle RMSE list).
        collect: list receiving (X_A before the forecast, forecast) pairs (copies)."""
        torch = self.torch
        rm = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ncycles):
            if collect is not None:
                before = self.X.clone()
            self.forecast(method)
            if collect is not None:
                collect.append((before, self.X.clone()))
            self.analysis()
            rm.append(self.rmse())
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        return float(np.mean(rm)), ncycles / el, rm

    def close(self):
        self.plan.close()


def train_surrogate(xs, ys, steps=1500, batch=16, lr=2e-3, seed=4242, master=None, packed=None, log_every=100):
    """Trains the surrogate on rows (xs[i] -> ys[i]) with the library's kernels (Adam,
    cosine-decayed learning rate, minibatches drawn by the counter-based generator).
    xs, ys: CUDA float32 (n, nstate).  Returns (master, packed, [(step, mse)])."""
    import torch
    n, nstate = xs.shape
    if master is None:
        master, packed = surrogate_init(nstate, seed, xs.device)
    _, _, tw = enkf.enkf_surrogate_sizes(nstate, batch)
    ws = torch.empty(tw, dtype=torch.uint8, device=xs.device)
    mom = torch.zeros_like(master)
    vel = torch.zeros_like(master)
    sq = torch.zeros(1, device=xs.device)
    picks = torch.from_numpy((synth.u64(seed, 7, steps * batch) % np.uint64(n)).astype(np.int64)).to(xs.device)
    log = []
    for step in range(1, steps + 1):
        idx = picks[(step - 1) * batch: step * batch]
        xb = xs.index_select(0, idx).contiguous()
        yb = ys.index_select(0, idx).contiguous()
        lr_t = lr * 0.5 * (1.0 + math.cos(math.pi * (step - 1) / steps))
        enkf.enkf_surrogate_train_step(master, mom, vel, step, lr_t, packed, xb, yb, ws, sq)
        if log_every and (step % log_every == 0 or step == 1):
            log.append((step, float(sq.item()) / xb.numel()))
    return master, packed, log


def surrogate_init(nstate, seed=4242, device="cuda"):
    """Initial FP32 master parameters: W ~ N(0, gain^2 / fan_in) (gain sqrt(2) for the GELU
    layers, 0.1 for the output layer), biases zero; packed copy for the kernels."""
    import torch
    n, pbytes, _ = enkf.enkf_surrogate_sizes(nstate, 1)
    z = synth.normal_matrix(seed, 1, n, 1)[0]
    shapes = [((64, 1, 5), 64), ((64, 64, 5), 64), ((64, 64, 5), 64), ((1, 64, 5), 1)]
    out, off = np.zeros(n), 0
    for l, (ws, nb) in enumerate(shapes):
        nw = int(np.prod(ws))
        gain = math.sqrt(2.0) if l < 3 else 0.1
        out[off:off + nw] = z[off:off + nw] * gain / math.sqrt(ws[1] * ws[2])
        off += nw + nb
    master = torch.from_numpy(out.astype(np.float32)).to(device)
    packed = torch.empty(pbytes, dtype=torch.uint8, device=device)
    enkf.enkf_surrogate_pack(master, packed)
    return master, packed
