#!/usr/bin/env python3
"""Benchmark of the iterative Sherman-Morrison EnKF analysis on one GB300.

Workload (default): the panel workload -- Nstate = 2^22, Nobs = 2^20 (every 4th
state variable observed), Nens = 256; deviations dX_B[i,e] = s_i N(0,1) with
s_i ~ U[0.5, 2], variances r_j ~ U[0.5, 1.5], innovations D ~ N(0,1), and the
background equal in value to the deviations but held in a buffer of its own.
``--workload large_single`` takes Nstate = 2^21, Nobs = 2^19, Nens = 128.  One step
= the whole analysis through the C ABI: V = H dX_B / sqrt(Nens-1) on the device,
Step 1 + Step 2 of the iterative Sherman-Morrison formula, one step of iterative
refinement, M = V^T Z / sqrt(Nens-1), X_A = X_B + dX_B M.  Inputs (several GB) are
larger than L2, so no flush is needed between steps.

The headline path is the panel form on tcgen05 tensor cores (32 levels per pass,
operands split in three BF16 pieces, FP64-class denominators) with one refinement
step (``--mode`` selects the other panel variants or the plain FP32 level-streaming
path, ``--no-refine`` drops the refinement); the FP64 plain path is timed in the
same run as the comparator, with the errors of every result against it.
``--impl reference`` times the FP64 CPU oracle instead (bounded sample of the same
workload).  Other workloads (``--workload``): the batched local analyses, the
single Lorenz-96 analysis (one call and CUDA-graph replays), the Lorenz-96 cycle
with the learned surrogate, and the rows beside the analysis (inflation, partial
localization, block-diagonal R, pivoting); each prints its own JSON line.

Prints ONE JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "analyses/s"
NSTATE, NOBS, NENS, STRIDE = 1 << 21, 1 << 19, 128, 4
WORKLOAD = f"large_single Nstate={NSTATE} Nobs={NOBS} Nens={NENS} (every {STRIDE}th variable observed)"


def flops(nstate, nobs, nens):
    """Flop convention: F_solve = 6 Nobs Nens^2 + 3 Nobs Nens (Sec. 3.2 counts, a
    multiply-add = 2), F_M = 2 Nobs Nens^2, F_XA = 2 Nstate Nens^2 + Nstate Nens."""
    return 6 * nobs * nens ** 2 + 3 * nobs * nens + 2 * nobs * nens ** 2 + 2 * nstate * nens ** 2 + nstate * nens


def level_bytes(nobs, nens, w):
    """Algorithmic bytes of the level-streaming kernel per launch: Step 1 reads D, V
    and writes Z, U (4 N Nobs); level k reads and writes its 2N-1-k active columns
    and reads u_k and v_{k+1} (2 columns); summed: w Nobs (3 N^2 + 5 N)."""
    return w * nobs * (3 * nens * nens + 5 * nens)


def panel_bytes(nobs, nens, b, w):
    """Algorithmic bytes of one panel-kernel launch: the first pass reads the 2N columns
    of [U | Z] and b columns of V; panel p (start k0) reads and writes its 2N - k0 - b
    trailing columns, reads the b panel columns of U and the next b columns of V, and
    rewrites the b panel columns with their final values."""
    cols = 2 * nens + b
    for k0 in range(0, nens, b):
        bp = min(b, nens - k0)
        nb = min(b, max(0, nens - k0 - bp))
        cols += 2 * (2 * nens - k0 - bp) + bp + nb + 2 * bp
    return w * nobs * cols


def correction_bytes(nobs, nens, b, w):
    """Algorithmic bytes of the refinement's correction sweep (the tensor-core kernel with
    the stored factors): the first pass reads the N columns of the scaled residual and b
    columns of V; panel p reads and writes the N columns, reads its b final U columns and
    the next b columns of V."""
    cols = nens + b
    for k0 in range(0, nens, b):
        bp = min(b, nens - k0)
        nb = min(b, max(0, nens - k0 - bp))
        cols += 2 * nens + bp + nb
    return w * nobs * cols


def read_bf16_sustained():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["bf16_tflops_sustained"])
    except Exception:  # noqa: BLE001
        return 1700.0


def measure_fma_peaks(dev, local):
    """FP32 and FP64 CUDA-core multiply-add peaks measured on this GPU by the library's own
    microbenchmark (enkf_fma_peak_launch: 16 independent FMA chains per thread, 4 CTAs of 256
    threads per SM), timed with CUDA events after a warm-up, the SM clock sampled meanwhile.
    Returns {"fp32_tflops", "fp64_tflops", "sm_mhz", "how"}."""
    import torch
    from paper_1302_3876_gb300 import enkf
    sink = torch.zeros(2, dtype=torch.float64, device=dev)
    out = {}
    with ClockSampler(local) as clk:
        for name, prec, iters in (("fp32_tflops", enkf.ENKF_FP32, 1 << 16), ("fp64_tflops", enkf.ENKF_FP64, 1 << 12)):
            enkf.enkf_fma_peak_launch(prec, iters, 4, sink)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            best = float("inf")
            flops = 0.0
            for _ in range(5):
                e0.record()
                flops = enkf.enkf_fma_peak_launch(prec, iters, 4, sink)
                e1.record()
                torch.cuda.synchronize(dev)
                best = min(best, e0.elapsed_time(e1))
            out[name] = flops / (best / 1e3) / 1e12
    out["sm_mhz"] = clk.summary().get("sm_mhz")
    out["how"] = ("enkf_fma_peak_launch: 4 CTAs x 256 threads per SM, 16 independent FMA chains per thread, "
                  "best of 5 launches by CUDA events")
    return out


def read_bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["bf16_tflops"])
    except Exception:  # noqa: BLE001
        return 1900.0


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:  # noqa: BLE001
        return 6800.0, "fallback"


def profile_traffic(kernel_src: str, summary_name: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the
    current source of the kernel (sha256 recorded in the summary)."""
    path = os.path.join(ROOT, "profiles", summary_name)
    try:
        text = open(path).read()
        sha = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()
        m_sha = re.search(r"source_sha256:\s*([0-9a-f]{64})", text)
        m_tr = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
        if m_sha and m_tr and m_sha.group(1) == sha:
            return float(m_tr.group(1))
    except OSError:
        pass
    return None


class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        mhz, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                mhz.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not mhz:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(mhz)}


def aggregate_ranks(t_ms: float, steps: int, world: int, device=None):
    """Replicas on `world` ranks each time `steps` analyses: the job's time is the
    slowest rank's (all-reduce MAX), and the whole-job throughput counts every
    rank's analyses: value = world * steps / t_max."""
    t_max = t_ms
    if world > 1:
        import torch
        import torch.distributed as dist
        tt = torch.tensor([t_ms], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max = float(tt.item())
    return t_max, world * steps / (t_max / 1e3)


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


CPU_FRAC = {"panel_single": 5, "large_single": 3}   # row sample of the oracle: 1/2^k of the rows


def cpu_oracle_sample(frac_log2: int, seconds: float, seed_offset: int = 0):
    """Times the FP64 oracle on a row sample of the workload: Nobs and Nstate divided
    by 2^frac_log2, Nens unchanged (cost is linear in Nobs and Nstate)."""
    import numpy as np
    import oracle
    import synth
    nobs, nstate = NOBS >> frac_log2, NSTATE >> frac_log2
    gen = synth.panel_single if NENS == 256 else synth.large_single
    w = gen(nstate, nobs, NENS, dtype=np.float64)
    dXB, r, D = w["dXB"], w["r"], w["D"]
    oracle.build()
    runs, t0 = 0, time.perf_counter()
    while True:
        V = oracle.observe_deviations(dXB, nobs, STRIDE)
        oracle.analysis(r, V, D, dXB, dXB, refine=False)     # the paper's steps: one solve
        runs += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    per_run = el / runs
    return {
        "value": (1.0 / per_run) / (1 << frac_log2),
        "unit": METRIC,
        "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)),
        "kind": "oracle",
        "sample": f"Nobs={nobs}, Nstate={nstate}, Nens={NENS} (1/{1 << frac_log2} of the rows), {runs} run(s) "
                  f"in {el:.1f} s; analyses/s scaled by 1/{1 << frac_log2}",
        "seconds_per_sample": per_run,
    }


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    if args.workload not in HEADLINE:
        args.workload = "panel_single"
    set_headline(args)
    frac = CPU_FRAC[args.workload]
    per_step = []
    for _ in range(args.warmup):
        cpu_oracle_sample(frac, 0.0)
    sample = None
    for _ in range(args.steps):
        sample = cpu_oracle_sample(frac, 0.0)
        per_step.append(sample["seconds_per_sample"] * (1 << frac))
    value = args.steps / sum(per_step)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(per_step) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": f"1/{1 << frac} of the rows per step; each step's time is "
                                                   f"the sample's time x {1 << frac} (extrapolated)"},
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": sample["cores"], "kind": "oracle",
                         "sample": sample["sample"]},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


HEADLINE = {
    # name: (Nstate, Nobs, Nens, description)
    "panel_single": (1 << 22, 1 << 20, 256, "panel_single Nstate=4194304 Nobs=1048576 Nens=256 "
                     "(every 4th variable observed)"),
    "large_single": (1 << 21, 1 << 19, 128, "large_single Nstate=2097152 Nobs=524288 Nens=128 "
                     "(every 4th variable observed)"),
}
MODES = {"panel32": "ENKF_PANEL_FP32", "bf16": "ENKF_PANEL_BF16", "fp16": "ENKF_PANEL_FP16",
         "bf16x3": "ENKF_PANEL_BF16X3", "fp32": "ENKF_FP32"}
PATH_NAME = {"panel32": "panel form on FP32 CUDA cores, b=%d (FP64 gamma)",
             "bf16": "panel form on tensor cores, split BF16 operands, b=%d (FP64 gamma)",
             "bf16x3": "panel form on tcgen05 tensor cores (TMEM accumulators, TMA), BF16 operands split in three, "
                       "b=%d (FP64-class gamma)",
             "fp16": "panel form on tensor cores, FP16 operands, b=%d (FP64 gamma)",
             "fp32": "FP32 plain level-streaming (FP64 gamma and cross-CTA sums)"}


def set_headline(args):
    global NSTATE, NOBS, NENS, WORKLOAD
    NSTATE, NOBS, NENS, WORKLOAD = HEADLINE[args.workload]
    if args.scale_div > 1:
        NSTATE //= args.scale_div
        NOBS //= args.scale_div
        WORKLOAD = f"{args.workload}/{args.scale_div} Nstate={NSTATE} Nobs={NOBS} Nens={NENS}"


def run_ours(args):
    set_headline(args)
    import numpy as np
    import torch
    import torch.distributed as dist

    world, rank, local = dist_setup()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import synth
    from paper_1302_3876_gb300 import enkf
    enkf.load(build_if_missing=True)

    # cpu baseline first (rank 0, before any large device allocation)
    cpu = cpu_oracle_sample(CPU_FRAC[args.workload], args.cpu_seconds) \
        if (rank == 0 and world == 1 and not args.no_cpu) else None
    peaks = measure_fma_peaks(dev, local)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    gen = synth.panel_single if args.workload == "panel_single" else synth.large_single
    w = gen(NSTATE, NOBS, NENS, dtype=np.float32)
    h_dX = torch.from_numpy(w["dXB"]).pin_memory()
    h_D = torch.from_numpy(w["D"]).pin_memory()
    h_r = torch.from_numpy(w["r"]).pin_memory()
    del w
    dX = h_dX.to(dev)
    XB = dX.clone()     # the background (equal to the deviations, R-9), in a buffer of its own
    D = h_D.to(dev)
    r = h_r.to(dev)
    V = torch.empty(NENS, NOBS, dtype=torch.float32, device=dev)
    Z = torch.empty(NENS, NOBS, dtype=torch.float32, device=dev)
    XA = torch.empty_like(dX)
    M = torch.empty(NENS * NENS, dtype=torch.float32, device=dev)
    mode = getattr(enkf, MODES[args.mode])
    refine = args.refine and args.mode != "fp32"
    plan = enkf.Plan(NSTATE, NOBS, NENS, mode, panel_b=args.panel_b if args.mode != "fp32" else 0,
                     flags=enkf.ENKF_FLAG_REFINE if refine else 0, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        plan.obs_prep(STRIDE, 0, None, dX, V)
        plan.analysis(r, V, D, dXB=dX, XB=XB, XA=XA, Z=Z, M=M)

    for _ in range(args.warmup):
        step()
    barrier()
    inf = plan.analysis(r, V, D, dXB=dX, XB=XB, XA=XA, Z=Z, M=M, info=True)   # status check, untimed
    enkf.enkf_ism_profile(plan.handle, True)
    barrier()
    with ClockSampler(local) as clk:
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        barrier()
    t_ms = ev0.elapsed_time(ev1)
    phases = enkf.enkf_ism_profile_read(plan.handle)
    enkf.enkf_ism_profile(plan.handle, False)
    t_max, value = aggregate_ranks(t_ms, args.steps, world, dev)

    # end to end through the API with host buffers, pipelined as a serving loop would run it: two
    # sets of device buffers; step i's inputs -- the background ensemble X_B, the perturbed
    # observations Y and the variances, what a filter hands the analysis -- are copied in on one
    # stream while step i-1 computes, and step i-2's X_A is copied out on another.  The prep forms
    # the mean, the deviations, V and D = Y - H X_B on the device (enkf_inflate_prep with alpha = 1:
    # the centering prep whose FP32 form sums the members in compensated FP32).
    # Every step copies all of its inputs in from pinned host memory and its X_A out inside the
    # timed region.
    e2e_ms = float("nan")
    h2d = d2h = 0
    if not args.no_e2e:
        h_XB = h_dX.clone().pin_memory()
        # Y = D + H X_B (FP32 on the host, once), so that the device's D = Y - H X_B is the workload's
        h_Y = (h_D + h_XB[:, ::STRIDE][:, :NOBS]).contiguous().pin_memory()
        h_XA = [torch.empty(XA.shape, dtype=XA.dtype).pin_memory() for _ in range(2)]
        Ybufs = [torch.empty_like(D), torch.empty_like(D)]
        # two buffer sets of their own (the timed step's inputs stay as they are for the comparison)
        bufs = [(torch.empty_like(dX), torch.empty_like(XB), torch.empty_like(D), torch.empty_like(r),
                 torch.empty_like(XA)) for _ in range(2)]
        s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        e2e_steps = max(2, min(args.steps, 10))

        def e2e_run(nsteps):
            ev_in = [torch.cuda.Event() for _ in range(2)]
            ev_done = [torch.cuda.Event() for _ in range(2)]
            ev_out = [torch.cuda.Event() for _ in range(2)]
            start = torch.cuda.Event()
            start.record(stream)
            s_in.wait_event(start)
            for i in range(nsteps):
                b = i & 1
                bdX, bXB, bD, br, bXA = bufs[b]
                bY = Ybufs[b]
                with torch.cuda.stream(s_in):
                    if i >= 2:
                        s_in.wait_event(ev_done[b])      # step i-2 no longer reads these inputs
                    bXB.copy_(h_XB, non_blocking=True)
                    bY.copy_(h_Y, non_blocking=True)
                    br.copy_(h_r, non_blocking=True)
                    ev_in[b].record(s_in)
                stream.wait_event(ev_in[b])
                if i >= 2:
                    stream.wait_event(ev_out[b])         # step i-2's X_A has left this buffer
                # the centering prep (FP32 storage: compensated FP32 member sums) with alpha = 1
                enkf.enkf_inflate_prep(STRIDE, 1.0, bXB, V, dXB=bdX, Y=bY, D=bD)
                plan.analysis(br, V, bD, dXB=bdX, XB=bXB, XA=bXA, Z=Z, M=M)
                ev_done[b].record(stream)
                with torch.cuda.stream(s_out):
                    s_out.wait_event(ev_done[b])
                    h_XA[b].copy_(bXA, non_blocking=True)
                    ev_out[b].record(s_out)
            for b in range(min(2, nsteps)):
                stream.wait_event(ev_out[b])

        e2e_run(2)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e2e_run(e2e_steps)
        e1.record(stream)
        barrier()
        e2e_ms = e0.elapsed_time(e1) / e2e_steps
        h2d = (h_XB.numel() + h_Y.numel() + h_r.numel()) * 4
        d2h = h_XA[0].numel() * 4
        del h_XA, h_XB, h_Y, bufs, Ybufs
        # the timed step's outputs again, for the comparison below
        step()
        barrier()

    # plain FP64 comparator on the same values (fewer steps: it is FP64-ALU bound), and the
    # errors of this path against it on every result
    fp64 = None
    if not args.no_fp64:
        dX64 = dX.double()
        D64 = D.double()
        r64 = r.double()
        V64 = torch.empty(NENS, NOBS, dtype=torch.float64, device=dev)
        Z64 = torch.empty(NENS, NOBS, dtype=torch.float64, device=dev)
        XA64 = torch.empty_like(dX64)
        M64 = torch.empty(NENS * NENS, dtype=torch.float64, device=dev)
        plan64 = enkf.Plan(NSTATE, NOBS, NENS, enkf.ENKF_FP64, device=dev)

        def step64():
            plan64.obs_prep(STRIDE, 0, None, dX64, V64)
            plan64.analysis(r64, V64, D64, dXB=dX64, XB=dX64, XA=XA64, Z=Z64, M=M64)

        step64()
        barrier()
        k64 = max(1, min(args.steps, 3))
        enkf.enkf_ism_profile(plan64.handle, True)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(k64):
            step64()
        f1.record(stream)
        barrier()
        ph64 = enkf.enkf_ism_profile_read(plan64.handle)
        ms64 = f0.elapsed_time(f1) / k64

        def relerr(a, b):
            return float(torch.linalg.norm(a.double() - b) / torch.linalg.norm(b))

        errs = {"Z": relerr(Z, Z64), "M": relerr(M, M64), "XA": relerr(XA, XA64),
                "increment": relerr(XA.double() - dX64, XA64 - dX64)}
        lv64 = ph64.get("ism_solve", (float("nan"), 1))
        lv64_ms = lv64[0] / max(lv64[1], 1)
        f_solve = 6 * NOBS * NENS ** 2 + 3 * NOBS * NENS
        fp64 = {"path": "plain FP64 level-streaming", "ms_per_step": ms64, "analyses_per_s": 1e3 / ms64,
                "speedup_over_fp64": ms64 / (t_max / args.steps),
                "rel_err_vs_fp64": errs, "meets_1e-5_on_every_result": all(v <= 1e-5 for v in errs.values()),
                "solve_roofline": {"kernel": "ism_levels_kernel<double,2>", "bound": "alu",
                                   "achieved": f_solve / (lv64_ms / 1e3) / 1e12, "peak": peaks["fp64_tflops"],
                                   "unit": "TFLOP/s",
                                   "frac": f_solve / (lv64_ms / 1e3) / 1e12 / peaks["fp64_tflops"],
                                   "peak_kind": "measured (FP64 FMA microbenchmark)", "avg_launch_ms": lv64_ms}}
        plan64.close()
        del dX64, D64, r64, V64, Z64, XA64, M64

    if rank != 0:
        return
    peak, peak_kind = read_peaks()
    lv_ms, lv_n = phases.get("ism_solve", (float("nan"), 0))
    lv_avg = lv_ms / max(lv_n, 1)
    src_dir = os.path.join(ROOT, "paper_1302_3876_gb300", "csrc")
    f_solve = 6 * NOBS * NENS ** 2 + 3 * NOBS * NENS
    fp32_peak = peaks["fp32_tflops"]
    fp32_kind = f"measured (FP32 FMA microbenchmark, {peaks['how']})"
    if args.mode == "fp32":
        lb = level_bytes(NOBS, NENS, 4)
        achieved = lb / (lv_avg / 1e3) / 1e9
        roofline = {"kernel": "ism_levels_kernel<float,4>", "bound": "hbm", "achieved": achieved, "peak": peak,
                    "unit": "GB/s", "frac": achieved / peak, "peak_kind": f"{peak_kind} (MEASURED_PEAKS hbm_gbs)",
                    "algorithmic_bytes_per_launch": lb, "avg_launch_ms": lv_avg,
                    "traffic": profile_traffic(os.path.join(src_dir, "ism_stream.cu"),
                                               f"ism_levels_{args.workload}_fp32.md")}
    elif args.mode == "bf16x3" and "panel_kernel" in phases:
        # the tcgen05 panel kernel alone (phase 6: CUDA events around its launch inside the step)
        k_ms, k_n = phases["panel_kernel"]
        k_avg = k_ms / max(k_n, 1)
        pb = panel_bytes(NOBS, NENS, args.panel_b, 4)
        achieved = pb / (k_avg / 1e3) / 1e9
        bf16_sus = read_bf16_sustained()
        t_flops = 6 * f_solve      # six BF16 products per FP32 multiply-add of the trailing update and dots
        roofline = {"kernel": "ism_panel_tc05_kernel", "bound": "hbm", "achieved": achieved, "peak": peak,
                    "unit": "GB/s", "frac": achieved / peak, "peak_kind": f"{peak_kind} (MEASURED_PEAKS hbm_gbs)",
                    "algorithmic_bytes_per_launch": pb, "avg_launch_ms": k_avg,
                    "tensor_view": {"tensor_flops_per_launch": t_flops,
                                    "achieved_tflops": t_flops / (k_avg / 1e3) / 1e12,
                                    "peak_tflops": bf16_sus,
                                    "frac": t_flops / (k_avg / 1e3) / 1e12 / bf16_sus,
                                    "peak_kind": "measured (MEASURED_PEAKS bf16_tflops_sustained: the kernel is "
                                                 "timed inside a long step)"},
                    "traffic": profile_traffic(os.path.join(src_dir, "ism_panel_tc05.cu"),
                                               f"ism_panel_tc05_{args.workload}.md")}
        if "correction_kernel" in phases:
            c_ms, c_n = phases["correction_kernel"]
            c_avg = c_ms / max(c_n, 1)
            cb = correction_bytes(NOBS, NENS, args.panel_b, 4)
            roofline["correction_launch"] = {
                "kernel": "ism_panel_tc05_kernel (correction sweep)", "algorithmic_bytes_per_launch": cb,
                "avg_launch_ms": c_avg, "achieved_gbs": cb / (c_avg / 1e3) / 1e9,
                "frac": cb / (c_avg / 1e3) / 1e9 / peak}
    elif args.mode in ("bf16", "fp16", "bf16x3"):
        pb = panel_bytes(NOBS, NENS, args.panel_b, 4)
        achieved = pb / (lv_avg / 1e3) / 1e9
        mult = {"bf16": 3, "fp16": 1, "bf16x3": 6}[args.mode]   # tensor products per operand pair
        bf16_peak = read_bf16_peak()
        roofline = {"kernel": "ism_panel_kernel<%d>" % {"bf16": 1, "fp16": 2, "bf16x3": 3}[args.mode], "bound": "hbm",
                    "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "peak_kind": f"{peak_kind} (MEASURED_PEAKS hbm_gbs)", "algorithmic_bytes_per_launch": pb,
                    "avg_launch_ms": lv_avg,
                    "tensor_view": {"tensor_flops_per_launch": mult * f_solve,
                                    "achieved_tflops": mult * f_solve / (lv_avg / 1e3) / 1e12,
                                    "peak_tflops": bf16_peak,
                                    "frac": mult * f_solve / (lv_avg / 1e3) / 1e12 / bf16_peak,
                                    "note": "mma.sync m16n8k16; fp16 and bf16 share the dense peak"},
                    "traffic": profile_traffic(os.path.join(src_dir, "ism_panel.cu"),
                                               f"ism_panel_{args.workload}_{args.mode}.md")}
    else:
        achieved = f_solve / (lv_avg / 1e3) / 1e12
        pb = panel_bytes(NOBS, NENS, args.panel_b, 4)
        roofline = {"kernel": "ism_panel_kernel<0>", "bound": "alu", "achieved": achieved, "peak": fp32_peak,
                    "unit": "TFLOP/s", "frac": achieved / fp32_peak, "peak_kind": fp32_kind,
                    "algorithmic_flops_per_launch": f_solve, "avg_launch_ms": lv_avg,
                    "hbm_view": {"algorithmic_bytes_per_launch": pb, "achieved_gbs": pb / (lv_avg / 1e3) / 1e9,
                                 "peak_gbs": peak, "frac": pb / (lv_avg / 1e3) / 1e9 / peak},
                    "traffic": profile_traffic(os.path.join(src_dir, "ism_panel.cu"),
                                               f"ism_panel_{args.workload}_fp32.md")}
    inner = ("panel_kernel", "correction_kernel")      # kernels timed inside other phases
    total_ms = sum(v[0] for k, v in phases.items() if k not in inner)
    ms_step = t_max / args.steps
    # library kernels per step: the prep; the solve (Step 1 and the panel kernel on the tcgen05
    # path); without refinement the Gram, the assembly of M, the split images of M and X_A; with
    # it the Gram of V and U, P, the residual (prep, -P, images, X_A-type product), the
    # correction, V^T delta (the identity on the tcgen05 path, a Gram elsewhere), the update of
    # Z and M, and X_A (an exact Gram of V and Z1 for FP16 instead of P)
    tc5_path = args.mode == "bf16x3" and args.panel_b == 32
    solve_launches = 2 if tc5_path else 1
    if not refine:
        after = 5
    elif args.mode == "fp16":
        after = 14
    else:
        after = 12 if tc5_path else 13
    launches = 1 + solve_launches + after
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nstate": NSTATE, "nobs": NOBS, "nens": NENS,
                   "path": PATH_NAME[args.mode] % args.panel_b if "%" in PATH_NAME[args.mode] else
                   PATH_NAME[args.mode],
                   "refine": refine,
                   "x_b": "a buffer of its own (values equal to dX_B)",
                   "l2": "inputs > L2 (129 MB); no flush", "parallelism": f"replicas x{world}"},
        "gflops": flops(NSTATE, NOBS, NENS) / (ms_step / 1e3) / 1e9,
        "gamma_min": inf.gamma_min, "gamma_max": inf.gamma_max,
        "roofline": roofline,
        "measured_peaks": {"fp32_tflops": peaks["fp32_tflops"], "fp64_tflops": peaks["fp64_tflops"],
                           "sm_mhz_during": peaks["sm_mhz"], "hbm_gbs": peak,
                           "bf16_tflops": read_bf16_peak(), "how": peaks["how"]},
        "phases_ms_per_step": {k: v[0] / max(v[1], 1) for k, v in phases.items()},
        "phase_share": {k: v[0] / total_ms for k, v in phases.items() if k not in inner} if total_ms > 0 else {},
        "e2e": None if args.no_e2e else {
            "value": world / (e2e_ms / 1e3), "unit": METRIC, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
            "note": "pinned host buffers; copies in (X_B, the perturbed observations Y, r; the prep forms "
                    "the mean, dX_B, V and D = Y - H X_B on the device), compute and the copy out of X_A of "
                    "consecutive steps overlap on three streams (two device buffer sets)"},
        "gpu_launches": launches * args.steps,
        "clocks": clk.summary(),
        "comparator_fp64": fp64,
        "cpu_baseline": cpu and {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")},
    }
    print(json.dumps(line), flush=True)
    plan.close()


# ---------------------------------------------------------------------------
# Other workloads (not the default line): the panel workload, the batched
# workload, the Lorenz-96 cycle with the learned surrogate, and the next rows.
# ---------------------------------------------------------------------------

def _events_ms(fn, k):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(k):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / k


def run_panel_single(args):
    """Nstate = 2^22, Nobs = 2^20 (every 4th), Nens = 256: the tensor-core panel forms (split BF16 and
    FP16, each also with one refinement step; three-piece BF16), the FP32-core panel form, and the plain
    FP64 path."""
    import numpy as np
    import torch
    import synth
    from paper_1302_3876_gb300 import enkf
    enkf.load(build_if_missing=True)
    nstate, nobs, nens = 1 << 22, 1 << 20, 256
    w = synth.panel_single(dtype=np.float32)
    dev = torch.device("cuda")
    dX = torch.from_numpy(w["dXB"]).to(dev)
    D = torch.from_numpy(w["D"]).to(dev)
    r = torch.from_numpy(w["r"]).to(dev)
    del w
    V = torch.empty(nens, nobs, device=dev)
    XA = torch.empty_like(dX)
    Mo = torch.empty(nens * nens, device=dev)
    results = {}
    outs = {}
    for name, mode, flags in (("bf16+refine", enkf.ENKF_PANEL_BF16, enkf.ENKF_FLAG_REFINE),
                              ("fp16+refine", enkf.ENKF_PANEL_FP16, enkf.ENKF_FLAG_REFINE),
                              ("bf16", enkf.ENKF_PANEL_BF16, 0), ("bf16x3", enkf.ENKF_PANEL_BF16X3, 0),
                              ("panel32", enkf.ENKF_PANEL_FP32, 0)):
        plan = enkf.Plan(nstate, nobs, nens, mode, flags=flags, device=dev)

        def step():
            plan.obs_prep(4, 0, None, dX, V)
            plan.analysis(r, V, D, dXB=dX, XB=dX, XA=XA, M=Mo)

        for _ in range(args.warmup):
            step()
        enkf.enkf_ism_profile(plan.handle, True)
        ms = _events_ms(step, args.steps)
        ph = enkf.enkf_ism_profile_read(plan.handle)
        results[name] = {"ms_per_step": ms, "analyses_per_s": 1e3 / ms,
                         "phases_ms": {k: v[0] / max(v[1], 1) for k, v in ph.items()}}
        outs[name] = (XA.clone(), Mo.clone())
        plan.close()
    ref64 = None
    if not args.no_fp64:
        dX64, D64, r64 = dX.double(), D.double(), r.double()
        V64 = torch.empty(nens, nobs, dtype=torch.float64, device=dev)
        XA64 = torch.empty_like(dX64)
        M64 = torch.empty(nens * nens, dtype=torch.float64, device=dev)
        plan = enkf.Plan(nstate, nobs, nens, enkf.ENKF_FP64, device=dev)

        def step64():
            plan.obs_prep(4, 0, None, dX64, V64)
            plan.analysis(r64, V64, D64, dXB=dX64, XB=dX64, XA=XA64, M=M64)

        step64()
        ms64 = _events_ms(step64, 1)
        results["fp64_plain"] = {"ms_per_step": ms64, "analyses_per_s": 1e3 / ms64}
        for name, (xa, mo) in outs.items():
            results[name]["rel_err_vs_fp64"] = {
                "XA": float(torch.linalg.norm(xa.double() - XA64) / torch.linalg.norm(XA64)),
                "increment": float(torch.linalg.norm(xa.double() - XA64) / torch.linalg.norm(XA64 - dX64)),
                "M": float(torch.linalg.norm(mo.double() - M64) / torch.linalg.norm(M64))}
            results[name]["speedup_over_fp64_plain"] = ms64 / results[name]["ms_per_step"]
        plan.close()
        ref64 = ms64
    best = min((v["ms_per_step"], k) for k, v in results.items() if k != "fp64_plain"
               and v.get("rel_err_vs_fp64", {"XA": 0})["XA"] <= 1e-5)
    print(json.dumps({"metric": METRIC, "workload": f"panel_single Nstate={nstate} Nobs={nobs} Nens={nens}",
                      "value": 1e3 / best[0], "unit": METRIC, "best_path_at_1e-5": best[1],
                      "fp64_plain_ms": ref64, "paths": results, "data": "synthetic"}), flush=True)


def run_lorenz_small(args):
    """Lorenz-96 Nstate = 40, F = 8, truth spun up 1000 RK4 steps (dt 0.01) on the device, 20 members
    = truth + N(0, 0.1^2), every 2nd variable observed with R = 0.01 I and perturbed observations;
    the plain FP64 path (obs-space prep with centering, then the analysis).  Latency-bound: one call
    timed alone (median of 1000, CUDA events), 10^4 calls replayed from a captured CUDA graph, and the
    FP64 oracle on one host core (median of 1000)."""
    os.environ["OMP_NUM_THREADS"] = "1"     # the oracle's timing is on one core
    import numpy as np
    import torch
    import synth
    from paper_1302_3876_gb300 import enkf
    enkf.load(build_if_missing=True)
    dev = torch.device("cuda")
    d = synth.lorenz_small_draws()
    nstate, nobs, nens, stride = d["nstate"], d["nobs"], d["nens"], d["obs_stride"]
    truth = torch.from_numpy(d["truth0"].copy()).to(dev).reshape(1, nstate)
    enkf.enkf_forecast(truth, d["F"], 0.01, 1000)                       # spin-up on the device (RK4)
    XB = (truth + torch.from_numpy(d["ens_noise"]).to(dev)).contiguous()
    Y = ((truth[0, ::stride] + torch.from_numpy(d["obs_noise"]).to(dev))[None, :]
         + torch.from_numpy(d["pert"]).to(dev)).contiguous()
    r = torch.full((nobs,), d["r"], dtype=torch.float64, device=dev)
    dX = torch.empty_like(XB)
    V = torch.empty(nens, nobs, dtype=torch.float64, device=dev)
    D = torch.empty_like(V)
    XA = torch.empty_like(XB)
    plan = enkf.Plan(nstate, nobs, nens, enkf.ENKF_FP64, device=dev)
    stream = torch.cuda.current_stream()

    def call():
        plan.obs_prep(stride, 1, XB, dX, V, Y=Y, D=D)
        plan.analysis(r, V, D, dXB=dX, XB=XB, XA=XA)

    for _ in range(max(args.warmup, 3)):
        call()
    inf = plan.analysis(r, V, D, dXB=dX, XB=XB, XA=XA, info=True)
    assert inf.status == 0
    ref = XA.clone()
    # (a) one call at a time
    single = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(1000):
        e0.record(stream)
        call()
        e1.record(stream)
        e1.synchronize()
        single.append(e0.elapsed_time(e1))
    t_single = statistics.median(single)
    # (b) 10^4 calls replayed from a CUDA graph of one call
    plan.analysis(r, V, D, dXB=dX, XB=XB, XA=XA, info=True)           # nothing pending at capture
    g = torch.cuda.CUDAGraph()
    s_cap = torch.cuda.Stream()
    s_cap.wait_stream(stream)
    with torch.cuda.stream(s_cap):
        with torch.cuda.graph(g, stream=s_cap):
            call()
    stream.wait_stream(s_cap)
    nrep = 10000
    for _ in range(10):
        g.replay()
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        e0.record(stream)
        for _ in range(nrep):
            g.replay()
        e1.record(stream)
        torch.cuda.synchronize()
    t_graph = e0.elapsed_time(e1) / nrep
    inf = plan.analysis(r, V, D, dXB=dX, XB=XB, XA=XA, info=True)
    assert inf.status == 0 and torch.equal(XA, ref)
    plan.close()
    # FP64 oracle on one host core, same values
    import oracle
    XBh, Yh = XB.cpu().numpy().astype(np.float64), Y.cpu().numpy().astype(np.float64)
    rh = np.full(nobs, d["r"])

    def oracle_call():
        _, dXo = oracle.ensemble_deviations(XBh)
        Vo = oracle.observe_deviations(dXo, nobs, stride)
        Do = oracle.innovations(Yh, XBh, stride)
        return oracle.analysis(rh, Vo, Do, XBh, dXo, refine=False)     # the paper's steps: one solve

    oracle_call()
    t_or = []
    for _ in range(1000):
        t0 = time.perf_counter()
        out = oracle_call()
        t_or.append(time.perf_counter() - t0)
    t_oracle = statistics.median(t_or)
    err = float(np.linalg.norm(ref.cpu().numpy() - out["XA"]) / np.linalg.norm(out["XA"]))
    print(json.dumps({
        "metric": METRIC, "workload": f"lorenz_small Nstate={nstate} Nobs={nobs} Nens={nens} (plain FP64 path)",
        "value": 1e3 / t_graph, "unit": METRIC, "dtype": "f64", "data": "synthetic",
        "single_call": {"analyses_per_s": 1e3 / t_single, "latency_us": 1e3 * t_single,
                        "how": "median of 1000 calls, CUDA events around obs prep + analysis, synchronised"},
        "graph_replay": {"analyses_per_s": 1e3 / t_graph, "latency_us": 1e3 * t_graph, "calls": nrep,
                         "how": "one call (obs prep + analysis) captured in a CUDA graph, replayed back to back"},
        "gpu_launches_per_analysis": 2,
        "kernels_per_analysis": ["center_observe_kernel<double>",
                                 "small_analysis_kernel<double> (Step 1, Step 2, M and X_A in one CTA)"],
        "clocks": clk.summary(),
        "rel_err_XA_vs_oracle": err,
        "cpu_baseline": {"value": 1.0 / t_oracle, "unit": METRIC, "cores": 1, "kind": "oracle",
                         "sample": "the same analysis (prep included), median of 1000 calls"},
    }), flush=True)


def run_batch_local(args):
    """8192 independent problems (Nobs log-uniform in [16, 4096], Nens in {32,64,96,128}) in one persistent
    launch replayed from a CUDA graph, panel widths autotuned; plain FP64 path per problem on a sample."""
    import numpy as np
    import torch
    import synth
    from paper_1302_3876_gb300 import enkf
    enkf.load(build_if_missing=True)
    base, descs, nout = synth.batch_local_packed(8192)
    dev = torch.device("cuda")
    fp32_peak = measure_fma_peaks(dev, 0)["fp32_tflops"]
    tin = torch.from_numpy(base).to(dev)
    tout = torch.empty(nout, device=dev)
    plan, wsb = enkf.enkf_ism_batch_plan(descs)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    widths = enkf.enkf_ism_batch_autotune(plan, tin, tout, ws)
    for _ in range(args.warmup):
        enkf.enkf_ism_batch(plan, tin, tout, ws)
    ms = _events_ms(lambda: enkf.enkf_ism_batch(plan, tin, tout, ws), args.steps)
    enkf.enkf_ism_batch_plan_destroy(plan)
    flops = sum(6 * d["nobs"] * d["nens"] ** 2 + 3 * d["nobs"] * d["nens"] + 2 * d["nobs"] * d["nens"] ** 2
                for d in descs)
    # plain FP64 comparator on every 32nd problem, scaled by 32
    sample = descs[::32]
    t64 = 0.0
    for d in sample:
        n, N = d["nobs"], d["nens"]
        V = tin[d["V"]:d["V"] + n * N].view(N, n).double()
        Dm = tin[d["D"]:d["D"] + n * N].view(N, n).double()
        rr = tin[d["r"]:d["r"] + n].double()
        Z = torch.empty_like(Dm)
        Mm = torch.empty(N * N, dtype=torch.float64, device=dev)
        p = enkf.Plan(1, n, N, enkf.ENKF_FP64, device=dev)
        p.analysis(rr, V, Dm, Z=Z, M=Mm)
        t64 += _events_ms(lambda: p.analysis(rr, V, Dm, Z=Z, M=Mm), 1)
        p.close()
    ms64 = t64 * len(descs) / len(sample)
    print(json.dumps({"metric": "problems/s", "workload": "batch_local 8192 problems", "value": 8192 / (ms / 1e3),
                      "unit": "problems/s", "ms_per_batch": ms, "gflops": flops / (ms / 1e3) / 1e9,
                      "fp32_alu_frac": flops / (ms / 1e3) / 1e12 / fp32_peak,
                      "fp32_peak_tflops": fp32_peak, "fp32_peak_kind": "measured (FP32 FMA microbenchmark)",
                      "widths_per_class": widths,
                      "fp64_plain_per_problem_ms_est": ms64,
                      "speedup_over_fp64_plain": ms64 / ms, "data": "synthetic"}), flush=True)


def run_lorenz_cycle(args):
    """Lorenz-96 Nstate=4096, Nens=256, 200 cycles of 5 RK4 steps, every 2nd variable observed, R = 0.25 I:
    the filter with RK4, with the learned surrogate (trained on filter trajectories of a separate seed), and
    with persistence."""
    import torch
    from paper_1302_3876_gb300 import cycle as C
    from paper_1302_3876_gb300 import enkf
    enkf.load(build_if_missing=True)
    t0 = time.perf_counter()
    train = C.LorenzCycle(4096, 256, seed=555)
    pairs = []
    train.run(args.train_cycles, "rk4", collect=pairs)
    xs = torch.cat([a for a, _ in pairs]).contiguous()
    ys = torch.cat([b for _, b in pairs]).contiguous()
    train.close()
    del pairs
    ts = time.perf_counter()
    master, packed, log = C.train_surrogate(xs, ys, steps=args.train_steps, batch=16, lr=2e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - ts
    out = {}
    for method in ("rk4", "surrogate", "persistence"):
        cyc = C.LorenzCycle(4096, 256)
        if method == "surrogate":
            cyc.set_surrogate(packed)
        rmse, cps, per_cycle = cyc.run(200, method)
        # the time mean over all 200 cycles is that of a filter that has lost the truth (no inflation);
        # the first 8 cycles are where the RK4 filter still tracks it
        out[method] = {"analysis_rmse": rmse, "cycles_per_s": cps,
                       "analysis_rmse_first_8_cycles": float(sum(per_cycle[:8]) / 8),
                       "per_cycle_rmse_first_8": [round(v, 4) for v in per_cycle[:8]]}
        cyc.close()
    # forecast-only timing of the two models on the same ensemble
    cyc = C.LorenzCycle(4096, 256)
    cyc.set_surrogate(packed)
    X = cyc.X
    rk = _events_ms(lambda: enkf.enkf_forecast(X, 8.0, 0.01, 5), 20)
    sg = _events_ms(lambda: enkf.enkf_forecast(X, 8.0, 0.01, 1, method=enkf.ENKF_FORECAST_SURROGATE,
                                               weights=packed, workspace=cyc.sur_ws), 20)
    cyc.close()
    print(json.dumps({"metric": "cycles/s", "workload": "lorenz_cycle Nstate=4096 Nens=256, 200 cycles",
                      "value": out["surrogate"]["cycles_per_s"], "unit": "cycles/s", "methods": out,
                      "forecast_ms": {"rk4_5_steps": rk, "surrogate": sg,
                                      "surrogate_tflops": 2 * 4096 * 256 * 41600 / (sg / 1e3) / 1e12},
                      "training": {"pairs": int(xs.shape[0]), "steps": args.train_steps, "seconds": train_s,
                                   "mse_log": log[-3:]},
                      "wall_s": time.perf_counter() - t0, "data": "synthetic"}), flush=True)


def run_next_rows(args):
    """The rows beside the analysis, each timed by CUDA events on its own and set against its roofline:
    inflation fused into the prep (Nstate 2^21, every 4th variable observed, 128 members, FP32), partial
    localization (the Lorenz-96 cycle size Nstate 4096 / Nobs 2048 / 256 members with the paper's weights
    exp(-d / Nstate), and a 64-point cut-off at Nstate 2^21 / Nobs 2^19 / 128 members), the block-diagonal
    R path (32 x 32 blocks at Nobs 2^19, 128 members: whitening, analysis with r = 1, unwhitening), the
    pivoted solve, one rank's share of the row-sharded analysis (the panel workload split over 8 ranks),
    and the Lorenz-96 filter with inflation and localization against the unlocalized filter (analysis RMSE)."""
    import torch
    import synth
    from paper_1302_3876_gb300 import cycle as C
    from paper_1302_3876_gb300 import enkf
    enkf.load(build_if_missing=True)
    hbm, hbm_src = read_peaks()
    dev = torch.device("cuda")
    fp32 = measure_fma_peaks(dev, 0)["fp32_tflops"]
    gen = torch.Generator(device=dev)
    gen.manual_seed(synth.seed_for("next_rows"))
    k = max(3, min(args.steps, 50))
    out = {}
    part = args.next_part

    if part in ("all", "inflate"):
        nstate, nobs, nens, stride = NSTATE, NOBS, NENS, STRIDE
        X = torch.randn(nens, nstate, device=dev, generator=gen) + 8.0
        Y = torch.randn(nens, nobs, device=dev, generator=gen) + 8.0
        dX, V, D = torch.empty_like(X), torch.empty(nens, nobs, device=dev), torch.empty(nens, nobs, device=dev)
        fn = lambda: enkf.enkf_inflate_prep(stride, 1.01, X, V, dXB=dX, Y=Y, D=D)  # noqa: E731
        for _ in range(args.warmup):
            fn()
        ms = _events_ms(fn, k)
        nbytes = 4 * nens * (3 * nstate + 3 * nobs)    # X_B read and written, dX_B written; Y read, V and D written
        out["inflate_prep"] = {"config": f"Nstate={nstate} Nobs={nobs} Nens={nens} FP32", "ms": ms,
                               "roofline": {"bound": "hbm", "achieved": nbytes / (ms / 1e3) / 1e9, "peak": hbm,
                                            "unit": "GB/s", "frac": nbytes / (ms / 1e3) / 1e9 / hbm,
                                            "peak_source": hbm_src, "bytes": nbytes}}
        del X, Y, dX, V, D

    if part in ("all", "localize"):
        cases = [("lorenz_cycle_paper_weights", 4096, 2, 256, 4096.0, None, torch.float32),
                 ("lorenz_cycle_paper_weights_fp64", 4096, 2, 256, 4096.0, None, torch.float64),
                 ("large_cutoff64", NSTATE, STRIDE, NENS, 32.0, 64.0, torch.float32)]
        for name, nstate, stride, nens, length, radius, dt in cases:
            nobs = (nstate - 1) // stride + 1
            dX = torch.randn(nens, nstate, device=dev, generator=gen, dtype=dt)
            XB = dX + 8.0
            V = torch.randn(nens, nobs, device=dev, generator=gen, dtype=dt) / math.sqrt(nens - 1)
            Z = torch.randn(nens, nobs, device=dev, generator=gen, dtype=dt)
            XA = torch.empty_like(XB)
            fn = lambda: enkf.enkf_localized_update(stride, length, radius, dX, V, Z, XB, XA)  # noqa: E731
            for _ in range(args.warmup):
                fn()
            ms = _events_ms(fn, k)
            if radius is None:
                pairs = nstate * nobs
            else:
                pairs = nobs * min(nstate, 2 * int(math.floor(radius)) + 1)
            fl = 4 * nens * pairs                           # (S V^T) entry and its use in T Z: 2 N + 2 N flops
            nbytes = (4 if dt == torch.float32 else 8) * nens * (3 * nstate + 2 * nobs)
            peak = fp32 if dt == torch.float32 else None
            out["localized_update_" + name] = {
                "config": f"Nstate={nstate} Nobs={nobs} Nens={nens} length={length} radius={radius} "
                          f"{'FP32' if dt == torch.float32 else 'FP64'}",
                "ms": ms, "pairs": pairs, "gflop": fl / 1e9, "tflops": fl / (ms / 1e3) / 1e12,
                "roofline": {"bound": "alu", "achieved": fl / (ms / 1e3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                             "frac": (fl / (ms / 1e3) / 1e12 / peak) if peak else None,
                             "peak_source": "measured FP32 CUDA-core peak (FMA microbenchmark)" if peak else None},
                "hbm_gbs_compulsory": nbytes / (ms / 1e3) / 1e9}
            del dX, XB, V, Z, XA

    if part in ("all", "rblock"):
        nstate, nobs, nens, bs = NSTATE, NOBS, NENS, 32
        nblk = nobs // bs
        A = torch.randn(nblk, bs, bs, device=dev, generator=gen, dtype=torch.float64)
        R = A @ A.transpose(1, 2) / bs + torch.diag_embed(0.5 + torch.rand(nblk, bs, device=dev, generator=gen,
                                                                             dtype=torch.float64))
        L = torch.empty_like(R)
        enkf.enkf_rblock_factor(nobs, bs, R, L)
        dX = torch.randn(nens, nstate, device=dev, generator=gen)
        D0 = torch.randn(nens, nobs, device=dev, generator=gen)
        V, D, Z = torch.empty(nens, nobs, device=dev), torch.empty_like(D0), torch.empty_like(D0)
        XA = torch.empty_like(dX)
        ones = torch.ones(nobs, device=dev)
        plan = enkf.Plan(nstate, nobs, nens, enkf.ENKF_PANEL_FP32, panel_b=32, device=dev)
        phase = {}

        def step():
            plan.obs_prep(STRIDE, 0, None, dX, V)
            D.copy_(D0)
            enkf.enkf_rblock_whiten(bs, L, V, D)
            plan.analysis(ones, V, D, dXB=dX, XB=dX, XA=XA, Z=Z)
            enkf.enkf_rblock_unwhiten(bs, L, Z)

        for _ in range(args.warmup):
            step()
        ms = _events_ms(step, k)
        phase["whiten_ms"] = _events_ms(lambda: enkf.enkf_rblock_whiten(bs, L, V, D), k)
        phase["unwhiten_ms"] = _events_ms(lambda: enkf.enkf_rblock_unwhiten(bs, L, Z), k)
        plan.close()
        nb_w = 4 * 4 * nobs * nens                          # V and D read and written
        out["rblock_analysis"] = {
            "config": f"Nstate={nstate} Nobs={nobs} Nens={nens} blocks {bs}x{bs}, panel FP32 analysis",
            "ms_per_analysis": ms, "analyses_per_s": 1e3 / ms, **phase,
            "whiten_roofline": {"bound": "hbm", "achieved": nb_w / (phase["whiten_ms"] / 1e3) / 1e9, "peak": hbm,
                                "unit": "GB/s", "frac": nb_w / (phase["whiten_ms"] / 1e3) / 1e9 / hbm,
                                "fp64_gflop": nobs * 2 * nens * bs / 1e9}}
        del A, R, L, dX, D0, V, D, Z, XA

    if part in ("all", "pivot"):
        nobs, nens = 1 << 18, 64
        res = {}
        for name, dt, mode in (("fp32", torch.float32, enkf.ENKF_FP32), ("fp64", torch.float64, enkf.ENKF_FP64)):
            r = 0.5 + torch.rand(nobs, device=dev, generator=gen, dtype=dt)
            V = torch.randn(nens, nobs, device=dev, generator=gen, dtype=dt) / math.sqrt(nens - 1)
            D = torch.randn(nens, nobs, device=dev, generator=gen, dtype=dt)
            Z = torch.empty_like(D)
            M = torch.empty(nens * nens, device=dev, dtype=dt)
            ws = torch.empty(enkf.enkf_ism_pivot_workspace(nobs, nens, mode), dtype=torch.uint8, device=dev)
            fn = lambda: enkf.enkf_ism_solve_pivot(r, V, D, Z, ws, M=M, sync=False)  # noqa: E731
            for _ in range(args.warmup):
                fn()
            ms = _events_ms(fn, min(k, 10))
            plan = enkf.Plan(1, nobs, nens, mode, device=dev)
            fn0 = lambda: plan.analysis(r, V, D, Z=Z, M=M)  # noqa: E731
            for _ in range(args.warmup):
                fn0()
            ms0 = _events_ms(fn0, min(k, 10))
            plan.close()
            w = 4 if dt == torch.float32 else 8
            # per level: the dots pass reads v_p and the active columns, the update pass reads and
            # writes them and reads the remaining v_i (their dots for the next choice)
            nbytes = sum(w * nobs * (1 + (nens + nens - kk) + 2 * (nens + nens - kk - 1) + (nens - kk - 1))
                         for kk in range(nens))
            res[name] = {"ms_pivoted": ms, "ms_unpivoted_plain_path": ms0, "launches": 4 * nens + 4,
                         "roofline": {"bound": "hbm", "achieved": nbytes / (ms / 1e3) / 1e9, "peak": hbm,
                                      "unit": "GB/s", "frac": nbytes / (ms / 1e3) / 1e9 / hbm, "bytes": nbytes}}
            del r, V, D, Z, M, ws
        out["pivoted_solve"] = {"config": f"Nobs={nobs} Nens={nens}", "paths": res}

    if part in ("all", "rows"):
        # N-1: one rank's share of the row-sharded analysis, the panel workload split over 8 ranks by
        # observation rows (Nobs 2^17, Nstate 2^19, 256 members, FP32; inputs larger than L2).  One GPU
        # holds one rank here, so the exchange is the identity: the timed region is the rank's own work
        # (Step 1, one level pass per level, the Gram of the final columns, M, X_A and the status read),
        # without the collectives (2N doubles per level and one N x N Gram across the ranks).
        from paper_1302_3876_gb300 import sharded
        nobs, nens = (1 << 20) // 8, 256
        nstate = nobs * STRIDE
        r = 0.5 + torch.rand(nobs, device=dev, generator=gen)
        V = torch.randn(nens, nobs, device=dev, generator=gen) / math.sqrt(nens - 1)
        D = torch.randn(nens, nobs, device=dev, generator=gen)
        dX = torch.randn(nens, nstate, device=dev, generator=gen)
        XB = dX + 8.0
        XA = torch.empty_like(XB)
        fn = lambda: sharded.sharded_analysis(r, V, D, dX, XB, XA, lambda t: None)  # noqa: E731
        for _ in range(args.warmup):
            fn()
        ms = _events_ms(fn, min(k, 10))
        w = 4
        # Step 1 reads r, D and V and writes Z and U (and reads v_0); level k reads and writes the N
        # columns of Z and the N - k - 1 active columns of U, and reads u_k and v_{k+1}
        lvl = w * nobs * (4 * nens + 2) + sum(w * nobs * (2 * (2 * nens - kk - 1) + (2 if kk + 1 < nens else 1))
                                              for kk in range(nens))
        nbytes = lvl + 2 * w * nobs * nens + 3 * w * nstate * nens     # + the Gram's V and U, X_A's three arrays
        out["rows_block"] = {
            "config": f"one rank of 8: Nobs={nobs} Nstate={nstate} Nens={nens} FP32, exchange not timed",
            "ms_per_analysis": ms, "launches": 2 * nens + 5, "level_pass_bytes": lvl,
            "roofline": {"bound": "hbm", "achieved": nbytes / (ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": nbytes / (ms / 1e3) / 1e9 / hbm, "bytes": nbytes, "peak_source": hbm_src}}
        del r, V, D, dX, XB, XA

    if part in ("all", "cycle"):
        # partial localization leaves (R + V V^T)^{-1} unlocalized: with short correlation lengths the
        # cycle diverges (the analysis then reports ENKF_ERR_NUMERIC), which is recorded, not raised
        res = {}
        for name, kw in (("rk4", {}),
                         ("rk4_paper_localization", {"loc_length": 4096.0, "loc_radius": None}),
                         ("rk4_paper_localization_inflation1.02", {"loc_length": 4096.0, "loc_radius": None,
                                                                    "inflation": 1.02}),
                         ("rk4_localization_length64_radius128_inflation1.05",
                          {"loc_length": 64.0, "loc_radius": 128.0, "inflation": 1.05})):
            cyc = C.LorenzCycle(4096, 256, **kw)
            try:
                rmse, cps, _ = cyc.run(args.cycles, "rk4")
                res[name] = {"analysis_rmse": rmse, "cycles_per_s": cps}
            except enkf.EnkfError as e:
                torch.cuda.synchronize()
                res[name] = {"numeric_error_in_cycle": cyc.cycle_index, "status": enkf.status_name(e.status)}
            cyc.close()
        out["lorenz_cycle"] = {"config": f"Nstate=4096 Nens=256 Nobs=2048, {args.cycles} cycles of 5 RK4 steps",
                               "methods": res}

    print(json.dumps({"workload": "next_rows", "rows": out, "steps": k, "warmup": args.warmup,
                      "data": "synthetic"}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--mode", choices=["panel32", "bf16", "fp16", "bf16x3", "fp32"], default="bf16x3",
                    help="headline path: panel form on tcgen05 tensor cores with three-piece BF16 operands (bf16x3, "
                         "default), on FP32 CUDA cores (panel32), on mma.sync tensor cores with split BF16 (bf16) or "
                         "FP16 (fp16) operands, or the FP32 level-streaming path (fp32)")
    ap.add_argument("--panel-b", type=int, default=32)
    ap.add_argument("--refine", action=argparse.BooleanOptionalAction, default=True,
                    help="one step of iterative refinement (panel modes; on by default: the refined FP32 path is "
                         "the one that meets 1e-5 on Z, M, X_A and the increment)")
    ap.add_argument("--workload", choices=["panel_single", "large_single", "panel_paths", "lorenz_small",
                                           "batch_local", "lorenz_cycle", "next_rows"], default="panel_single")
    ap.add_argument("--next-part", choices=["all", "inflate", "localize", "rblock", "pivot", "rows", "cycle"],
                    default="all",
                    help="next_rows workload: run one part only")
    ap.add_argument("--cycles", type=int, default=200, help="next_rows workload: assimilation cycles per filter")
    ap.add_argument("--train-cycles", type=int, default=60)
    ap.add_argument("--train-steps", type=int, default=1500)
    ap.add_argument("--scale-div", type=int, default=1,
                    help="divide Nobs and Nstate by this factor (small case for profiler captures)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "panel_paths":
        run_panel_single(args)
    elif args.workload == "lorenz_small":
        run_lorenz_small(args)
    elif args.workload == "batch_local":
        run_batch_local(args)
    elif args.workload == "lorenz_cycle":
        run_lorenz_cycle(args)
    elif args.workload == "next_rows":
        run_next_rows(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
