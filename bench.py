#!/usr/bin/env python
"""Benchmark of the DuQuad GB300 library (one JSON line on rank 0).

Default workload: the single large dense QP (n=20000, p=10000, FP32 iterates,
FP64 constants and residuals, augmented ADFGM, last iterate and average,
eps=1e-3).  One step is one pass of the whole hot path on one synthetic
instance: problem handle over device-resident Q, G (transposed copy built),
FP64 power iteration for lambda_max(Q) and ||G||^2, the full DFOM solve with
its inner FGM loop, stopping certificates and FP64 residuals.

  value    solves/s with inputs already in HBM (CUDA events on the library's stream)
  e2e      solves/s through the C ABI from pinned host double arrays, the upload
           and the download of the outputs inside the timed region
  roofline the inner-iteration GEMV (the dominant kernel) timed live with CUDA
           events inside the library: algorithmic bytes / device time vs the
           measured HBM copy bandwidth
  cpu_baseline the FP64 oracle on the host cores on a bounded sample

Other workloads: --workload small (n=50 FP64 DFGM), uneven (10000 mixed QPs,
one persistent launch), mpc (16384 shared-matrix QPs), served (Poisson stream).
Multi-GPU: replicas only (independent instances per rank, no collectives).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "QP solves/s at eps=1e-3"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")


def load_peaks():
    try:
        with open(PEAKS) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ workloads

class LargeDense:
    """n=20000, p=10000 dense QP, FP32, ADFGM, last + average, eps = 1e-3."""

    name = "large_dense_n20000_p10000_fp32_adfgm"

    def __init__(self, args, device):
        import torch

        import workloads as W
        self.n, self.p = args.n, args.p
        self.alg = args.alg
        self.eps = args.eps
        self.dev = device
        d = W.large_dense(n=self.n, p=self.p, seed=1, device=f"cuda:{device}")
        self.d = d
        self.lmin = d["lmin_Q"]
        self.eps_in = args.eps_in
        self.check_every = args.check_every
        self.inner_check_every = args.inner_check_every
        self.h_inputs = None
        torch.cuda.synchronize()

    def opts(self, D):
        return D.opts(self.alg, eps_out=self.eps, eps_in=self.eps_in, check_every=self.check_every,
                      inner_check_every=self.inner_check_every, engine=D.ENGINE_GRID, max_outer=20000)

    def step_device(self, D, ctx, outs):
        d = self.d
        P = D.Problem(ctx, d["Q"], d["q"], d["G"], d["g"], d["lb"], d["ub"], prec=D.FP32, lmin_Q=self.lmin)
        res = P.solve(self.opts(D), device_out=outs)
        P.close()
        return res

    def host_inputs(self):
        import torch
        if self.h_inputs is None:
            self.h_inputs = {k: v.double().cpu().pin_memory() for k, v in self.d.items() if k != "lmin_Q"}
        return self.h_inputs

    def step_host(self, D, ctx):
        h = self.host_inputs()
        P = D.Problem(ctx, h["Q"], h["q"], h["G"], h["g"], h["lb"], h["ub"], prec=D.FP32, lmin_Q=self.lmin)
        out = P.solve(self.opts(D))
        P.close()
        return out

    def h2d_bytes(self):
        n, p = self.n, self.p
        return 8 * (n * n + p * n + 3 * n + p)

    def d2h_bytes(self):
        return 8 * (2 * self.n + self.p)


def run_gpu(args):
    import torch

    from paper_1504_05708_gb300 import duquad as D
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    wl = LargeDense(args, local)
    stream = torch.cuda.current_stream()
    ctx = D.Context(local, stream)
    n, p = wl.n, wl.p
    outs = (torch.empty(n, device="cuda"), torch.empty(n, device="cuda"), torch.empty(p, device="cuda"))

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up (also builds the kernels' caches)
    for _ in range(args.warmup):
        res = wl.step_device(D, ctx, outs)
    barrier()
    ctx.stats(reset=True)
    ctx.profile(True)
    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    results = []
    for _ in range(args.steps):
        results.append(wl.step_device(D, ctx, outs)[0])
    ev1.record(stream)
    barrier()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    st = ctx.stats(reset=True)
    ctx.profile(False)
    ms_max = ms
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_max = float(t.item())
    value = world * args.steps / (ms_max / 1e3)

    # end to end through the C ABI from pinned host memory
    e2e = None
    if not args.no_e2e:
        wl.host_inputs()
        barrier()
        t0 = time.perf_counter()
        for _ in range(max(1, min(args.steps, 2))):
            wl.step_host(D, ctx)
        barrier()
        e2e_s = (time.perf_counter() - t0) / max(1, min(args.steps, 2))
        e2e = {"value": world / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": wl.h2d_bytes(),
               "d2h_bytes_per_step": wl.d2h_bytes()}
    ctx.stats(reset=True)

    peaks, kind = load_peaks()
    achieved = st["gemv_bytes"] / (st["gemv_ms"] / 1e3) / 1e9 if st["gemv_ms"] > 0 else None
    r0 = results[-1]
    inner = statistics.mean(r.inner_iters for r in results)
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl.name, "n": n, "p": p, "alg": wl.alg, "eps": wl.eps,
                   "eps_in": wl.eps_in, "outputs": "last+average", "check_every": wl.check_every,
                   "inner_check_every": wl.inner_check_every,
                   "l2": "inputs larger than L2 (Q 1.6 GB, G 0.8 GB, G' 0.8 GB)",
                   "parallelism": f"replicas{world}"},
        "solve": {"status": r0.status, "outer_iters": r0.outer_iters, "inner_iters_mean": inner,
                  "f_last": r0.f_last, "infeas_last": r0.infeas_last, "f_avg": r0.f_avg,
                  "infeas_avg": r0.infeas_avg, "d_lb": r0.d_lb, "converged_last": r0.converged_last,
                  "converged_avg": r0.converged_avg},
        "roofline": {"kernel": "k_rows<float> inner-iteration GEMV", "bound": "hbm", "achieved": achieved,
                     "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": (achieved / peaks["hbm_gbs"]) if achieved else None, "traffic": None,
                     "peak_kind": kind, "launches_timed": st["gemv_launches"],
                     "gemv_share_of_step": (st["gemv_ms"] / ms) if ms > 0 else None},
        "gpu_launches": st["launches"],
        "clocks": clk,
        "e2e": e2e,
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_large(wl, inner, r0.outer_iters, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def cpu_baseline_large(wl, inner_per_solve, outer_per_solve, budget_s):
    """The FP64 oracle, single-threaded, on the same instance: time a bounded run of
    inner FOM iterations, scale by the GPU's iteration count per solve."""
    import numpy as np

    import oracle as O
    d = wl.d
    qp = O.QP(d["Q"].double().cpu().numpy(), d["q"].double().cpu().numpy(), d["G"].double().cpu().numpy(),
              d["g"].double().cpu().numpy(), d["lb"].double().cpu().numpy(), d["ub"].double().cpu().numpy())
    mu = np.zeros(wl.p)
    x0 = np.zeros(wl.n)
    rho = 1.0 / 3.0
    t0 = time.perf_counter()
    O.fom(qp, rho, mu, 6.0, 0.01, x0, fixed=1)
    t_step = time.perf_counter() - t0
    k = max(1, int(budget_s / max(t_step, 1e-9)) - 1)
    t0 = time.perf_counter()
    O.fom(qp, rho, mu, 6.0, 0.01, x0, fixed=k)
    t_step = (time.perf_counter() - t0) / k
    per_solve = t_step * inner_per_solve
    return {"value": 1.0 / per_solve, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": f"{k + 1} inner FOM iterations of the FP64 oracle on the same n={wl.n} instance "
                      f"({t_step:.3f} s each), scaled by the GPU run's {inner_per_solve:.0f} inner "
                      f"iterations per solve"}


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores, same metric and config."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    import numpy as np

    import oracle as O
    import workloads as W
    import torch
    d = W.large_dense(n=args.n, p=args.p, seed=1, device="cuda" if torch.cuda.is_available() else "cpu")
    qp = O.QP(*(d[k].double().cpu().numpy() for k in ("Q", "q", "G", "g", "lb", "ub")))
    del d
    mu, x0 = np.zeros(args.p), np.zeros(args.n)
    inner_per_solve = args.ref_inner_per_solve
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        O.fom(qp, 1.0 / 3.0, mu, 6.0, 0.01, x0, fixed=args.ref_inner_sample)
        dt = (time.perf_counter() - t0) / args.ref_inner_sample
        if s >= args.warmup:
            times.append(dt)
    t_step = statistics.mean(times)
    value = 1.0 / (t_step * inner_per_solve)
    sample = (f"{args.ref_inner_sample} inner FOM iterations per step of the FP64 oracle on the n={args.n}, "
              f"p={args.p} instance, scaled to a solve of {inner_per_solve} inner iterations")
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step * inner_per_solve * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": LargeDense.name, "n": args.n, "p": args.p, "alg": args.alg, "eps": args.eps},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=20000)
    ap.add_argument("--p", type=int, default=10000)
    ap.add_argument("--alg", default="ADFGM")
    ap.add_argument("--eps", type=float, default=1e-3)
    ap.add_argument("--eps-in", type=float, default=1e-5)
    ap.add_argument("--check-every", type=int, default=10)
    ap.add_argument("--inner-check-every", type=int, default=5)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-inner-sample", type=int, default=8)
    ap.add_argument("--ref-inner-per-solve", type=int, default=2000)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
