#!/usr/bin/env python
"""Benchmark of the DuQuad GB300 library (one JSON line on rank 0).

Default workload: the single large dense QP (n=20000, p=10000, FP32 iterates,
FP64 constants and residuals, augmented ADFGM, last iterate and average,
eps=1e-3).  One step is one pass of the whole hot path on one synthetic
instance: problem handle over device-resident Q, G (transposed copy built),
the Lanczos estimates of lambda_max(Q) and ||G||^2, the full DFOM solve with
its inner FGM loop, stopping certificates and FP64 residuals.

  value    solves/s with inputs already in HBM (CUDA events on the library's stream)
  e2e      solves/s through the C ABI from pinned host double arrays, the upload
           and the download of the outputs inside the timed region
  roofline the inner-iteration GEMV (the dominant kernel) timed live with CUDA
           events inside the library: algorithmic bytes / device time vs the
           measured HBM copy bandwidth
  cpu_baseline the FP64 oracle on the host cores on a bounded sample

Other workloads: --workload small (n=50 FP64 DFGM), uneven (10000 mixed QPs,
one persistent launch), mpc (16384 shared-matrix QPs), served (Poisson stream),
sweep (the paper's eps_in sensitivity and outer-iteration-count studies), sparse
(one CSR QP, n = 2e6, p = 1e6).
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
# DRAM bytes (read + write) per algorithmic byte of the large-dense kernels, each from one ncu
# capture (k_v2_pass at n = 12000, k_rows at n = 8192), applied to the full-size launches: both
# kernels read every matrix element once, so traffic grows in proportion to the bytes a launch
# processes
TRAFFIC_RATIO = {"k_v2_pass": 1.0068, "k_rows": 1.0115}
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


def replica_rate(ms_local, steps, world, device=None):
    """Replicas only: every rank times its own `steps` solves; the job's time is the
    maximum over ranks and its rate counts the solves of all ranks (weak scaling).
    Returns (ms_max, solves_per_s).  No data crosses ranks, only this one scalar."""
    ms_max = float(ms_local)
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms_max], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_max = float(t.item())
    return ms_max, world * steps / (ms_max / 1e3)


# ------------------------------------------------------------------ workloads

class LargeDense:
    """n=20000, p=10000 dense QP, FP32, ADFGM, last + average, eps = 1e-3."""

    name = "large_dense_n20000_p10000_fp32_adfgm"

    @staticmethod
    def workload_name(n, p, alg, equality=False):
        """The workload as named in the JSON line, with its actual sizes."""
        if equality:
            return f"large_dense_eq_n{n}_p{p}_fp32_{alg.lower()}_hessian"
        return f"large_dense_n{n}_p{p}_fp32_{alg.lower()}"

    def __init__(self, args, device, equality=False):
        import torch

        import workloads as W
        self.n, self.p = args.n, args.p
        self.alg = args.alg
        self.eps = args.eps
        self.dev = device
        self.equality = equality
        self.name = self.workload_name(self.n, self.p, self.alg, equality)
        d = W.large_dense(n=self.n, p=self.p, seed=1, device=f"cuda:{device}", equality=equality)
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
        P = D.Problem(ctx, d["Q"], d["q"], d["G"], d["g"], d["lb"], d["ub"], prec=D.FP32, lmin_Q=self.lmin,
                      cone=D.CONE_EQ if self.equality else D.CONE_INEQ)
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
        P = D.Problem(ctx, h["Q"], h["q"], h["G"], h["g"], h["lb"], h["ub"], prec=D.FP32, lmin_Q=self.lmin,
                      cone=D.CONE_EQ if self.equality else D.CONE_INEQ)
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
    wl = LargeDense(args, local, equality=args.workload == "eq")
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
    ms_max, value = replica_rate(ms, args.steps, world, device="cuda")

    # end to end through the C ABI from pinned host memory
    e2e = None
    if not args.no_e2e:
        wl.host_inputs()
        wl.step_host(D, ctx)  # warm-up: the context's upload staging buffer and copy stream
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
    # the library takes the single-pass iteration for n % 4 == 0, n <= 20480 unless DQ_GRID_SINGLE_PASS=0
    single_pass = n % 4 == 0 and n <= 20480 and os.environ.get("DQ_GRID_SINGLE_PASS", "1") != "0"
    r0 = results[-1]
    inner = statistics.mean(r.inner_iters for r in results)
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl.name, "n": n, "p": p, "alg": wl.alg, "eps": wl.eps,
                   "eps_in": wl.eps_in, "outputs": "last+average", "check_every": wl.check_every,
                   "inner_check_every": wl.inner_check_every,
                   "l2": ("inputs larger than L2 (packed H = Q + rho G'G 0.8 GB per inner iteration)"
                          if wl.equality else "inputs larger than L2 (packed Q 0.8 GB, G 0.8 GB per inner iteration)"),
                   "cone": "K={0}, Hessian mode (H built in every step)" if wl.equality else "K=R^p_-",
                   "parallelism": f"replicas{world}"},
        "solve": {"status": r0.status, "outer_iters": r0.outer_iters, "inner_iters_mean": inner,
                  "f_last": r0.f_last, "infeas_last": r0.infeas_last, "f_avg": r0.f_avg,
                  "infeas_avg": r0.infeas_avg, "d_lb": r0.d_lb, "converged_last": r0.converged_last,
                  "converged_avg": r0.converged_avg},
        "roofline": {"kernel": (("k_v2_pass<float> single-pass inner iteration (packed H)" if wl.equality else
                                 "k_v2_pass<float> single-pass inner iteration (packed Q, one read of G)")
                                if single_pass else "k_rows<float> inner-iteration GEMV"),
                     "bound": "hbm", "achieved": achieved,
                     "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": (achieved / peaks["hbm_gbs"]) if achieved else None,
                     "traffic": (st["gemv_bytes"] / st["gemv_launches"] *
                                 TRAFFIC_RATIO["k_v2_pass" if single_pass else "k_rows"])
                     if st["gemv_launches"] else None,
                     "traffic_unit": "bytes per launch (scaled from a smaller capture)",
                     "peak_kind": kind, "launches_timed": st["gemv_launches"],
                     "gemv_share_of_step": (st["gemv_ms"] / ms) if ms > 0 else None,
                     "reduce": ({"kernel": "k_v2_reduce", "us_per_launch": st["reduce_ms"] / st["reduce_launches"] * 1e3,
                                 "share_of_step": st["reduce_ms"] / ms} if st.get("reduce_launches") else None)},
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
              d["g"].double().cpu().numpy(), d["lb"].double().cpu().numpy(), d["ub"].double().cpu().numpy(),
              cone=O.CONE_EQ if getattr(wl, "equality", False) else O.CONE_INEQ)
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
            "config": {"workload": LargeDense.workload_name(args.n, args.p, args.alg), "n": args.n, "p": args.p,
                       "alg": args.alg, "eps": args.eps},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ other workloads

FP32_FFMA_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # 80.5: SMs x FP32 lanes x 2 flops x max SM clock
FP64_SM_TFLOPS = 1.25 / 152                         # nominal FP64 rate of one SM


def _timed(ctx, stream, fn, steps, warmup):
    """Warm-up, then `steps` calls of fn between CUDA events on the library's stream."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ctx.stats(reset=True)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    outs = [fn() for _ in range(steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), clocks.stop(), ctx.stats(reset=True), outs


def _base_line(args, value, ms, workload, dtype, cfg, clk, st, extra):
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": dict(workload=workload, parallelism="replicas1", **cfg), "gpu_launches": st["launches"],
            "clocks": clk}
    line.update(extra)
    return line


def _oracle_pool(tasks, budget_s):
    """Run oracle solves (callables) on all host cores until the budget; returns (solves/s, cores, done)."""
    from concurrent.futures import ThreadPoolExecutor
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    done = 0
    with ThreadPoolExecutor(cores) as ex:
        futs = []
        it = iter(tasks)
        for _ in range(cores):
            f = next(it, None)
            if f is None:
                break
            futs.append(ex.submit(f))
        while futs:
            fut = futs.pop(0)
            fut.result()
            done += 1
            if time.perf_counter() - t0 < budget_s:
                f = next(it, None)
                if f is not None:
                    futs.append(ex.submit(f))
    dt = time.perf_counter() - t0
    return done / dt, cores, done


def run_small(args):
    """n=50, p=25 FP64 DFGM (one instance, one thread block, eps=1e-4)."""
    import torch

    import oracle as O
    import workloads as W
    from paper_1504_05708_gb300 import duquad as D
    inst = W.single_dense(n=50, p=25, seed=0)
    stream = torch.cuda.current_stream()
    ctx = D.Context(0, stream)
    t = {k: torch.tensor(getattr(inst, k), dtype=torch.float64, device="cuda") for k in ("Q", "q", "G", "g", "lb", "ub")}
    P = D.Problem(ctx, t["Q"], t["q"], t["G"], t["g"], t["lb"], t["ub"], prec=D.FP64, lmin_Q=inst.lmin_Q)
    o = D.opts("DFGM", eps_out=1e-4, engine=D.ENGINE_CTA, fresh_constants=1)
    outs = (torch.empty(50, dtype=torch.float64, device="cuda"), torch.empty(50, dtype=torch.float64, device="cuda"),
            torch.empty(25, dtype=torch.float64, device="cuda"))
    ms, clk, st, res = _timed(ctx, stream, lambda: P.solve(o, device_out=outs)[0], args.steps, args.warmup)
    r = res[-1]
    # where a solve's time goes: the same solve with the handle's constants (no Lanczos runs),
    # and one outer iteration of one inner iteration (launch, set-up, evaluation, copies)
    o_keep = D.opts("DFGM", eps_out=1e-4, engine=D.ENGINE_CTA)
    o_min = D.opts("DFGM", engine=D.ENGINE_CTA, fixed_outer=1, fixed_inner=1)
    ms_keep = _timed(ctx, stream, lambda: P.solve(o_keep, device_out=outs)[0], args.steps, 2)[0] / args.steps
    ms_min = _timed(ctx, stream, lambda: P.solve(o_min, device_out=outs)[0], args.steps, 2)[0] / args.steps
    ms_solve = ms / args.steps
    breakdown = {"solve_ms": ms_solve, "lanczos_ms": ms_solve - ms_keep,
                 "iterations_ms": ms_keep - ms_min, "launch_setup_eval_ms": ms_min,
                 "us_per_inner_iteration": 1e3 * (ms_keep - ms_min) / max(r.inner_iters - 1, 1)}
    # e2e: host arrays through the ABI (handle creation, upload, solve, download, destroy)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        H = D.Problem(ctx, inst.Q, inst.q, inst.G, inst.g, inst.lb, inst.ub, prec=D.FP64, lmin_Q=inst.lmin_Q)
        H.solve(o)
        H.close()
    e2e_s = (time.perf_counter() - t0) / args.steps
    flops = r.inner_iters * 2.0 * 50 * 50 + r.outer_iters * 4.0 * 50 * 25
    peaks, kind = load_peaks()
    qp = O.QP(inst.Q, inst.q, inst.G, inst.g, inst.lb, inst.ub)
    c = O.constants(qp, O.DFGM, lmin_Q=inst.lmin_Q)
    tasks = [lambda: O.dfom(qp, O.DFGM, c, eps_out=1e-4, eps_in=O.default_eps_in(O.DFGM, 1e-4, c.Ld))] * 200000
    cpu_v, cores, done = _oracle_pool(tasks[:], min(args.cpu_seconds, 10.0))
    line = _base_line(args, args.steps / (ms / 1e3), ms, "single_dense_n50_p25_fp64_dfgm", "f64",
                      {"n": 50, "p": 25, "alg": "DFGM", "eps": 1e-4, "l2": "single 40 KB instance (latency-bound)"},
                      clk, st, {
                          "solve": {"status": r.status, "outer_iters": r.outer_iters, "inner_iters": r.inner_iters,
                                    "f_last": r.f_last, "infeas_last": r.infeas_last},
                          "breakdown": breakdown,
                          "roofline": {"kernel": "cta_solve_kernel<double>", "bound": "alu",
                                       "achieved": flops / (ms / args.steps / 1e3) / 1e12, "peak": FP64_SM_TFLOPS,
                                       "unit": "TFLOP/s", "frac": flops / (ms / args.steps / 1e3) / 1e12 / FP64_SM_TFLOPS,
                                       "traffic": None,
                                       "peak_kind": "derived: one SM's share (1/152) of the nominal 1.25 TFLOP/s FP64; "
                                                    "one instance runs in one thread block"},
                          "e2e": {"value": 1.0 / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": 8 * (50 * 50 + 25 * 50 + 3 * 50 + 25),
                                  "d2h_bytes_per_step": 8 * (2 * 50 + 25)},
                          "cpu_baseline": {"value": cpu_v, "unit": "solves/s", "cores": cores, "kind": "oracle",
                                           "sample": f"{done} FP64 oracle solves of the same instance on {cores} host threads"}})
    print(json.dumps(line), flush=True)
    P.close()
    ctx.close()


SWEEP_EPS = 1e-2
SWEEP_EPS_IN = (1e-1, 1e-2, 1e-3, 1e-4, 1e-5, 1e-6)
SWEEP_K = (1, 2, 5, 10, 20, 50, 100, 200, 500)
SWEEP_N = (10, 50, 100, 200, 300, 400, 500)


def run_sweep(args):
    """The paper's two parameter studies, run as persistent launches on the GPU (FP64, thread-block
    engine), with F* of every QP from a long FP64 oracle run on the host cores.

    (A) Inner accuracy (Sec. 4, Fig. dfgm_sensitivity): one strongly convex QP (n = 100, p = 50,
        eps = 1e-2); DGM and DFGM with the inner loop stopped at eps_in in SWEEP_EPS_IN, each run
        for k outer iterations, k in SWEEP_K; primal suboptimality |F - F*| and dist_K of the
        average and the last iterate at every (algorithm, eps_in, k).
    (B) Outer iteration counts (Sec. 6, Fig. comparison_dfo): `count` random QPs (default 25)
        per n in SWEEP_N (p = n/2, Q > 0, K = R^p_-), eps = 1e-2, stopped as in the paper on
        |F(u) - F*| <= eps and dist_K(Gu + g) <= eps (stop_fstar), for DGM and DFGM with the
        last iterate and the average as output: outer iterations per (n, algorithm, output).
    The table goes to --out (JSON); the printed line's value is study (B)'s solves/s."""
    from concurrent.futures import ThreadPoolExecutor

    import numpy as np
    import torch

    import oracle as O
    import workloads as W
    from paper_1504_05708_gb300 import duquad as D
    per_n = args.count or 25
    stream = torch.cuda.current_stream()
    ctx = D.Context(0, stream)

    def fstar(inst):  # F(x) of a long FP64 ADFGM run: |F(x) - F*| <= 1e-5, 1e-3 of the studies' eps
        qp = O.QP(inst.Q, inst.q, inst.G, inst.g, inst.lb, inst.ub)
        c = O.constants(qp, O.ADFGM, lmin_Q=inst.lmin_Q)
        r = O.dfom(qp, O.ADFGM, c, eps_out=1e-5, eps_in=1e-9, outer_check_every=5, max_outer=50000,
                   max_inner=50000)
        return O.F(qp, r.x_last if r.converged_last else r.x_avg), r.d_lb

    # (A) one QP, algorithms x eps_in x outer counts
    a_inst = W.single_dense(n=100, p=50, seed=11, g_scale=0.02)
    insts_b = [(n, W.single_dense(n=n, p=n // 2, seed=5000 + 97 * n + i, g_scale=0.02)) for n in SWEEP_N
               for i in range(per_n)]
    t0 = time.perf_counter()
    with ThreadPoolExecutor(os.cpu_count() or 1) as ex:
        fs = list(ex.map(fstar, [a_inst] + [i for _, i in insts_b]))
    oracle_s = time.perf_counter() - t0
    fa = fs[0][0]
    a_probs, a_ops, a_keys = [], [], []
    for alg in ("DGM", "DFGM"):
        for ein in SWEEP_EPS_IN:
            for k in SWEEP_K:
                a_probs.append(D.Problem(ctx, a_inst.Q, a_inst.q, a_inst.G, a_inst.g, a_inst.lb, a_inst.ub,
                                         prec=D.FP64, lmin_Q=a_inst.lmin_Q))
                a_ops.append(D.opts(alg, eps_out=SWEEP_EPS, eps_in=ein, fixed_outer=k, max_inner=100000,
                                    engine=D.ENGINE_CTA))
                a_keys.append((alg, ein, k))
    (a_outs, a_res) = D.solve_many(a_probs, a_ops)
    qa = O.QP(a_inst.Q, a_inst.q, a_inst.G, a_inst.g, a_inst.lb, a_inst.ub)
    table_a = []
    for (alg, ein, k), (xl, xa, _), r in zip(a_keys, a_outs, a_res):
        table_a.append({"alg": alg, "eps_in": ein, "k": k, "inner_iters": int(r.inner_iters),
                        "subopt_avg": abs(O.F(qa, xa[0]) - fa), "infeas_avg": O.infeas(qa, xa[0]),
                        "subopt_last": abs(O.F(qa, xl[0]) - fa), "infeas_last": O.infeas(qa, xl[0])})
    for P in a_probs:
        P.close()
    # (B) outer iteration counts at |F - F*| <= eps, dist_K <= eps
    b_probs, b_ops, b_keys = [], [], []
    for (n, inst), (f_star, _) in zip(insts_b, fs[1:]):
        for alg in ("DGM", "DFGM"):
            for out in (D.OUT_LAST, D.OUT_AVERAGE):
                b_probs.append(D.Problem(ctx, inst.Q, inst.q, inst.G, inst.g, inst.lb, inst.ub, prec=D.FP64,
                                         lmin_Q=inst.lmin_Q))
                b_ops.append(D.opts(alg, eps_out=SWEEP_EPS, output=out, max_outer=200000, f_star=f_star,
                                    engine=D.ENGINE_CTA))
                b_keys.append((n, alg, "last" if out == D.OUT_LAST else "average"))
    ms, clk, st, res = _timed(ctx, stream, lambda: D.solve_many(b_probs, b_ops), args.steps, args.warmup)
    b_outs, b_res = res[-1]
    rows = {}
    for (n, alg, out), r in zip(b_keys, b_res):
        rows.setdefault((n, alg, out), []).append(r)
    table_b = []
    for (n, alg, out), rs in sorted(rows.items()):
        it = np.array([r.outer_iters for r in rs], float)
        table_b.append({"n": n, "p": n // 2, "alg": alg, "output": out, "qps": len(rs),
                        "converged": sum(1 for r in rs if r.status == 0),
                        "outer_mean": float(it.mean()), "outer_min": int(it.min()), "outer_max": int(it.max()),
                        "inner_mean": float(np.mean([r.inner_iters for r in rs]))})
    # a re-scored check of (B)'s outputs: |F - F*| and dist_K in FP64 by the oracle
    worst = 0.0
    for (n, inst), (f_star, _), i in zip(insts_b, fs[1:], range(0, len(b_keys), 4)):
        qp = O.QP(inst.Q, inst.q, inst.G, inst.g, inst.lb, inst.ub)
        for j in range(4):
            xl, xa, _ = b_outs[i + j]
            x = xl[0] if b_keys[i + j][2] == "last" else xa[0]
            if b_res[i + j].status == 0:
                worst = max(worst, abs(O.F(qp, x) - f_star), O.infeas(qp, x))
    count = len(b_probs)
    table = {"eps": SWEEP_EPS, "study_A": {"n": 100, "p": 50, "seed": 11, "f_star": fa, "rows": table_a},
             "study_B": {"per_n": per_n, "rows": table_b, "worst_rescored": worst},
             "oracle_fstar_seconds": oracle_s}
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    with open(args.out, "w") as f:
        json.dump(table, f, indent=1)
    line = _base_line(args, count * args.steps / (ms / 1e3), ms, f"sweep_outer_counts_{per_n}x{len(SWEEP_N)}_fp64",
                      "f64", {"n": list(SWEEP_N), "p": "n/2", "eps": SWEEP_EPS, "algs": "DGM/DFGM x last/average",
                              "stop": "|F - F*| <= eps and dist_K <= eps (F* from the FP64 oracle)",
                              "l2": "all instances fit L2 (latency-bound sweep)"}, clk, st, {
                          "sweep": {"table": args.out, "worst_rescored": worst,
                                    "converged": sum(1 for r in b_res if r.status == 0), "solves": count},
                          "roofline": None, "e2e": None, "cpu_baseline": None})
    print(json.dumps(line), flush=True)
    for P in b_probs:
        P.close()
    ctx.close()


def run_sparse(args):
    """One large sparse QP in CSR form (Sec. 5's sparse case): n = 2e6, p = 1e6, Q a random-graph
    Laplacian + diag (about 9 nonzeros per row), G with 8 per row; FP32 ADFGM, eps = 1e-3, last
    iterate and average.  A step is one solve on the device-resident handle with the Lanczos
    constants recomputed; e2e adds handle creation from host CSR arrays and the download."""
    import numpy as np
    import torch

    import oracle as O
    import workloads as W
    from paper_1504_05708_gb300 import duquad as D
    n, p = args.n, args.p
    d = W.sparse_qp(n=n, p=p, seed=6)
    stream = torch.cuda.current_stream()
    ctx = D.Context(0, stream)

    def make():
        return D.SparseProblem(ctx, (d["Q_rowptr"], d["Q_col"], d["Q_val"]), d["q"],
                               (d["G_rowptr"], d["G_col"], d["G_val"]), d["g"], d["lb"], d["ub"], prec=D.FP32,
                               lmin_Q=d["lmin_Q"])
    P = make()
    o = D.opts(args.alg, eps_out=args.eps, eps_in=args.eps_in, check_every=args.check_every,
               inner_check_every=args.inner_check_every, max_outer=20000, fresh_constants=1)
    outs = (torch.empty(n, device="cuda"), torch.empty(n, device="cuda"), torch.empty(p, device="cuda"))
    ms, clk, st, res = _timed(ctx, stream, lambda: P.solve(o, device_out=outs)[0], args.steps, args.warmup)
    ctx.profile(True)
    ctx.stats(reset=True)
    r = P.solve(o, device_out=outs)[0]
    torch.cuda.synchronize()
    pst = ctx.stats(reset=True)
    ctx.profile(False)
    r = res[-1]
    e2e = None
    if not args.no_e2e:  # host CSR arrays through the ABI: create (validate, G', upload), solve, download
        Pw = make()
        Pw.solve(o)
        Pw.close()
        t0 = time.perf_counter()
        for _ in range(max(1, min(args.steps, 2))):
            Pe = make()
            Pe.solve(o)
            Pe.close()
        e2e_s = (time.perf_counter() - t0) / max(1, min(args.steps, 2))
        nnz = d["Q_col"].size + d["G_col"].size
        e2e = {"value": 1.0 / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": 12 * nnz + 4 * (n + p + 2) + 8 * (3 * n + p),
               "d2h_bytes_per_step": 8 * (2 * n + p)}
    peaks, kind = load_peaks()
    achieved = pst["gemv_bytes"] / (pst["gemv_ms"] / 1e3) / 1e9 if pst["gemv_ms"] > 0 else None
    # CPU baseline: the oracle's FOM step (FP64, scipy.sparse products) on the same data, scaled
    import scipy.sparse as sp
    Q = sp.csr_matrix((d["Q_val"], d["Q_col"], d["Q_rowptr"]), shape=(n, n))
    G = sp.csr_matrix((d["G_val"], d["G_col"], d["G_rowptr"]), shape=(p, n))
    y = np.zeros(n)
    t0, k = time.perf_counter(), 0
    while time.perf_counter() - t0 < min(args.cpu_seconds, 10.0):
        y = O.sampled_fom_step(q=d["q"], g=d["g"], G=G, Q_rows=None, rows=None, y=y, mu=np.zeros(p), rho=0.3,
                               L=40.0, lb=d["lb"], ub=d["ub"], Qy_full=Q @ y)
        k += 1
    per = (time.perf_counter() - t0) / k
    line = _base_line(args, args.steps / (ms / 1e3), ms, f"sparse_csr_n{n}_p{p}_fp32_{args.alg.lower()}", "f32",
                      {"n": n, "p": p, "nnz_Q": int(d["Q_col"].size), "nnz_G": int(d["G_col"].size),
                       "alg": args.alg, "eps": args.eps, "eps_in": args.eps_in, "outputs": "last+average",
                       "l2": "inputs larger than L2 (CSR arrays 0.3 GB)"}, clk, st, {
                          "solve": {"status": r.status, "outer_iters": r.outer_iters, "inner_iters": r.inner_iters,
                                    "f_last": r.f_last, "infeas_last": r.infeas_last, "f_avg": r.f_avg,
                                    "infeas_avg": r.infeas_avg, "d_lb": r.d_lb,
                                    "converged_last": r.converged_last, "converged_avg": r.converged_avg},
                          "roofline": {"kernel": "k_csr_form + k_csr_rows (CSR products of the inner iteration)",
                                       "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                       "frac": achieved / peaks["hbm_gbs"] if achieved else None, "traffic": None,
                                       "peak_kind": kind, "launches_timed": pst["gemv_launches"],
                                       "share_of_step": pst["gemv_ms"] / (ms / args.steps)},
                          "e2e": e2e,
                          "cpu_baseline": {"value": 1.0 / (per * max(r.inner_iters, 1)), "unit": "solves/s", "cores": 1,
                                           "kind": "oracle",
                                           "sample": f"{k} FOM steps of the oracle (FP64, scipy.sparse products) on the "
                                                     f"same instance ({per:.3f} s each), scaled by the GPU run's "
                                                     f"{r.inner_iters} inner iterations"}})
    print(json.dumps(line), flush=True)
    P.close()
    ctx.close()


UNEVEN_MAX_OUTER = 50000


def run_uneven(args):
    """10000 independent QPs, n ~ U{16..512}, p = n/2, mixed algorithms, one persistent launch."""
    import numpy as np
    import torch

    import oracle as O
    import workloads as W
    from paper_1504_05708_gb300 import duquad as D
    count = args.count
    insts = W.uneven_batch_device(count, 3, device="cuda")
    stream = torch.cuda.current_stream()
    ctx = D.Context(0, stream)
    probs, ops = [], []
    for d in insts:
        probs.append(D.Problem(ctx, d["Q"], d["q"], d["G"], d["g"], d["lb"], d["ub"], prec=D.FP32, lmin_Q=1.0))
        # DGM/ADGM converge at O(1/k) (Sec. 4): on the kappa ~ 1e4 instances the FP64 oracle
        # itself needs up to ~11000 outer iterations, so the limit leaves room for them
        ops.append(D.opts(d["alg"], eps_out=1e-3, max_outer=UNEVEN_MAX_OUTER, fresh_constants=1))
    tot_n = sum(d["n"] for d in insts)
    tot_p = sum(d["p"] for d in insts)
    bx = torch.empty(2 * tot_n, device="cuda")
    bl = torch.empty(tot_p, device="cuda")
    douts, on, op = [], 0, 0
    for d in insts:
        douts.append((bx[on:on + d["n"]], bx[tot_n + on:tot_n + on + d["n"]], bl[op:op + d["p"]]))
        on += d["n"]
        op += d["p"]
    tune = D.autotune(probs, ops, sample=256)
    peaks, kind = load_peaks()
    ms, clk, st, res = _timed(ctx, stream, lambda: D.solve_many(probs, ops, device_outs=douts), args.steps, args.warmup)
    rs = res[-1]
    nn = np.array([d["n"] for d in insts], float)
    pp = np.array([d["p"] for d in insts], float)
    aug = np.array([d["alg"] in ("ADGM", "ADFGM") for d in insts])
    inner = np.array([r.inner_iters for r in rs], float)
    flops = float(np.sum(inner * (2 * nn * nn + np.where(aug, 4 * nn * pp, 0.0))))
    tflops = flops / (ms / args.steps / 1e3) / 1e12
    # matrix bytes the algorithm streams: Q (and G, G' when rho > 0) per inner iteration, G and
    # G' once per outer iteration when rho = 0 (the batch's 5.4 GB of matrices exceed L2)
    outer = np.array([r.outer_iters for r in rs], float)
    mbytes = float(np.sum(inner * 4 * (nn * nn + np.where(aug, 2 * nn * pp, 0.0)) +
                          outer * np.where(aug, 0.0, 8 * nn * pp)))
    gbs = mbytes / (ms / args.steps / 1e3) / 1e9
    conv = sum(1 for r in rs if r.status == 0)
    # CPU baseline: the FP64 oracle on a sample of the same instances, all host cores
    sample = list(range(0, count, max(1, count // 400)))

    def task(i):
        d = insts[i]
        qp = O.QP(d["Q"].double().cpu().numpy(), d["q"].double().cpu().numpy(), d["G"].double().cpu().numpy(),
                  d["g"].double().cpu().numpy(), -np.ones(d["n"]), np.ones(d["n"]))
        a = O.ALG_NAMES[d["alg"]]
        c = O.constants(qp, a, lmin_Q=1.0)
        return lambda: O.dfom(qp, a, c, eps_out=1e-3, eps_in=O.default_eps_in(a, 1e-3, c.Ld),
                              max_outer=UNEVEN_MAX_OUTER)
    cpu_tasks = [task(i) for i in sample]
    cpu_v, cores, done = _oracle_pool(cpu_tasks, args.cpu_seconds)
    mean_cost = float(np.mean(nn[sample] ** 2)) / float(np.mean(nn ** 2))
    # only converged solves count
    line = _base_line(args, conv * args.steps / (ms / 1e3), ms, "uneven_10000_n16_512_fp32_mixed", "f32",
                      {"count": count, "n": "U{16..512}", "p": "n/2", "algs": "DGM/DFGM/ADGM/ADFGM", "eps": 1e-3,
                       "autotuned": {"threads": tune[0], "smem_cap": tune[1]}, "graph": True,
                       "l2": "5.4 GB of matrices, larger than L2"}, clk, st, {
                          "solve": {"converged": conv, "inner_iters_mean": float(inner.mean()),
                                    "inner_iters_p99": float(np.percentile(inner, 99)),
                                    "inner_iters_max": float(inner.max()),
                                    "n_of_max": int(nn[int(np.argmax(inner))]),
                                    "work_share_top1pct": float(np.sort(inner * nn * nn)[::-1][:max(1, count // 100)].sum()
                                                                / max((inner * nn * nn).sum(), 1.0))},
                          "roofline": {"kernel": "cta_solve_kernel<float> (persistent)", "bound": "hbm",
                                       "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                       "frac": gbs / peaks["hbm_gbs"], "traffic": None, "peak_kind": kind,
                                       "note": "matrix bytes streamed per iteration by the algorithm; instances "
                                               "whose matrices fit shared memory read them there",
                                       "alu": {"achieved": tflops, "peak": FP32_FFMA_TFLOPS, "unit": "TFLOP/s",
                                               "frac": tflops / FP32_FFMA_TFLOPS,
                                               "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"}},
                          "e2e": None,
                          "cpu_baseline": {"value": cpu_v * mean_cost, "unit": "solves/s", "cores": cores, "kind": "oracle",
                                           "sample": f"{done} of {len(sample)} sampled instances solved by the FP64 oracle on "
                                                     f"{cores} threads, rate scaled by the sample's mean n^2 vs the batch's"}})
    print(json.dumps(line), flush=True)
    for P in probs:
        P.close()
    ctx.close()


def run_mpc(args):
    """16384 condensed-MPC QPs sharing Q, G: tensor cores (bf16 hi/lo) vs plain FP32 on the same batch."""
    import numpy as np
    import torch

    import oracle as O
    import workloads as W
    from paper_1504_05708_gb300 import duquad as D
    B = args.count
    d = W.mpc_batch(batch=B)
    # lambda_min of the shared 100 x 100 Q, known to the user (one small eigen-solve of
    # the condensed MPC Hessian, done once offline); 0.999 keeps it a strict lower bound
    lmin = float(np.linalg.eigvalsh(d["Q"])[0]) * 0.999
    stream = torch.cuda.current_stream()
    ctx = D.Context(0, stream)
    dev = {k: torch.tensor(d[k], dtype=torch.float32, device="cuda") for k in ("Q", "qs", "G", "gs", "lb", "ub")}
    Pt = D.Problem(ctx, dev["Q"], dev["qs"], dev["G"], dev["gs"], dev["lb"], dev["ub"], prec=D.BF16X3, batch=B, lmin_Q=lmin)
    Pf = D.Problem(ctx, dev["Q"], dev["qs"], dev["G"], dev["gs"], dev["lb"], dev["ub"], prec=D.FP32, batch=B, lmin_Q=lmin)
    mo = args.max_outer or 20000
    ot = D.opts("DFGM", eps_out=1e-3, eps_in=1e-5, check_every=5, inner_check_every=3, max_outer=mo,
                fresh_constants=1)
    of = D.opts("DFGM", eps_out=1e-3, eps_in=1e-5, check_every=5, inner_check_every=3, max_outer=mo,
                engine=D.ENGINE_CTA, fresh_constants=1)
    outs = (torch.empty(B, 100, device="cuda"), torch.empty(B, 100, device="cuda"), torch.empty(B, 600, device="cuda"))
    ms, clk, st, res = _timed(ctx, stream, lambda: Pt.solve(ot, device_out=outs), args.steps, args.warmup)
    msf, clkf, stf, resf = _timed(ctx, stream, lambda: Pf.solve(of, device_out=outs), 1, 0)
    rs = res[-1]
    inner = np.array([r.inner_iters for r in rs], float)
    outer = np.array([r.outer_iters for r in rs], float)
    useful = float(np.sum(inner * 2 * 100 * 100 + outer * 4 * 600 * 100))
    issued_tile_iter = 3 * 2 * 128 * 112 * 112
    tflops = useful / (ms / args.steps / 1e3) / 1e12
    peaks, kind = load_peaks()
    sample = list(range(0, B, max(1, B // 200)))
    cs = O.constants(O.QP(d["Q"], d["qs"][0], d["G"], d["gs"][0], d["lb"], d["ub"]), O.DFGM, lmin_Q=lmin)

    def task(b):
        qp = O.QP(d["Q"], d["qs"][b], d["G"], d["gs"][b], d["lb"], d["ub"])
        return lambda: O.dfom(qp, O.DFGM, cs, eps_out=1e-3, eps_in=1e-5, outer_check_every=5, inner_check_every=3,
                              max_outer=20000)
    cpu_v, cores, done = _oracle_pool([task(b) for b in sample], args.cpu_seconds)
    line = _base_line(args, B * args.steps / (ms / 1e3), ms, "mpc_batch_16384_n100_p600_bf16x3_dfgm", "bf16x3",
                      {"batch": B, "n": 100, "p": 600, "alg": "DFGM", "eps": 1e-3, "eps_in": 1e-5,
                       "check_every": 5, "inner_check_every": 3,
                       "lmin_Q": lmin, "l2": "per-instance state streamed per outer iteration"}, clk, st, {
                          "fp32_plain": {"value": B / (msf / 1e3), "unit": "solves/s",
                                         "engine": "CTA engine, one instance per thread block, FP32"},
                          "solve": {"converged": int(sum(1 for r in rs if r.status == 0)),
                                    "inner_iters_mean": float(inner.mean()), "outer_iters_mean": float(outer.mean()),
                                    "outer_iters_p99": float(np.percentile(outer, 99)), "outer_iters_max": float(outer.max())},
                          "roofline": {"kernel": "k_tc_solve (tcgen05 bf16 hi/lo)", "bound": "tensor",
                                       "achieved": tflops, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                                       "frac": tflops / peaks["bf16_tflops"], "traffic": None, "peak_kind": kind,
                                       "note": f"useful flops (2n^2 per inner iteration, 4pn per outer); issued "
                                               f"per tile-iteration {issued_tile_iter} (3 products, padding)"},
                          "e2e": None,
                          "cpu_baseline": {"value": cpu_v, "unit": "solves/s", "cores": cores, "kind": "oracle",
                                           "sample": f"{done} of {len(sample)} sampled instances, FP64 oracle on {cores} threads"}})
    print(json.dumps(line), flush=True)
    Pt.close()
    Pf.close()
    ctx.close()


def run_served(args):
    """Poisson stream of solve requests into the persistent request loop."""
    import numpy as np
    import torch

    import oracle as O
    import workloads as W
    from paper_1504_05708_gb300 import duquad as D
    rate, dur = args.rate, args.duration
    times, kinds, picks = W.served_stream(rate=rate, duration=dur, seed=4)
    ctx = D.Context(0)
    pool = W.uneven_batch_device(args.pool, 5, device="cuda")
    probs = []
    for dd in pool:
        probs.append(D.Problem(ctx, dd["Q"], dd["q"], dd["G"], dd["g"], dd["lb"], dd["ub"], prec=D.FP32, lmin_Q=1.0))
    mpc = W.mpc_batch(batch=64, seed=6)
    mpc["lmin_Q"] = float(np.linalg.eigvalsh(mpc["Q"])[0]) * 0.999  # known for the shared Hessian
    mpc_probs = [D.Problem(ctx, mpc["Q"], mpc["qs"][i], mpc["G"], mpc["gs"][i], mpc["lb"], mpc["ub"], prec=D.FP32,
                           lmin_Q=mpc["lmin_Q"]) for i in range(8)]
    ops = {a: D.opts(a, eps_out=1e-3, max_outer=UNEVEN_MAX_OUTER) for a in W.ALGS}
    om = D.opts("DFGM", eps_out=1e-3, eps_in=1e-5, check_every=5, max_outer=20000, warm_start=1)
    rng = np.random.default_rng(7)
    for P, dd in zip(probs, pool):  # constants once per handle
        P.solve(ops[dd["alg"]])
    for P in mpc_probs:
        P.solve(om)
    # requests prepared up front: the submission loop only times and submits
    reqs = []
    for k, (ta, kind, pick) in enumerate(zip(times, kinds, picks)):
        if kind == 1:
            i = int(pick) % len(mpc_probs)
            reqs.append((ta, mpc_probs[i], om, mpc["qs"][i] + 0.1 * rng.standard_normal(100), 100, 600,
                         ("mpc", i) if k % 100 == 0 else None))
        else:
            i = int(pick) % len(probs)
            reqs.append((ta, probs[i], ops[pool[i]["alg"]], rng.standard_normal(pool[i]["n"]), pool[i]["n"],
                         pool[i]["p"], ("qp", i) if k % 100 == 0 else None))
    ctx.serve_start(slots=1024, hbm_budget_bytes=32 << 30)
    from collections import deque
    pending = deque()          # (ticket, t_submit, n, p, info, q) in submission order
    lat, meta = [], []
    lock = threading.Lock()
    done_flag = [False]

    def poller():  # polls a window of the oldest outstanding tickets
        while True:
            with lock:
                window = list(pending)[:256]
            if not window:
                if done_flag[0]:
                    return
                time.sleep(0.0005)
                continue
            finished = set()
            for tk, t0, n, p, info, q in window:
                r = ctx.poll(tk, n, p)
                if r is not None:
                    lat.append(time.perf_counter() - t0)
                    finished.add(tk)
                    if info is not None:
                        meta.append((info, q, r))
            if finished:
                with lock:
                    keep = [e for e in pending if e[0] not in finished]
                    pending.clear()
                    pending.extend(keep)
            else:
                time.sleep(0.0002)
    th = threading.Thread(target=poller, daemon=True)
    th.start()
    start = time.perf_counter()
    for ta, P, o, q, n, p, info in reqs:
        while time.perf_counter() - start < ta:
            pass
        tk = ctx.submit(P, o, q=q)
        with lock:
            pending.append((tk, time.perf_counter(), n, p, info, q))
    offered = time.perf_counter() - start
    done_flag[0] = True
    th.join(timeout=args.drain)
    total = time.perf_counter() - start
    drained = not th.is_alive()
    if drained:
        ctx.serve_stop()
    lat_ms = np.array(lat) * 1e3
    # plain per-instance FP32 form on the same mix: the first requests of the stream solved one
    # at a time (dq_solve, one launch and one synchronisation each), for a bounded time
    plain_n, t0 = 0, time.perf_counter()
    if drained:
        for ta, P, o, q, n, p, info in reqs:
            P.set_vectors(q=q)
            P.solve(o)
            plain_n += 1
            if time.perf_counter() - t0 > args.plain_seconds:
                break
    plain_s = time.perf_counter() - t0
    # FP64 oracle error on the 1% sample (every 100th request), host threads, bounded time
    host = {}
    for i in set(info[1] for info, *_ in meta if info[0] == "qp"):
        dd = pool[i]
        host[i] = (dd["Q"].double().cpu().numpy(), dd["G"].double().cpu().numpy(), dd["g"].double().cpu().numpy())

    def rescore(item):
        info, q, (stt, xl, xa, lm, r) = item
        kind, i = info
        if kind == "qp":
            dd = pool[i]
            Qh, Gh, gh = host[i]
            qp = O.QP(Qh, q, Gh, gh, -np.ones(dd["n"]), np.ones(dd["n"]))
            a = O.ALG_NAMES[dd["alg"]]
        else:
            qp = O.QP(mpc["Q"], q, mpc["G"], mpc["gs"][i], mpc["lb"], mpc["ub"])
            a = O.DFGM
        # a lower bound of F* from the oracle (ADFGM converges fastest; its d_lb bounds F* whatever
        # algorithm the request used), 1e-4 below F* at most
        c = O.constants(qp, O.ADFGM, lmin_Q=1.0 if kind == "qp" else mpc["lmin_Q"])
        ro = O.dfom(qp, O.ADFGM, c, eps_out=1e-4, eps_in=1e-8, outer_check_every=5, max_outer=20000)
        x = xl if r.converged_last else xa
        # the served answer re-scored in FP64: objective gap to the oracle's lower bound, infeasibility
        return float(O.F(qp, x) - ro.d_lb), float(O.infeas(qp, x))
    from concurrent.futures import ThreadPoolExecutor
    errs, t_or = [], time.perf_counter()
    sample = meta[:args.oracle_sample] if args.oracle_sample > 0 else meta
    with ThreadPoolExecutor(os.cpu_count() or 1) as ex:
        futs = [ex.submit(rescore, m) for m in sample]
        for f in futs:
            left = args.oracle_seconds - (time.perf_counter() - t_or)
            try:
                errs.append(f.result(timeout=max(left, 0.01)))
            except Exception:
                break
        for f in futs:
            f.cancel()
    line = {"metric": METRIC, "value": len(lat) / total, "unit": "solves/s", "n_gpus": 1, "steps": 1, "warmup": 0,
            "ms_per_step": total * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "served_poisson", "rate_per_s": rate, "duration_s": dur, "pool": args.pool,
                       "mpc_fraction": 0.05, "slots": 1024, "parallelism": "replicas1"},
            "served": {"requests": int(len(times)), "completed": int(len(lat)), "offered_s": offered,
                       "drained": drained,
                       "p50_ms": float(np.percentile(lat_ms, 50)) if len(lat_ms) else None,
                       "p99_ms": float(np.percentile(lat_ms, 99)) if len(lat_ms) else None,
                       "oracle_gap_max": max(e[0] for e in errs) if errs else None,
                       "oracle_infeas_max": max(e[1] for e in errs) if errs else None,
                       "oracle_sampled": len(errs), "oracle_sample_of": len(meta), "eps": 1e-3,
                       "plain_fp32": {"value": plain_n / plain_s if plain_n else None, "unit": "solves/s",
                                      "solves": plain_n,
                                      "how": "the stream's first requests one at a time through dq_solve "
                                             "(thread-block engine, one launch and one synchronisation each)"}}}
    print(json.dumps(line), flush=True)
    if not drained:  # requests still in flight: leave without tearing the loop down under them
        os._exit(0)
    for P in probs + mpc_probs:
        P.close()
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="large", choices=["large", "eq", "small", "uneven", "mpc", "served",
                                                             "sweep", "sparse"])
    ap.add_argument("--out", default="sweep_table.json", help="sweep workload: where the table goes")
    ap.add_argument("--count", type=int, default=None)
    ap.add_argument("--rate", type=float, default=20000.0)
    ap.add_argument("--duration", type=float, default=0.5)
    ap.add_argument("--drain", type=float, default=120.0)
    ap.add_argument("--oracle-sample", type=int, default=20, help="served: requests re-scored (0: the whole 1%% sample)")
    ap.add_argument("--oracle-seconds", type=float, default=120.0, help="served: time budget of the re-scoring")
    ap.add_argument("--plain-seconds", type=float, default=15.0, help="served: time budget of the plain FP32 leg")
    ap.add_argument("--max-outer", type=int, default=0, help="cap on outer iterations (mpc workload; profiling)")
    ap.add_argument("--pool", type=int, default=2000)
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
    ap.add_argument("--ref-inner-per-solve", type=int, default=5246)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "small":
        run_small(args)
    elif args.workload == "uneven":
        args.count = args.count or 10000
        run_uneven(args)
    elif args.workload == "mpc":
        args.count = args.count or 16384
        run_mpc(args)
    elif args.workload == "served":
        run_served(args)
    elif args.workload == "sweep":
        run_sweep(args)
    elif args.workload == "sparse":
        if args.n == 20000 and args.p == 10000:  # the dense defaults: take the sparse case's sizes
            args.n, args.p = 2_000_000, 1_000_000
        run_sparse(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
