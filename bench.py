#!/usr/bin/env python
"""Benchmark of the decomposed-kernel GP hot path on GB300.

One step = one full fit (eigenfunction tables, fused Phi generation + Gram
on the tensor cores, split reduction and assembly of A, Cholesky (float32
pivots, panels and update products on a float64 trailing matrix), inverse,
solve + float64 refinement, operand packing) followed by one full predict
(mean and variance) of the largest single-GPU workload: p=3, n=16 (M=4096),
N=2,000,000 training points x ~ N(0, 0.5^2 I_3), 200,000 test points. Inputs
are resident in device memory when the timed region starts; L2 is flushed
(256 MiB write) between timed steps (the step's own working set, ~1.5 GB,
is far larger than L2 as well). The p=2, n=20 (M=400, N=200,000) workload
is timed too and reported as a secondary key.

Prints one JSON line (rank 0). ``--impl reference`` times the FP64 CPU oracle
on the host cores instead (a bounded sample of the same workload per step).
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

METRIC = "fit+predict points/s at M=n^p; serve p50/p99 ms; mixed vs FP64 GPU at err ≤1e-4"
UNIT = "points/s"
WORKLOAD = ("p=3, n=16 (M=4096), N=2,000,000 train x~N(0,0.5^2 I_3), "
            "y=exp(-|x|^2)+sum_i sin(2x_i)+0.05 noise, 200,000 test points from the same law, "
            "eps=1.2, alpha=1, sigma2=0.0025")
WORKLOAD2 = ("p=2, n=20 (M=400), N=200,000 train x~U[-1,1]^2, y=sin(3x1)cos(2x2)+0.05 noise, "
             "50,000 test points, eps=1, alpha=0.8, sigma2=0.0025")
# bounded samples of the workload for the CPU oracle (first rows of the same arrays)
REF_SAMPLE = (10_000, 1_000)       # --impl reference, per step
CPU_SAMPLE = (40_000, 4_000)       # cpu_baseline and the accuracy check of our arm
FP64_SAMPLE = (500_000, 50_000)    # the float64 GPU form (linear in N; timed on a quarter)
FP64_PEAK_TFLOPS = 1.25  # nominal GB300 float64 rate (no measured figure available)
# float32 SIMT rate from unit counts and clocks: 152 SMs x 128 FMA/clock x 2 flops x 2.07 GHz
FP32_SIMT_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return dict(hbm=d["hbm_gbs"], bf16=d["bf16_tflops"], bf16_sus=d["bf16_tflops_sustained"],
                    src="measured")
    except Exception:
        return dict(hbm=6800.0, bf16=1900.0, bf16_sus=1700.0, src="fallback")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def traffic_from_profile(kernel_file: str, name: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current source of the kernel (matching sha256 prefix), else None."""
    src = os.path.join(ROOT, "paper_2403_12797_gb300", "csrc", kernel_file)
    prof = os.path.join(ROOT, "profiles", f"{name}.md")
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        txt = open(prof).read()
    except Exception:
        return None
    m_h = re.search(r"source_sha256_16:\s*([0-9a-f]{16})", txt)
    m_t = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not m_h or not m_t or m_h.group(1) != h:
        return None
    return float(m_t.group(1))


# ----------------------------------------------------------------------------- reference arm

def run_reference(args):
    """The FP64 CPU oracle on the host cores, each step a bounded sample of
    the benchmark workload (its first REF_SAMPLE training and test rows)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import fagp as O
    from paper_2403_12797_gb300 import workloads as W
    pr = W.workload3()
    Ns_, Nt_ = REF_SAMPLE
    X, y, Xs = pr.X[:Ns_], pr.y[:Ns_], pr.Xs[:Nt_]

    def step():
        m = O.fit(X, y, pr.n, pr.eps, pr.alpha, pr.sigma2)
        O.predict(m, Xs)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    v = (Ns_ + Nt_) / dt
    cores = os.cpu_count()
    sample = f"first {Ns_} train and {Nt_} test points of the workload per step"
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": WORKLOAD, "sample": sample},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------------- our arm

GROUPS = ("eig_tables", "colexp", "syrk_tc", "syrk64", "assemble", "cholesky", "tri_inverse", "solve_refine",
          "predict_tc", "predict64")


def profile_groups(L, C):
    groups = {}
    for g in GROUPS:
        n_, ms_ = C.c_int64(), C.c_double()
        if L.gp_profile_query(g.encode(), C.byref(n_), C.byref(ms_)) == 0:
            groups[g] = {"launches": n_.value, "total_ms": ms_.value}
    return groups


def timed_steps(step, steps, flush, stream, torch):
    """CUDA-event time (ms) of each of `steps` calls of step(), L2 flushed before each."""
    times = []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return times


def roofline_of(name, groups, pr, prec, steps, pk, profile_name, peak_kind):
    """Roofline object of one kernel group: algorithmic work per launch over its
    average CUDA-event launch time inside the timed steps."""
    M, N, Ns = pr.M, pr.N, pr.Ns
    # the mixed Gram runs on CTA pairs (gp_syrk_tc2.cu) for M > 384 (p <= 4)
    pair = M > 384 and pr.p <= 4 and prec != "fp64"
    work = {
        "syrk_tc": ("tensor", N * M * (M + 1) + 2 * N * M, "TFLOP/s",
                    "gp_syrk_tc2.cu" if pair else "gp_syrk_tc.cu"),
        "predict_tc": ("tensor", Ns * M * (M + 1) + 4 * Ns * M, "TFLOP/s", "gp_predict_tc.cu"),
        # the exact column maxima: one product and one max per value of Phi
        "colexp": ("alu", 2 * N * M, "TFLOP/s", "gp_syrk_tc.cu"),
        "cholesky": ("alu", M ** 3 / 3, "TFLOP/s", "gp_factor.cu"),
        "tri_inverse": ("alu", M ** 3 / 3, "TFLOP/s", "gp_factor.cu"),
    }
    if name not in work or name not in groups:
        return None
    g = groups[name]
    bound, units, unit, src = work[name]
    per_launch_ms = g["total_ms"] / max(1, g["launches"])
    achieved = units / (per_launch_ms / 1e3) / 1e12
    if bound == "tensor":
        peak = pk["bf16_sus"] if peak_kind == "sustained" else pk["bf16"]
        psrc = (f"measured bf16 dense, {peak_kind} (fp16 operands run at the bf16 rate)"
                if pk["src"] == "measured" else "fallback")
    elif prec == "fp64":
        peak, psrc = FP64_PEAK_TFLOPS, "nominal fp64 (2 DFMA/clock/SM x 152 SMs x 2.07 GHz)"
    else:
        # mixed: the inverse is float32, and the Cholesky's trailing updates
        # (nearly all of its M^3 / 3 flops) are float32 products
        peak, psrc = FP32_SIMT_PEAK_TFLOPS, "fp32 SIMT from unit counts and clocks"
    if name == "syrk_tc" and pair:
        profile_name = profile_name.replace("syrk_tc", "syrk_tc2")
    return {"kernel": name, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak, "traffic": traffic_from_profile(src, profile_name),
            "peak_source": psrc, "avg_launch_ms": per_launch_ms, "units_per_launch": units}


def run_ours(args):
    import ctypes as C

    import torch

    # the batch autotuner's plans persist across runs in the build folder
    os.environ.setdefault("GPFAGP_TUNE_CACHE", os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                            "paper_2403_12797_gb300", "_build", "tune_cache.tsv"))

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2403_12797_gb300 import _lib
    from paper_2403_12797_gb300 import build as _build
    from paper_2403_12797_gb300 import workloads as W

    if rank == 0:
        _build.build()
    if world > 1:
        dist.barrier()
    L = _lib.lib()
    L.gp_kernel_launches.restype = C.c_int64
    L.gp_profile_query.argtypes = [C.c_char_p, C.c_void_p, C.c_void_p]

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    main_w2 = args.workload == 2
    pr = W.workload2() if main_w2 else W.workload3()
    if args.train_rows or args.test_rows:
        # a smaller case of the same workload (profiling captures), never the default
        pr = _sub(pr, args.train_rows or pr.N, args.test_rows or pr.Ns)
    dev = torch.device("cuda", local)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    prec = args.prec

    def make_step(p):
        X = torch.from_numpy(p.X).to(dev)
        y = torch.from_numpy(p.y).to(dev)
        Xs = torch.from_numpy(p.Xs).to(dev)
        mean = torch.empty(p.Ns, dtype=torch.float64, device=dev)
        var = torch.empty(p.Ns, dtype=torch.float64, device=dev)

        if world == 1:
            def step():
                # fit and predict through the one-call entry point (the same kernels
                # as fit() then predict(), without the host round trip between them)
                m, _, _ = _lib.fit_predict(X, y, p.n, p.eps, p.alpha, p.sigma2, Xs, prec=prec,
                                           mean_out=mean, var_out=var)
                m.free()
        else:
            from paper_2403_12797_gb300 import dist as D

            def step():
                # this rank's shard of the training rows: its packed Gram, one
                # NCCL all-reduce of it in device memory, the same fit on
                # every rank; then this rank's own test points
                m = D.fit_sharded(X, y, p.n, p.eps, p.alpha, p.sigma2, prec=prec, device=dev, local=True)
                m.predict(Xs, mean_out=mean, var_out=var)
                m.free()
        return step, (X, y, Xs, mean, var)

    step, (X, y, Xs, mean, var) = make_step(pr)
    for _ in range(args.warmup):
        step()
    barrier()

    L.gp_profile_reset()
    L.gp_profile_enable(1)
    launches0 = L.gp_kernel_launches()
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    times = timed_steps(step, args.steps, flush, stream, torch)
    barrier()
    clk = clocks.stop()
    launches = L.gp_kernel_launches() - launches0
    L.gp_profile_enable(0)
    groups = profile_groups(L, C)

    t_all = torch.tensor([sum(times)], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t_all, op=dist.ReduceOp.MAX)
    t_max_ms = float(t_all.item())
    points = (pr.N + pr.Ns) * args.steps * world
    value = points / (t_max_ms / 1e3)

    # ---- roofline of the dominant kernel group (device time inside the timed steps).
    # The timed loop runs for seconds, so tensor-core kernels are held to the
    # sustained (power-capped) bf16 rate.
    pk = peaks()
    tag = "w2" if main_w2 else "w3"
    peak_kind = "burst" if main_w2 else "sustained"
    total_dev = sum(g["total_ms"] for g in groups.values()) or 1.0
    shares = {k: round(v["total_ms"] / total_dev, 4) for k, v in groups.items()}
    dom = max((k for k in groups if k in ("syrk_tc", "predict_tc", "cholesky", "tri_inverse")),
              key=lambda k: groups[k]["total_ms"], default=None)
    roofline = roofline_of(dom, groups, pr, prec, args.steps, pk, f"{dom}_{tag}", peak_kind) if dom else None
    kernels = {k: roofline_of(k, groups, pr, prec, args.steps, pk, f"{k}_{tag}", peak_kind)
               for k in ("syrk_tc", "predict_tc", "cholesky", "tri_inverse", "colexp") if k in groups}
    if kernels.get("syrk_tc") is not None:
        # four fp16 products per pair of Phi values (s1 s1', s1 lo', lo s1', lo lo')
        kernels["syrk_tc"]["executed_tflops"] = kernels["syrk_tc"]["achieved"] * 4

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t_max_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": ("f16 tensor (integer + remainder slices, f32 acc in exact 4096-row blocks) "
                     "+ f32 pivots, panels and update products on an f64 trailing matrix, "
                     "f64 refinement") if prec != "fp64" else "f64",
           "data": "synthetic",
           "config": {"workload": WORKLOAD2 if main_w2 else WORKLOAD, "prec": prec,
                      "l2": "flushed between steps (256 MiB write); inputs and tables exceed L2",
                      "parallelism": ("single GPU" if world == 1 else
                                      f"row-sharded fit over {world} GPUs: every rank holds one shard of "
                                      "the workload's size (the same rows), one NCCL all-reduce of the "
                                      "packed Gram in device memory, the factorisation replicated, each "
                                      "rank predicting its own test points")},
           "gpu_launches": int(launches), "clocks": clk, "roofline": roofline,
           "kernels": kernels, "kernel_shares": shares,
           # device time of the kernel groups per step; the rest of ms_per_step is the
           # host's turnaround inside the API calls (status reads, the fit -> predict handoff)
           "device_busy_ms_per_step": sum(g["total_ms"] for g in groups.values()) / args.steps}

    if world == 1 and not main_w2 and not args.quick:
        # the p=2, n=20 workload as a secondary key (same step, same timing rules;
        # on one GPU only: with several, the step holds a collective)
        pr2 = W.workload2()
        step2, _ = make_step(pr2)
        for _ in range(3):
            step2()
        torch.cuda.synchronize()
        t2 = timed_steps(step2, 20, flush, stream, torch)
        out["workload2"] = {"workload": WORKLOAD2, "value": (pr2.N + pr2.Ns) * len(t2) / (sum(t2) / 1e3),
                            "unit": UNIT, "ms_per_step": sum(t2) / len(t2), "steps": len(t2)}
    if rank == 0:
        # the log marginal likelihood of the fitted model (the objective of
        # hyperparameter learning), from device-resident y; outside the timed steps
        m = _lib.fit(X, y, pr.n, pr.eps, pr.alpha, pr.sigma2, prec=prec)
        lml = m.log_marginal(y)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(5):
            lml = m.log_marginal(y)
        out["log_marginal"] = {"value": lml, "ms_per_call": (time.perf_counter() - t0) / 5 * 1e3}
        m.free()
    if rank == 0 and not args.quick:
        out.update(compare_and_baselines(args, pr, main_w2, dev, stream, _lib, torch))
        if not args.no_extras:
            out["batched_fit"] = batched_fit_bench(_lib, torch, dev)
            out["serving"] = serving_bench(_lib, torch, dev)
            out["serving_fp64"] = serving_bench(_lib, torch, dev, prec="fp64")
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def _sub(pr, N_, Ns_):
    """The first N_ training and Ns_ test rows of a workload."""
    import dataclasses
    return dataclasses.replace(pr, X=pr.X[:N_].copy(), y=pr.y[:N_].copy(), Xs=pr.Xs[:Ns_].copy())


def _errs(mean, var, mo, vo, O):
    import numpy as np
    return {"err_mean_rel_l2": O.relerr(mean, mo), "err_var_rel_l2": O.relerr(var, vo),
            "err_mean_max_abs_rel": float(np.max(np.abs(mean - mo)) / np.max(np.abs(mo))),
            "err_var_max_rel": float(np.max(np.abs(var - vo) / vo))}


def compare_and_baselines(args, pr, main_w2, dev, stream, _lib, torch):
    """The float64 GPU form's throughput, the end-to-end host-buffer number,
    the oracle's CPU time on a bounded sample, and both GPU modes' errors
    against the oracle on that sample."""
    from oracle import fagp as O
    res = {}

    def fit_predict_dev(p, prec):
        X, y, Xs = (torch.from_numpy(a).to(dev) for a in (p.X, p.y, p.Xs))
        mean = torch.empty(p.Ns, dtype=torch.float64, device=dev)
        var = torch.empty(p.Ns, dtype=torch.float64, device=dev)

        def step():
            m, _, _ = _lib.fit_predict(X, y, p.n, p.eps, p.alpha, p.sigma2, Xs, prec=prec,
                                       mean_out=mean, var_out=var)
            m.free()
        return step, mean, var

    # ---- the plain float64 GPU form on a quarter of the workload (its cost is
    # linear in N and N*, so the rate carries over; the M^3 factorisation is
    # included in full)
    p64 = pr if main_w2 else _sub(pr, *FP64_SAMPLE)
    step64, _, _ = fit_predict_dev(p64, "fp64")
    step64()
    torch.cuda.synchronize()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    ts = timed_steps(step64, 3 if main_w2 else 1, flush, stream, torch)
    res["fp64_gpu"] = {"value": (p64.N + p64.Ns) / (statistics.mean(ts) / 1e3), "unit": UNIT,
                       "ms_per_step": statistics.mean(ts),
                       "sample": f"first {p64.N} train and {p64.Ns} test points of the workload"}

    # ---- end to end through the C ABI with pinned host buffers, copies inside
    # the timed region (before the oracle, whose host threads would compete)
    Xh = torch.from_numpy(pr.X).pin_memory().numpy()
    yh = torch.from_numpy(pr.y).pin_memory().numpy()
    Xsh = torch.from_numpy(pr.Xs).pin_memory().numpy()
    mh = torch.empty(pr.Ns, dtype=torch.float64).pin_memory().numpy()
    vh = torch.empty(pr.Ns, dtype=torch.float64).pin_memory().numpy()

    def e2e_step():
        m, _, _ = _lib.fit_predict(Xh, yh, pr.n, pr.eps, pr.alpha, pr.sigma2, Xsh, prec=args.prec,
                                   mean_out=mh, var_out=vh)
        m.free()

    for _ in range(3):
        e2e_step()
    n_e2e = max(3, min(args.steps, 10))
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        e2e_step()
    dt = (time.perf_counter() - t0) / n_e2e
    res["e2e"] = {"value": (pr.N + pr.Ns) / dt, "unit": UNIT, "steps": n_e2e,
                  "h2d_bytes_per_step": int((pr.N * pr.p + pr.N + pr.Ns * pr.p) * 8),
                  "d2h_bytes_per_step": int(pr.Ns * 2 * 8)}

    # ---- the oracle on a bounded sample: the CPU baseline and the accuracy
    # reference of both GPU modes on the same rows
    ps = pr if main_w2 else _sub(pr, *CPU_SAMPLE)
    t0 = time.perf_counter()
    mdl = O.fit(ps.X, ps.y, ps.n, ps.eps, ps.alpha, ps.sigma2)
    mo, vo = O.predict(mdl, ps.Xs)
    t_or = time.perf_counter() - t0
    sample = f"first {ps.N} train and {ps.Ns} test points of the workload, once"
    res["cpu_baseline"] = {"value": (ps.N + ps.Ns) / t_or, "unit": UNIT, "cores": os.cpu_count(),
                           "kind": "oracle", "sample": sample}
    acc = {"sample": sample, "tol_mean": 1e-4, "tol_var": 1e-3, "tol_fp64": 1e-10}
    for prec in ("mixed", "fp64"):
        stp, mean, var = fit_predict_dev(ps, prec)
        stp()
        torch.cuda.synchronize()
        acc[prec] = _errs(mean.cpu().numpy(), var.cpu().numpy(), mo, vo, O)
    res["accuracy"] = acc
    return res


def batched_fit_bench(_lib, torch, dev):
    """The batched-fit workload: 256 independent GPs of uneven shape fitted by
    one gp_fit_batch (inputs resident on the device), against the same fits
    one after another; mixed precision and float64. The first call of each
    mode tunes the plan (untimed; kept in GPFAGP_TUNE_CACHE)."""
    from paper_2403_12797_gb300 import workloads as W
    probs = W.workload4(count=256, Ns=1)
    items = [(torch.from_numpy(pr.X).to(dev), torch.from_numpy(pr.y).to(dev), pr.n, pr.eps, pr.alpha,
              pr.sigma2) for pr in probs]
    points = sum(pr.X.shape[0] for pr in probs)
    out = {"workload": "256 GPs: N log-uniform [1e3, 2e5], p in {1,2,3,4}, M = n^p <= 1024, "
                       "inputs on the device",
           "points": points}
    for prec in ("mixed", "fp64"):
        for m in _lib.fit_batch(items, prec=prec):  # tunes the plan for this batch, warms the pool
            m.free()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        models = _lib.fit_batch(items, prec=prec)
        torch.cuda.synchronize()
        t_batch = time.perf_counter() - t0
        graph, _ = _lib.batch_info()
        plan = _lib.batch_plan()
        for m in models:
            m.free()
        t0 = time.perf_counter()
        for it in items:
            _lib.fit(*it, prec=prec).free()
        torch.cuda.synchronize()
        t_seq = time.perf_counter() - t0
        out[prec] = {"ms": t_batch * 1e3, "points_per_s": points / t_batch,
                     "sequential_ms": t_seq * 1e3, "sequential_points_per_s": points / t_seq,
                     "speedup": t_seq / t_batch, "one_graph": bool(graph), "plan": plan}
    return out


def serving_bench(_lib, torch, dev, prec="mixed"):
    """The serving workload: 64 resident models (p in {2,3,4}, M <= 2048, N up
    to 5e5, fitted by one batched fit); a closed-loop burst gives the
    saturating request rate, then open-loop Poisson streams at 50 % and 80 %
    of it (predict sizes log-uniform on [1, 65536], 5 % refits with N
    log-uniform on [1e4, 5e5]) give p50/p99 latency and throughput.

    prec="fp64": the same models, streams and server with float64 models.
    Their training sets (and the refits') are cut to their first 20,000 rows,
    since float64 fits at 5e5 rows would take minutes on this GPU's float64
    units; a predict's cost does not depend on N."""
    from paper_2403_12797_gb300 import workloads as W
    cap = None if prec == "mixed" else 20_000
    mods = W.workload5_models(count=64)
    if cap:
        mods = [_sub(pr, cap, 0) for pr in mods]
    models = _lib.fit_batch([(pr.X, pr.y, pr.n, pr.eps, pr.alpha, pr.sigma2) for pr in mods], prec=prec)
    n_esc = sum(1 for m in models if m.gram_fp64)
    out = {"workload": "64 resident models: p in {2,3,4}, M <= 2048, N log-uniform [1e4, 5e5]; "
                       "predict sizes log-uniform [1, 65536], 5 % refits (N log-uniform [1e4, 5e5])"
                       + ("" if not cap else "; float64 models on the first 20,000 rows of each training "
                                             "set and of each refit"),
           "prec": prec,
           "models_fit_points": sum(pr.X.shape[0] for pr in mods),
           "models_gram_fp64": n_esc}

    def stream_of(count, rate, seed):
        st_ = W.workload5_stream(mods, count, rate, refit_frac=0.05, seed=seed)
        if cap:
            for r in st_:
                if r.kind == "refit":
                    r.refit = _sub(r.refit, cap, 0)
        return st_
    with _lib.Server(slots=8) as srv:
        ids = [srv.add_model(m) for m in models]
        # closed loop: a burst of the same request mix (5 % refits) submitted at once
        burst = stream_of(200, 1e9, 1)
        srv.reset_stats()
        t0 = time.perf_counter()
        tk = [srv.submit_refit(ids[r.model], r.refit.X, r.refit.y) if r.kind == "refit"
              else srv.submit_predict(ids[r.model], r.Xs) for r in burst]
        for t in tk:
            srv.wait(t, timeout=600.0)
        wall = time.perf_counter() - t0
        st = srv.stats()
        sat_rate = len(burst) / wall
        out["saturation"] = {"requests_per_s": sat_rate, "points_per_s": st["points_per_s"],
                             "refits": st["refits_done"], "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
                             "peak_inflight": st["peak_inflight"], "batches": st["batches"],
                             "peak_batch": st["peak_batch"]}
        out["refits_gram_fp64"] = sum(1 for i in ids if _lib.lib().gp_model_flags(srv.model_handle(i)) & 1)
        for frac in (0.5, 0.8):
            rate = frac * sat_rate
            stream = stream_of(max(20, int(rate * 3.0)), rate, 2)
            srv.reset_stats()
            t0 = time.perf_counter()
            tk = []
            for r in stream:
                delay = r.t_arrive - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(delay)
                if r.kind == "refit":
                    tk.append(srv.submit_refit(ids[r.model], r.refit.X, r.refit.y))
                else:
                    tk.append(srv.submit_predict(ids[r.model], r.Xs))
            for t in tk:
                srv.wait(t, timeout=600.0)
            st = srv.stats()
            out[f"load_{int(frac * 100)}"] = {
                "offered_requests_per_s": rate, "requests": len(stream),
                "refits": st["refits_done"], "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
                "points_per_s": st["points_per_s"], "peak_inflight": st["peak_inflight"],
                "batches": st["batches"], "peak_batch": st["peak_batch"]}
    return out


def run_sweep(args):
    """The paper's own timing sweep (Sec. 3; row f4): y = sum_i cos(x_i) + nu
    on N = 10,000 training and 1,000 test points for p in {1, 2, 4} over a
    range of n, each fit + predict timed end to end as the paper times it
    (host arrays in and out: allocation and copies inside), median of
    --steps runs after --warmup. Beside each GPU time, the FP64 CPU oracle on
    the host cores, once, on the points with M <= 2500 (the larger ones take
    minutes there). One JSON line; not part of the default run."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np
    from oracle import fagp as O
    from paper_2403_12797_gb300 import _lib, workloads as W
    grid = {1: (10, 50, 100, 200, 400), 2: (5, 10, 15, 20, 30, 40, 50), 4: (3, 5, 7, 9, 11)}
    rows = []
    for p, ns in grid.items():
        for n in ns:
            pr = W.workload6(p, n)
            mean = np.empty(pr.Ns)
            var = np.empty(pr.Ns)

            def step():
                m, _, _ = _lib.fit_predict(pr.X, pr.y, pr.n, pr.eps, pr.alpha, pr.sigma2, pr.Xs,
                                           prec=args.prec, mean_out=mean, var_out=var)
                m.free()

            for _ in range(args.warmup):
                step()
            ts = []
            for _ in range(args.steps):
                t0 = time.perf_counter()
                step()
                ts.append(time.perf_counter() - t0)
            t = statistics.median(ts)
            row = {"p": p, "n": n, "M": n ** p, "ms": t * 1e3, "points_per_s": (pr.N + pr.Ns) / t}
            if n ** p <= 2500:
                t0 = time.perf_counter()
                mdl = O.fit(pr.X, pr.y, pr.n, pr.eps, pr.alpha, pr.sigma2)
                mo, vo = O.predict(mdl, pr.Xs)
                row["cpu_oracle_ms"] = (time.perf_counter() - t0) * 1e3
                row["err_mean_rel_l2"] = O.relerr(mean, mo)
                row["err_var_rel_l2"] = O.relerr(var, vo)
            rows.append(row)
    print(json.dumps({"metric": "paper sweep: fit+predict time, host arrays in and out",
                      "unit": "ms", "prec": args.prec, "data": "synthetic",
                      "config": {"workload": "y = sum cos(x_i) + 0.1 noise, x~U[-1,1]^p, "
                                             "N = 10,000 train, 1,000 test points"},
                      "cpu_cores": os.cpu_count(),
                      "steps": args.steps, "warmup": args.warmup, "rows": rows}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--workload", type=int, default=3, choices=[2, 3],
                    help="3: p=3, n=16, M=4096, N=2e6 (the benchmark); 2: p=2, n=20, M=400, N=2e5")
    ap.add_argument("--quick", action="store_true", help="skip the comparisons (profiling runs)")
    ap.add_argument("--train-rows", type=int, default=0,
                    help="use only the first R training rows (smaller profiling captures)")
    ap.add_argument("--test-rows", type=int, default=0,
                    help="use only the first R test rows (smaller profiling captures)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched-fit and serving measurements")
    ap.add_argument("--sweep", action="store_true",
                    help="the paper's timing sweep (p in {1, 2, 4}, N = 10,000) instead of the benchmark")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if not args.quick else args.warmup
    if args.impl == "reference":
        run_reference(args)
    elif args.sweep:
        run_sweep(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
