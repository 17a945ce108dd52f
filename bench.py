#!/usr/bin/env python
"""Benchmark of the decomposed-kernel GP hot path on GB300.

One step = one full fit (eigenfunction tables, fused Phi generation + Gram
on the tensor cores, split reduction and assembly of A, float64 Cholesky,
inverse, solve + refinement, operand packing) followed by one full predict
(mean and variance) of the p=2, n=20 (M=400) workload: N=200,000 training
points, 50,000 test points. Inputs are resident in device memory when the
timed region starts; L2 is flushed (256 MiB write) between timed steps.

Prints one JSON line (rank 0). ``--impl reference`` times the FP64 CPU oracle
on the host cores instead (bounded sample of the same workload).
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
WORKLOAD = ("p=2, n=20 (M=400), N=200,000 train x~U[-1,1]^2, y=sin(3x1)cos(2x2)+0.05 noise, "
            "50,000 test points, eps=1, alpha=0.8, sigma2=0.0025")
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
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np
    from oracle import fagp as O
    from paper_2403_12797_gb300 import workloads as W
    pr = W.workload2()
    # bounded sample of the workload: a quarter of the training and test points
    Ns_, Nt_ = pr.N // 4, pr.Ns // 4
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
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": WORKLOAD, "sample": f"{Ns_} train + {Nt_} test points per step"},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"first {Ns_} train and {Nt_} test points of the workload"},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------------- our arm

def run_ours(args):
    import numpy as np
    import torch

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
    L.gp_kernel_launches.restype = __import__("ctypes").c_int64
    L.gp_profile_query.argtypes = [__import__("ctypes").c_char_p, __import__("ctypes").c_void_p,
                                   __import__("ctypes").c_void_p]

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    pr = W.workload2()
    dev = torch.device("cuda", local)
    X = torch.from_numpy(pr.X).to(dev)
    y = torch.from_numpy(pr.y).to(dev)
    Xs = torch.from_numpy(pr.Xs).to(dev)
    mean = torch.empty(pr.Ns, dtype=torch.float64, device=dev)
    var = torch.empty(pr.Ns, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(prec):
        # fit and predict through the one-call entry point (the same kernels
        # as fit() then predict(), without the host round trip between them)
        m, _, _ = _lib.fit_predict(X, y, pr.n, pr.eps, pr.alpha, pr.sigma2, Xs, prec=prec,
                                   mean_out=mean, var_out=var)
        m.free()

    prec = args.prec
    for _ in range(args.warmup):
        step(prec)
    barrier()

    import ctypes as C
    L.gp_profile_reset()
    L.gp_profile_enable(1)
    launches0 = L.gp_kernel_launches()
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    times = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(prec)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    barrier()
    clk = clocks.stop()
    launches = L.gp_kernel_launches() - launches0
    L.gp_profile_enable(0)
    groups = {}
    for g in ("eig_tables", "syrk_tc", "syrk64", "assemble", "cholesky", "tri_inverse",
              "solve_refine", "predict_tc", "predict64"):
        n_, ms_ = C.c_int64(), C.c_double()
        if L.gp_profile_query(g.encode(), C.byref(n_), C.byref(ms_)) == 0:
            groups[g] = {"launches": n_.value, "total_ms": ms_.value}

    t_step = sum(times) / len(times)
    t_all = torch.tensor([sum(times)], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t_all, op=dist.ReduceOp.MAX)
    t_max_ms = float(t_all.item())
    points = (pr.N + pr.Ns) * args.steps * world
    value = points / (t_max_ms / 1e3)

    # ---- roofline of the dominant kernel group (device time inside the timed steps)
    pk = peaks()
    M, N, Ns = pr.M, pr.N, pr.Ns
    work = {
        "syrk_tc": ("tensor", N * M * (M + 1) + 2 * N * M, pk["bf16"], "TFLOP/s", "gp_syrk_tc.cu"),
        "predict_tc": ("tensor", Ns * M * (M + 1) + 4 * Ns * M, pk["bf16"], "TFLOP/s", "gp_predict_tc.cu"),
        "cholesky": ("alu", M ** 3 / 3, FP64_PEAK_TFLOPS, "TFLOP/s", "gp_factor.cu"),
        "tri_inverse": ("alu", M ** 3 / 3, FP64_PEAK_TFLOPS if prec == "fp64" else FP32_SIMT_PEAK_TFLOPS,
                        "TFLOP/s", "gp_factor.cu"),
        "eig_tables": ("hbm", (N + Ns) * 2 * 8 + (N + Ns) * 2 * pr.n * 4, pk["hbm"], "GB/s", "gp_tables.cu"),
    }
    total_dev = sum(g["total_ms"] for g in groups.values()) or 1.0
    shares = {k: round(v["total_ms"] / total_dev, 4) for k, v in groups.items()}
    dom = max((k for k in groups if k in work), key=lambda k: groups[k]["total_ms"], default=None)

    def roof(name):
        g = groups[name]
        bound, units, peak, unit, src = work[name]
        per_launch_ms = g["total_ms"] / max(1, g["launches"]) * (1 if name != "eig_tables" else 2)
        # eig_tables runs twice per step (train and test); its work figure is per step
        per_launch_ms = g["total_ms"] / args.steps if name == "eig_tables" else per_launch_ms
        scale = 1e12 if unit == "TFLOP/s" else 1e9
        achieved = units / (per_launch_ms / 1e3) / scale
        tr = traffic_from_profile(src, f"{name}_w2")
        return {"kernel": name, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak, "traffic": tr,
                "peak_source": ("measured bf16 burst" if bound == "tensor" and pk["src"] == "measured"
                                else "measured HBM copy" if bound == "hbm" and pk["src"] == "measured"
                                else ("nominal fp64" if (name == "cholesky" or prec == "fp64")
                                      else "fp32 SIMT from unit counts and clocks") if bound == "alu"
                                else "fallback"),
                "avg_launch_ms": per_launch_ms}

    roofline = roof(dom) if dom else None
    roof_syrk = roof("syrk_tc") if "syrk_tc" in groups else None
    if roof_syrk is not None:
        # four fp16 products per pair of Phi values (s1 s1', s1 lo', lo s1', lo lo')
        roof_syrk["executed_tflops"] = roof_syrk["achieved"] * 4

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t_max_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": ("f16 tensor (integer + remainder slices, f32 acc in exact 1024-row blocks) "
                     "+ f64 factorisation") if prec != "fp64" else "f64",
           "data": "synthetic",
           "config": {"workload": WORKLOAD, "prec": prec, "l2": "flushed between steps (256 MiB write)",
                      "replicas": world},
           "gpu_launches": int(launches), "clocks": clk, "roofline": roofline,
           "roofline_syrk": roof_syrk, "kernel_shares": shares,
           # device time of the kernel groups per step; the rest of ms_per_step is the
           # host's turnaround inside the API calls (status reads, the fit -> predict handoff)
           "device_busy_ms_per_step": sum(g["total_ms"] for g in groups.values()) / args.steps}

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
        extra = compare_and_baselines(args, pr, X, y, Xs, dev, stream, _lib, torch, np)
        out.update(extra)
        if not args.no_extras:
            out["batched_fit"] = batched_fit_bench(_lib, torch, dev)
            out["serving"] = serving_bench(_lib, torch, dev)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def compare_and_baselines(args, pr, X, y, Xs, dev, stream, _lib, torch, np):
    """Errors of both GPU modes vs the FP64 oracle, the FP64 GPU form's
    throughput, the oracle's CPU time, and the end-to-end host-buffer number."""
    from oracle import fagp as O
    res = {}
    # ---- FP64 GPU form, same workload
    mean = torch.empty(pr.Ns, dtype=torch.float64, device=dev)
    var = torch.empty(pr.Ns, dtype=torch.float64, device=dev)

    def step(prec):
        m, _, _ = _lib.fit_predict(X, y, pr.n, pr.eps, pr.alpha, pr.sigma2, Xs, prec=prec,
                                   mean_out=mean, var_out=var)
        m.free()

    step("fp64")
    torch.cuda.synchronize()
    ts = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step("fp64")
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    m64, v64 = mean.cpu().numpy().copy(), var.cpu().numpy().copy()
    step(args.prec)
    torch.cuda.synchronize()
    mmx, vmx = mean.cpu().numpy().copy(), var.cpu().numpy().copy()

    # ---- end to end through the C ABI with pinned host buffers (before the
    # oracle, whose many host threads would compete with the API calls)
    Xh = torch.from_numpy(pr.X).pin_memory().numpy()
    yh = torch.from_numpy(pr.y).pin_memory().numpy()
    Xsh = torch.from_numpy(pr.Xs).pin_memory().numpy()
    mh = torch.empty(pr.Ns, dtype=torch.float64).pin_memory().numpy()
    vh = torch.empty(pr.Ns, dtype=torch.float64).pin_memory().numpy()

    def e2e_step():
        m, _, _ = _lib.fit_predict(Xh, yh, pr.n, pr.eps, pr.alpha, pr.sigma2, Xsh, prec=args.prec,
                                   mean_out=mh, var_out=vh)
        m.free()

    for _ in range(max(3, args.warmup)):
        e2e_step()
    n_e2e = max(3, args.steps)
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        e2e_step()
    dt = (time.perf_counter() - t0) / n_e2e
    res["e2e"] = {"value": (pr.N + pr.Ns) / dt, "unit": UNIT,
                  "h2d_bytes_per_step": int((pr.N * pr.p + pr.N + pr.Ns * pr.p) * 8),
                  "d2h_bytes_per_step": int(pr.Ns * 2 * 8)}
    # ---- oracle: accuracy reference and the CPU baseline (full workload, one pass)
    t0 = time.perf_counter()
    mdl = O.fit(pr.X, pr.y, pr.n, pr.eps, pr.alpha, pr.sigma2)
    mo, vo = O.predict(mdl, pr.Xs)
    t_or = time.perf_counter() - t0
    res["cpu_baseline"] = {"value": (pr.N + pr.Ns) / t_or, "unit": UNIT, "cores": os.cpu_count(),
                           "kind": "oracle",
                           "sample": "the full workload once (200,000 train + 50,000 test points)"}
    res["fp64_gpu"] = {"value": (pr.N + pr.Ns) / (statistics.mean(ts) / 1e3), "unit": UNIT,
                       "ms_per_step": statistics.mean(ts),
                       "err_mean_rel_l2": O.relerr(m64, mo), "err_var_rel_l2": O.relerr(v64, vo)}
    res["accuracy"] = {"prec": args.prec, "err_mean_rel_l2": O.relerr(mmx, mo),
                       "err_var_rel_l2": O.relerr(vmx, vo), "tol_mean": 1e-4, "tol_var": 1e-3}

    return res


def batched_fit_bench(_lib, torch, dev):
    """The batched-fit workload: 256 independent GPs of uneven shape fitted by
    one gp_fit_batch (inputs resident on the device), against the same fits
    one after another."""
    from paper_2403_12797_gb300 import workloads as W
    probs = W.workload4(count=256, Ns=1)
    items = [(torch.from_numpy(pr.X).to(dev), torch.from_numpy(pr.y).to(dev), pr.n, pr.eps, pr.alpha,
              pr.sigma2) for pr in probs]
    points = sum(pr.X.shape[0] for pr in probs)
    for m in _lib.fit_batch(items):  # tunes the plan for this batch, warms the pool
        m.free()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    models = _lib.fit_batch(items)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    graph, k = _lib.batch_info()
    for m in models:
        m.free()
    t0 = time.perf_counter()
    for it in items:
        _lib.fit(*it).free()
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    return {"workload": "256 GPs: N log-uniform [1e3, 2e5], p in {1,2,3,4}, M = n^p <= 1024, "
                        "mixed precision, inputs on the device",
            "points": points, "ms": t_batch * 1e3, "points_per_s": points / t_batch,
            "sequential_ms": t_seq * 1e3, "sequential_points_per_s": points / t_seq,
            "speedup": t_seq / t_batch, "one_graph": bool(graph), "tuned_k": k}


def serving_bench(_lib, torch, dev):
    """The serving workload: 64 resident models (p in {2,3,4}, M <= 2048, N up
    to 5e5, fitted by one batched fit); a closed-loop burst gives the
    saturating request rate, then open-loop Poisson streams at 50 % and 80 %
    of it (predict sizes log-uniform on [1, 65536], 5 % refits with N
    log-uniform on [1e4, 5e5]) give p50/p99 latency and throughput."""
    from paper_2403_12797_gb300 import workloads as W
    mods = W.workload5_models(count=64)
    models = _lib.fit_batch([(pr.X, pr.y, pr.n, pr.eps, pr.alpha, pr.sigma2) for pr in mods])
    n_esc = sum(1 for m in models if m.gram_fp64)
    out = {"workload": "64 resident models: p in {2,3,4}, M <= 2048, N log-uniform [1e4, 5e5]; "
                       "predict sizes log-uniform [1, 65536], 5 % refits (N log-uniform [1e4, 5e5])",
           "models_fit_points": sum(pr.X.shape[0] for pr in mods),
           "models_gram_fp64": n_esc}
    with _lib.Server(slots=8) as srv:
        ids = [srv.add_model(m) for m in models]
        # closed loop: a burst of the same request mix (5 % refits) submitted at once
        burst = W.workload5_stream(mods, 200, 1e9, refit_frac=0.05, seed=1)
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
                             "peak_inflight": st["peak_inflight"]}
        out["refits_gram_fp64"] = sum(1 for i in ids if _lib.lib().gp_model_flags(srv.model_handle(i)) & 1)
        for frac in (0.5, 0.8):
            rate = frac * sat_rate
            stream = W.workload5_stream(mods, max(20, int(rate * 3.0)), rate, refit_frac=0.05, seed=2)
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
                "points_per_s": st["points_per_s"], "peak_inflight": st["peak_inflight"]}
    return out


def run_sweep(args):
    """The paper's own timing sweep (Sec. 3; row f4): y = sum_i cos(x_i) + nu
    on N = 10,000 training and 1,000 test points for p in {1, 2, 4} over a
    range of n, each fit + predict timed end to end as the paper times it
    (host arrays in and out: allocation and copies inside), median of
    --steps runs after --warmup. One JSON line; not part of the default run."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np
    from paper_2403_12797_gb300 import _lib, workloads as W
    grid = {1: (10, 50, 100, 200, 400), 2: (5, 10, 15, 20, 30), 4: (3, 5, 7, 9, 11)}
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
            rows.append({"p": p, "n": n, "M": n ** p, "ms": t * 1e3,
                         "points_per_s": (pr.N + pr.Ns) / t})
    print(json.dumps({"metric": "paper sweep: fit+predict time, host arrays in and out",
                      "unit": "ms", "prec": args.prec, "data": "synthetic",
                      "config": {"workload": "y = sum cos(x_i) + 0.1 noise, x~U[-1,1]^p, "
                                             "N = 10,000 train, 1,000 test points"},
                      "steps": args.steps, "warmup": args.warmup, "rows": rows}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--quick", action="store_true", help="skip the comparisons (profiling runs)")
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
