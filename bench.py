"""Benchmark: LD subdomain bounds/s on synthetic CIFAR-shaped convnets.

One step = one pass of the whole bounding path over one batch of synthetic
subdomains: interval bounds of the root box (ld_intermediate_bounds), the
LD bound of every subdomain after T Adam iterations with CROWN
initialisation and the FP64 final bound (ld_bound), and the Danskin adjoint
of the bounds (ld_bound_backward).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload base|wide|deep]
                    [--impl ours|reference]

`value` is whole-job bounds/s with inputs resident in HBM, timed with CUDA
events per step, L2 flushed (a 512 MB write) between steps; `e2e` is the
same metric through the C ABI with host buffers and the host<->device copies
inside the timed region.  `--impl reference` times the FP64 CPU oracle on a
bounded sample of the same workload.  For N > 1 (torchrun), every rank
bounds its own batch of subdomains (weak scaling, no collective on the data
path); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (net, subdomains per GPU, iterations, split depth range, eps range)
    "base": ("base", 256, 100, (0, 8), (1 / 255, 8 / 255)),
    "wide": ("wide", 2048, 100, (0, 20), (1 / 255, 8 / 255)),
    "deep": ("deep", 128, 100, (0, 8), (1 / 255, 8 / 255)),
}
METRIC = "LD subdomain bounds/s on Base/Wide/Deep convnets, bf16 vs fp32 at ≤1e-3 gap"

# DRAM bytes (read + write) of one launch of the iterations, from ncu captures
# of the current kernels (profiles/); keyed by (workload, precision, engine,
# tile, threads per CTA, subdomains, iterations).  Only entries whose kernels have not changed since
# the capture are listed.
TRAFFIC = {
    # fused_kernel<2, 512>, one launch (CROWN start + 100 iterations): profiles/fused_kernel_base256.md
    ("base", "fp32", "fused", 2, 512, 256, 100): 8.02e6,
    # the seven launches of one BF16 iteration x 100 (cold-cache capture): profiles/tc_kernels_wide2048_bf16.md
    ("wide", "bf16", "tensor-core bf16", 0, 0, 2048, 100): 4.415e10,
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="base", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--subdomains", type=int, default=0, help="override subdomains per GPU (profiling runs)")
    ap.add_argument("--iters", type=int, default=0, help="override Adam iterations (profiling runs)")
    ap.add_argument("--engine", default="auto", choices=["auto", "layerwise", "fused"])
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--cta-threads", type=int, default=0, choices=[0, 256, 512])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16"],
                    help="arithmetic of the Adam iterations (the final bound is FP64 either way)")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the second leg (the other precision on the same inputs, with the bound gap)")
    ap.add_argument("--sweep", action="store_true",
                    help="batch-size x iterations sweep on the Deep net with 32 properties, BF16 and FP32 "
                         "(one JSON line per point; not the benchmark line)")
    ap.add_argument("--sweep-b", default="64,128,256,512,1024,2048,4096,8192")
    ap.add_argument("--sweep-t", default="50,200,500")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self, which):
        """Host time of the start or end of the timed region (samples outside are dropped)."""
        setattr(self, which, time.time())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t0, t1 = getattr(self, "t_start", 0.0), getattr(self, "t_end", float("inf"))
        for t, ln in self.lines:
            if not (t0 <= t <= t1 + 0.06):
                continue
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def peak_value(d, key_candidates, default):
    for k in key_candidates:
        if k in d and isinstance(d[k], (int, float)):
            return float(d[k])
    for v in d.values():
        if isinstance(v, dict):
            for k in key_candidates:
                if k in v and isinstance(v[k], (int, float)):
                    return float(v[k])
    return default


def macs_per_pass(specs):
    """Multiply-accumulates of one forward pass of the canonical-form net
    (the last layer folded to one output)."""
    total = 0
    for i, s in enumerate(specs):
        n_out = 1 if i == len(specs) - 1 else s.n_out
        if s.kind == "fc":
            total += n_out * s.n_in
        else:
            cout, cin, kh, kw = s.W.shape
            total += s.n_out * cin * kh * kw
    return total


def workload_config(wl, N, B, T, world):
    """The `config` object of the bench line (both arms)."""
    return {"workload": f"{wl['net']} convnet ({N} ReLUs), {B} subdomains/GPU, split depth "
                        f"{wl['depth'][0]}-{wl['depth'][1]}, T={T} Adam iterations, CROWN init, FP64 final "
                        f"bound, Danskin backward",
            "subdomains_per_gpu": B, "iterations": T, "parallelism": f"replicas x{world}"}


def make_workload(name, rank):
    from paper_2104_06718_gb300 import synth
    net_name, B, T, depth, eps = WORKLOADS[name]
    specs = synth.make_convnet(net_name)
    l0, u0, c = synth.image_property(rank, eps)
    return dict(name=name, net=net_name, specs=specs, l0=l0[None], u0=u0[None], margin=c, B=B, T=T, depth=depth,
                rank=rank)


def cpu_baseline(wl, masks, lbk, ubk, budget_s=15.0, max_sub=None):
    """Time the FP64 oracle on a bounded sample (first subdomains, same T)."""
    import oracle
    from paper_2104_06718_gb300 import synth  # noqa: F401
    specs = wl["specs"]
    W, b = oracle.fold_margin(specs[-1].W.astype(np.float64), specs[-1].b.astype(np.float64),
                              np.asarray(wl["margin"], np.float64))
    layers = []
    for s in specs[:-1]:
        if s.kind == "fc":
            layers.append(oracle.Layer("fc", s.W, s.b))
        else:
            layers.append(oracle.Layer("conv", s.W, s.b, in_shape=s.in_shape, stride=s.stride, pad=s.pad))
    layers.append(oracle.Layer("fc", W.astype(np.float32), b.astype(np.float32)))
    on = oracle.Net(layers)
    T = wl["T"]
    # calibrate: one subdomain, then size the sample to the budget
    t0 = time.perf_counter()
    oracle.ld_bound(on, wl["l0"].astype(np.float64), wl["u0"].astype(np.float64), lbk.astype(np.float64),
                    ubk.astype(np.float64), None, masks[:2], T)
    per = (time.perf_counter() - t0) / 2
    n = int(max(2, min(masks.shape[0], budget_s / max(per, 1e-6))))
    if max_sub:
        n = min(n, max_sub)
    t0 = time.perf_counter()
    oracle.ld_bound(on, wl["l0"].astype(np.float64), wl["u0"].astype(np.float64), lbk.astype(np.float64),
                    ubk.astype(np.float64), None, masks[:n], T)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "bounds/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"first {n} of {masks.shape[0]} subdomains of the {wl['name']} workload, T={T}, FP64 NumPy/SciPy "
                      f"(dense BLAS may use all {os.cpu_count()} cores; sparse conv products are single-threaded)"}


def run_reference(args):
    world, rank, local = dist_env()
    if rank != 0:
        return 0
    from paper_2104_06718_gb300 import synth
    import oracle
    wl = make_workload(args.workload, 0)
    specs = wl["specs"]
    W, b = oracle.fold_margin(specs[-1].W.astype(np.float64), specs[-1].b.astype(np.float64),
                              np.asarray(wl["margin"], np.float64))
    layers = []
    for s in specs[:-1]:
        layers.append(oracle.Layer("conv", s.W, s.b, in_shape=s.in_shape, stride=s.stride, pad=s.pad)
                      if s.kind == "conv" else oracle.Layer("fc", s.W, s.b))
    layers.append(oracle.Layer("fc", W.astype(np.float32), b.astype(np.float32)))
    on = oracle.Net(layers)
    lb, ub = oracle.ibp_bounds(on, wl["l0"].astype(np.float64), wl["u0"].astype(np.float64))
    lbk = np.concatenate([lb[k] for k in range(1, on.n)], axis=1)
    ubk = np.concatenate([ub[k] for k in range(1, on.n)], axis=1)
    amb = np.nonzero((lbk[0] < 0) & (ubk[0] > 0))[0]
    masks = synth.split_masks(lbk.shape[1], wl["B"], amb, wl["depth"], block=0)
    # each step: a bounded sample of the workload (same T, first S subdomains)
    t0 = time.perf_counter()
    oracle.ld_bound(on, wl["l0"].astype(np.float64), wl["u0"].astype(np.float64), lbk, ubk, None, masks[:2], wl["T"])
    per = (time.perf_counter() - t0) / 2
    budget_total = 120.0
    S = int(max(2, min(wl["B"], budget_total / max(per, 1e-6) / max(args.steps + args.warmup, 1))))
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.ld_bound(on, wl["l0"].astype(np.float64), wl["u0"].astype(np.float64), lbk, ubk, None, masks[:S],
                        wl["T"])
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = S * len(times) / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "bounds/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / max(len(times), 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {**workload_config(wl, lbk.shape[1], wl["B"], wl["T"], args.gpus),
                       "precision": "fp64 oracle (iterations and final bound)",
                       "oracle_sample": f"first {S} of {wl['B']} subdomains per step (the bound only: no IBP or "
                                        "backward in the timed region)"},
            "cpu_baseline": {"value": value, "unit": "bounds/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"first {S} of {wl['B']} subdomains per step, T={wl['T']}, FP64 NumPy/SciPy"},
            "e2e": {"value": value, "unit": "bounds/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_2104_06718_gb300 import build as ldbuild
    if rank == 0 or world == 1:
        ldbuild.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_2104_06718_gb300 import binding as ldb
    from paper_2104_06718_gb300 import synth
    wl = make_workload(args.workload, rank)
    if args.subdomains:
        wl["B"] = args.subdomains
    if args.iters:
        wl["T"] = args.iters
    B, T = wl["B"], wl["T"]
    net = ldb.Net(wl["specs"], margin=wl["margin"])
    net.reserve(B)
    dev = torch.device("cuda", torch.cuda.current_device())
    l0 = torch.as_tensor(wl["l0"], device=dev)
    u0 = torch.as_tensor(wl["u0"], device=dev)
    lbk, ubk = ldb.ld_intermediate_bounds(net, l0, u0)
    lb_h, ub_h = lbk.cpu().numpy(), ubk.cpu().numpy()
    amb = np.nonzero((lb_h[0] < 0) & (ub_h[0] > 0))[0]
    masks_np = synth.split_masks(net.N, B, amb, wl["depth"], block=rank)
    masks = torch.as_tensor(masks_np, device=dev)
    ones = torch.ones(B, dtype=torch.float64, device=dev)
    opts = ldb.Options(engine=args.engine, tile=args.tile, cta_threads=args.cta_threads, precision=args.precision)

    def step():
        lk, uk = ldb.ld_intermediate_bounds(net, l0, u0)
        out, rho = ldb.ld_bound(net, l0, u0, lk, uk, None, masks, n_iters=T, opts=opts, return_rho=True)
        g = ldb.ld_bound_backward(net, l0, u0, lk, uk, rho, grad_out=ones, masks=masks)
        return out, g

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    engine, tile, threads = net.tuned(B)
    if args.precision == "bf16":
        engine, tile, threads = "tensor-core bf16", 0, 0
    elif args.engine != "auto":
        engine, tile, threads = args.engine, args.tile, args.cta_threads
    # ---- device-resident timing
    sampler = ClockSampler(torch.cuda.current_device())
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.5)  # nvidia-smi takes a moment to report; only samples inside the timed region count
    sampler.mark("t_start")
    net.profile(True)
    net.profile_read("iter", reset=True)
    launches0 = ldb.launch_count()
    times = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out, g = step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    sampler.mark("t_end")
    launches = ldb.launch_count() - launches0
    iter_ms, iter_n = net.profile_read("iter")
    final_ms, final_n = net.profile_read("final")
    init_ms, _ = net.profile_read("init")
    ibp_ms, _ = net.profile_read("ibp")
    bwd_ms, _ = net.profile_read("backward", reset=True)
    net.profile(False)
    clocks = sampler.stop()
    t_local = sum(times) / 1000.0
    # ---- the other precision on the same inputs: bounds/s and the bound gap
    compare = None
    if not args.no_compare:
        other = "bf16" if args.precision == "fp32" else "fp32"
        o2 = ldb.Options(engine=args.engine, tile=args.tile, cta_threads=args.cta_threads, precision=other)

        def step2():
            lk, uk = ldb.ld_intermediate_bounds(net, l0, u0)
            o_, r_ = ldb.ld_bound(net, l0, u0, lk, uk, None, masks, n_iters=T, opts=o2, return_rho=True)
            g_ = ldb.ld_bound_backward(net, l0, u0, lk, uk, r_, grad_out=ones, masks=masks)
            return o_, g_

        for _ in range(args.warmup):
            step2()
        torch.cuda.synchronize()
        t2 = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out2, _ = step2()
            e1.record(stream)
            e1.synchronize()
            t2.append(e0.elapsed_time(e1))
        a32 = (out if args.precision == "fp32" else out2).cpu().numpy()
        a16 = (out2 if args.precision == "fp32" else out).cpu().numpy()
        fin = np.isfinite(a32) & np.isfinite(a16)
        rel = np.abs(a16[fin] - a32[fin]) / np.maximum(np.abs(a32[fin]), 1.0)
        signed = (a32[fin] - a16[fin]) / np.maximum(np.abs(a32[fin]), 1.0)
        compare = {"precision": other, "value": B * args.steps / (sum(t2) / 1000.0), "unit": "bounds/s",
                   "ms_per_step": sum(t2) / args.steps,
                   "bf16_vs_fp32_gap": {"median": float(np.median(rel)), "p99": float(np.percentile(rel, 99)),
                                        "max": float(rel.max()), "mean_fp32_minus_bf16": float(signed.mean()),
                                        "definition": "|q_bf16 - q_fp32| / max(|q_fp32|, 1) per subdomain, same "
                                                      "inputs and T; the bounds are FP64-evaluated at each run's rho"}}
    # ---- end to end through the C ABI with host buffers
    h_l0 = torch.as_tensor(wl["l0"]).pin_memory()
    h_u0 = torch.as_tensor(wl["u0"]).pin_memory()
    h_masks = torch.as_tensor(masks_np).pin_memory()
    h_out = torch.empty(B, dtype=torch.float64).pin_memory()
    h_gW = torch.empty(net.n_weights, dtype=torch.float32).pin_memory()
    h2d = h_l0.numel() * 4 + h_u0.numel() * 4 + h_masks.numel()
    d2h = B * 8 + net.n_weights * 4

    def e2e_step():
        d_l0 = h_l0.to(dev, non_blocking=True)
        d_u0 = h_u0.to(dev, non_blocking=True)
        d_m = h_masks.to(dev, non_blocking=True)
        lk, uk = ldb.ld_intermediate_bounds(net, d_l0, d_u0)
        out, rho = ldb.ld_bound(net, d_l0, d_u0, lk, uk, None, d_m, n_iters=T, opts=opts, return_rho=True)
        gg = ldb.ld_bound_backward(net, d_l0, d_u0, lk, uk, rho, grad_out=ones, masks=d_m)
        h_out.copy_(out, non_blocking=True)
        h_gW.copy_(gg["gW"], non_blocking=True)

    etimes = []
    if not args.no_e2e:
        e2e_step()
        torch.cuda.synchronize()
    for _ in range(0 if args.no_e2e else args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e2e_step()
        e1.record(stream)
        e1.synchronize()
        etimes.append(e0.elapsed_time(e1))
    te_local = sum(etimes) / 1000.0 if etimes else float("nan")
    if world > 1:
        from paper_2104_06718_gb300.replicas import max_over_ranks
        t_all, te_all = max_over_ranks([t_local, te_local], device=dev)
        torch.distributed.barrier()
    else:
        t_all, te_all = t_local, te_local
    total_bounds = B * args.steps * world
    value = total_bounds / t_all
    e2e_value = total_bounds / te_all
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0
    peaks, peak_src = measured_peaks()
    # Roofline of the dominant launch: the Adam iterations of one step (the
    # fused engine: one kernel; the layerwise and BF16 engines: one graph
    # launch).  Algorithmic work per subdomain-iteration: two linear passes of
    # `macs` multiply-adds (2 FLOP each), and, where the dual state streams,
    # rho, m, v read and written in FP32 (24 B per ReLU) plus the 2-bit split
    # mask (0.25 B per ReLU).  The fused engine keeps rho, m, v in shared
    # memory for the whole launch, so its bound is the FP32 pipe ("alu", peak
    # derived from unit counts and the maximum clock); the other engines
    # stream the state through HBM ("hbm", the measured copy bandwidth).
    avg_launch_s = (iter_ms / max(iter_n, 1)) / 1000.0
    bytes_per_launch = B * T * net.N * 24.25
    achieved_gbs = bytes_per_launch / avg_launch_s / 1e9
    hbm_peak = peak_value(peaks, ["hbm_gbs", "hbm_GBs", "hbm"], 6800.0)
    macs = macs_per_pass(wl["specs"])
    flops_per_launch = B * T * 2 * 2 * macs
    achieved_tflops = flops_per_launch / avg_launch_s / 1e12
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    max_mhz = clocks.get("sm_max_mhz") or 2070.0
    alu_peak = sm_count * 128 * 2 * max_mhz * 1e6 / 1e12   # FP32 FMA lanes x 2 FLOP x clock
    bf16_peak = peak_value(peaks, ["bf16_tflops_sustained", "bf16_tflops"], 1700.0)
    hbm_obj = {"achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": achieved_gbs / hbm_peak,
               "peak_source": f"{peak_src} copy bandwidth",
               "work_per_launch": f"{B} subdomains x {T} iterations x {net.N} ReLUs x 24.25 B "
                                  "(rho, m, v read + write FP32; 2-bit mask)"}
    alu_obj = {"achieved": achieved_tflops, "peak": alu_peak, "unit": "TFLOP/s", "frac": achieved_tflops / alu_peak,
               "peak_source": f"derived: {sm_count} SMs x 128 FP32 FMA/clk x 2 FLOP x {max_mhz:.0f} MHz",
               "work_per_launch": f"{B} x {T} x 2 passes x {macs} MAC x 2 FLOP",
               "frac_of_bf16_tensor_peak": achieved_tflops / bf16_peak}
    resident = engine == "fused"
    main = alu_obj if resident else hbm_obj
    roofline = {"bound": "alu" if resident else "hbm", "achieved": main["achieved"], "peak": main["peak"],
                "unit": main["unit"], "frac": main["frac"],
                "traffic": TRAFFIC.get((wl["name"], args.precision, engine, tile, threads, B, T)),
                "kernel": f"fused iterations (tile {tile}, {threads or 256} threads per CTA; rho, m, v resident "
                          "in shared memory)" if resident else f"{engine or 'auto'} iterations (one graph launch)",
                "avg_launch_ms": iter_ms / max(iter_n, 1),
                "peak_source": main["peak_source"], "work_per_launch": main["work_per_launch"],
                "other": {"hbm": hbm_obj} if resident else {"alu": alu_obj},
                "l2_note": "the dual state of this workload fits in the 129 MB L2" if B * net.N * 24.25 < 100e6
                           else "the dual state exceeds L2 and streams from HBM"}
    line = {
        "metric": METRIC, "value": value, "unit": "bounds/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * t_all / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16" if args.precision == "bf16" else "f32",
        "data": "synthetic",
        "config": {**workload_config(wl, net.N, B, T, world),
                   "precision": ("bf16 GEMM operands, fp32 accumulation and dual state" if args.precision == "bf16"
                                 else "fp32") + " iterations, fp64 final",
                   "l2": "flushed between steps (512 MB write)"},
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": "bounds/s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "roofline": roofline,
        "phases_ms_per_step": {"ibp": ibp_ms / args.steps, "init": init_ms / args.steps,
                               "iterations": iter_ms / args.steps, "final_fp64": final_ms / args.steps,
                               "backward": bwd_ms / args.steps},
        "engine": {"engine": engine, "tile": tile, "cta_threads": threads},
        "compare": compare,
        "peaks_source": peak_src,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, masks_np, lb_h, ub_h)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_sweep(args):
    """Deep net, 32 properties (eps ~ U[1/255, 16/255], one margin vector),
    B/32 subdomains per property with split depth 0-20, for every batch size
    and iteration count: bounds/s of BF16 and FP32 iterations (FP64 final
    bound either way) and the BF16-vs-FP32 gap on the same inputs."""
    import torch
    torch.cuda.set_device(0)
    from paper_2104_06718_gb300 import build as ldbuild
    ldbuild.build()
    from paper_2104_06718_gb300 import binding as ldb
    from paper_2104_06718_gb300 import synth
    n_props = 32
    specs = synth.make_convnet("deep")
    boxes = [synth.image_property(p, (1 / 255, 16 / 255)) for p in range(n_props)]
    margin = boxes[0][2]
    net = ldb.Net(specs, margin=margin)
    dev = torch.device("cuda", 0)
    l0 = torch.as_tensor(np.stack([b[0] for b in boxes]), device=dev)
    u0 = torch.as_tensor(np.stack([b[1] for b in boxes]), device=dev)
    lbk, ubk = ldb.ld_intermediate_bounds(net, l0, u0)
    lb_h, ub_h = lbk.cpu().numpy(), ubk.cpu().numpy()
    Bs = [int(x) for x in args.sweep_b.split(",")]
    Ts = [int(x) for x in args.sweep_t.split(",")]
    net.reserve(max(Bs))
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for B in Bs:
        per = B // n_props
        prop = np.repeat(np.arange(n_props, dtype=np.int32), per)
        parts = []
        for p in range(n_props):
            amb = np.nonzero((lb_h[p] < 0) & (ub_h[p] > 0))[0]
            parts.append(synth.split_masks(net.N, per, amb, (0, 20), block=p))
        masks = torch.as_tensor(np.concatenate(parts), device=dev)
        prop_d = torch.as_tensor(prop, device=dev)
        amb_counts = []
        for p in range(n_props):
            m = np.concatenate(parts)[p * per:(p + 1) * per]
            a = (lb_h[p] < 0) & (ub_h[p] > 0)
            amb_counts.append((a[None, :] & (m == 0)).sum(axis=1))
        amb_counts = np.concatenate(amb_counts)
        for T in Ts:
            res = {}
            for prec in ("fp32", "bf16"):
                opts = ldb.Options(precision=prec)
                for _ in range(max(args.warmup, 1)):
                    out = ldb.ld_bound(net, l0, u0, lbk, ubk, prop_d, masks, n_iters=T, opts=opts)
                torch.cuda.synchronize()
                times = []
                for _ in range(args.steps):
                    flush.fill_(1.0)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    out = ldb.ld_bound(net, l0, u0, lbk, ubk, prop_d, masks, n_iters=T, opts=opts)
                    e1.record(stream)
                    e1.synchronize()
                    times.append(e0.elapsed_time(e1))
                res[prec] = (B / (statistics.median(times) / 1000.0), out.cpu().numpy(), net.tuned(B))
            a32, a16 = res["fp32"][1], res["bf16"][1]
            fin = np.isfinite(a32) & np.isfinite(a16)
            rel = np.abs(a16[fin] - a32[fin]) / np.maximum(np.abs(a32[fin]), 1.0)
            print(json.dumps({"sweep": "deep", "subdomains": B, "iterations": T, "properties": n_props,
                              "fp32_bounds_per_s": res["fp32"][0], "bf16_bounds_per_s": res["bf16"][0],
                              "bf16_speedup": res["bf16"][0] / res["fp32"][0],
                              "fp32_engine": list(res["fp32"][2]),
                              "gap_median": float(np.median(rel)) if rel.size else None,
                              "gap_max": float(rel.max()) if rel.size else None,
                              "ambiguous_relus": {"min": int(amb_counts.min()), "median": float(np.median(amb_counts)),
                                                  "max": int(amb_counts.max())}}), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.sweep:
        return run_sweep(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
