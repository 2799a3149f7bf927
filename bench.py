"""Benchmark: LD subdomain bounds/s on synthetic CIFAR-shaped convnets.

One step = one pass of the whole bounding path over one batch of synthetic
subdomains: interval bounds of the root box (ld_intermediate_bounds), the
LD bound of every subdomain after T Adam iterations with CROWN
initialisation and the FP64 final bound (ld_bound), and the Danskin adjoint
of the bounds (ld_bound_backward).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload base|wide|deep|tiny]
                    [--precision fp32|bf16] [--impl ours|reference] [--no-configs]

The line's `value` is the headline workload (default: Base convnet, 256
subdomains, T = 100, FP32 iterations): whole-job bounds/s with inputs
resident in HBM, timed with CUDA events per step, L2 flushed (a 512 MB write)
between steps; `e2e` is the same metric through the C ABI with host buffers
and the host<->device copies inside the timed region.  The `configs` object
holds the metric's other configurations measured in the same run (Base with
BF16 iterations, Wide 2048 and Deep 128 with FP32 and BF16 iterations, the
Tiny MLP), each with its bounds/s, its own clocks and roofline fraction, and
its bound gap against the FP64 CPU oracle on a sample of its subdomains.
`cpu_baseline` and `--impl reference` time the FP64 CPU oracle on a bounded
sample of the same workload.  For N > 1 (torchrun), every rank bounds its
own batch of subdomains (weak scaling, no collective on the data path); the
time is the max over ranks.
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
    "tiny": ("tiny", 1, 200, (0, 0), None),
}
# The metric's other configurations, measured in the same run and reported in
# the line's `configs` object: key -> (workload, precision of the iterations).
CONFIGS = {
    "base256_bf16": ("base", "bf16"),
    "wide2048_fp32": ("wide", "fp32"),
    "wide2048_bf16": ("wide", "bf16"),
    "deep128_fp32_bwd": ("deep", "fp32"),
    "deep128_bf16": ("deep", "bf16"),
    "tiny_mlp_fp32": ("tiny", "fp32"),
}
METRIC = "LD subdomain bounds/s on Base/Wide/Deep convnets, bf16 vs fp32 at ≤1e-3 gap"

# DRAM bytes (read + write) of one launch of the iterations, from ncu captures;
# keyed by (workload, precision, engine, tile, threads per CTA, subdomains,
# iterations), each with the digest of that engine's sources at the capture
# (kernel_digest(engine)).  An entry whose digest differs from the current
# sources is not reported (the kernel changed since the capture).
TRAFFIC = {
    # ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum of one launch of the fused kernels
    # (fused_kernel<2, 512, 0|1> on Base, <1, 512, 0|1> on Wide and Deep): read + write
    ("base", "fp32", "fused", 2, 512, 256, 100): ("f3512387ae4d", 8013568),
    ("base", "bf16", "fused tensor-core bf16", 2, 512, 256, 100): ("b20cd24da710", 8575232),
    ("wide", "fp32", "fused", 1, 512, 2048, 100): ("f3512387ae4d", 119097600 + 98118144),
    ("deep", "fp32", "fused", 1, 512, 128, 100): ("f3512387ae4d", 8338688),
    ("deep", "bf16", "fused tensor-core bf16", 1, 512, 128, 100): ("b20cd24da710", 8386560),
    # the same metrics over the 7 launches of one iteration of the layer-wise tensor-core engine
    # (read 359.94 MB + write 75.89 MB) x the 100 iterations of its graph launch
    ("wide", "bf16", "tensor-core bf16", 0, 0, 2048, 100): ("81ea16f36381", (359940352 + 75886592) * 100),
}

# The sources each timed engine is compiled from (besides the shared header
# and the ABI header).
ENGINE_SOURCES = {"fused": ["ld_fused.cu", "ld_fused_impl.cuh"],
                  "fused tensor-core bf16": ["ld_fused_tc.cu", "ld_fused_impl.cuh", "ld_tcgen05.cuh"],
                  "tensor-core bf16": ["ld_tc.cu", "ld_tcgen05.cuh"], "layerwise": ["ld_passes.cu"]}


def kernel_digest(engine=None) -> str:
    """SHA-256 (first 12 hex digits) of the CUDA sources of the library, or,
    given an engine, of the sources that engine's kernels are built from."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2104_06718_gb300", "csrc")
    if engine is None:
        files = sorted(fn for fn in os.listdir(csrc) if fn.endswith((".cu", ".cuh", ".h")))
        paths = [(fn, os.path.join(csrc, fn)) for fn in files]
    else:
        files = ENGINE_SOURCES.get(engine, []) + ["ld_common.cuh"]
        paths = [(fn, os.path.join(csrc, fn)) for fn in files] + [("ld.h", os.path.join(ROOT, "include", "ld.h"))]
    h = hashlib.sha256()
    for fn, path in paths:
        h.update(fn.encode())
        with open(path, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="base", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--no-configs", action="store_true",
                    help="measure the headline workload only (profiling runs)")
    ap.add_argument("--config-steps", type=int, default=10, help="timed steps of each entry of `configs`")
    ap.add_argument("--subdomains", type=int, default=0, help="override subdomains per GPU (profiling runs)")
    ap.add_argument("--iters", type=int, default=0, help="override Adam iterations (profiling runs)")
    ap.add_argument("--engine", default="auto", choices=["auto", "layerwise", "fused"])
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--cta-threads", type=int, default=0, choices=[0, 256, 512])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16"],
                    help="arithmetic of the Adam iterations (the final bound is FP64 either way)")
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
    """Samples SM clocks and throttle reasons with nvidia-smi (every 50 ms)
    for the whole run; window(t0, t1) summarises the samples of one timed
    region."""

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
        time.sleep(0.5)  # nvidia-smi takes a moment to report

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def window(self, t0, t1):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.12)  # let the reader catch the samples of the window's end
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for t, ln in list(self.lines):
            if not (t0 <= t <= t1 + 0.06):
                continue
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons), "samples": len(sm)}

    def stop(self):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)


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


def make_workload(name, rank, B=0, T=0):
    from paper_2104_06718_gb300 import synth
    net_name, B0, T0, depth, eps = WORKLOADS[name]
    if net_name == "tiny":
        specs = synth.tiny_mlp(0)
        l0, u0 = synth.tiny_box(0)
        margin = None
    else:
        specs = synth.make_convnet(net_name)
        l0, u0, margin = synth.image_property(rank, eps)
        l0, u0 = l0[None], u0[None]
    return dict(name=name, net=net_name, specs=specs, l0=l0, u0=u0, margin=margin, B=B or B0, T=T or T0,
                depth=depth, rank=rank)


def ball_centre(wl):
    """Centre of the l2-ball variant of a workload: the midpoint of its box,
    [1, n0] float32 (the same array on both sides)."""
    return ((wl["l0"].astype(np.float64) + wl["u0"].astype(np.float64)) / 2).astype(np.float32)


def workload_config(wl, N, world, precision):
    """The `config` object of a bench line (both arms)."""
    net = "Tiny MLP 10-20-20-1" if wl["net"] == "tiny" else f"{wl['net']} convnet"
    return {"workload": f"{net} ({N} ReLUs), {wl['B']} subdomains/GPU, split depth {wl['depth'][0]}-"
                        f"{wl['depth'][1]}, T={wl['T']} Adam iterations, CROWN init, {precision} iterations, "
                        "FP64 final bound, Danskin backward",
            "subdomains_per_gpu": wl["B"], "iterations": wl["T"], "parallelism": f"replicas x{world}"}


# ----------------------------------------------------------------------------- oracle legs (CPU baseline)

def _outward_f32(lo, hi):
    l32 = lo.astype(np.float32)
    h32 = hi.astype(np.float32)
    l32 = np.where(l32.astype(np.float64) > lo, np.nextafter(l32, np.float32(-np.inf)), l32)
    h32 = np.where(h32.astype(np.float64) < hi, np.nextafter(h32, np.float32(np.inf)), h32)
    return l32.astype(np.float32), h32.astype(np.float32)


def oracle_problem(wl):
    """The workload as the FP64 oracle states it: the net with the margin
    folded in FP64, its interval bounds (rounded outward to float32, the
    form the library takes) and the split masks drawn from its own
    classification of the root-ambiguous ReLUs."""
    import oracle
    from paper_2104_06718_gb300 import synth
    specs = wl["specs"]
    layers = []
    for i, s in enumerate(specs):
        W, b = np.asarray(s.W, np.float64), np.asarray(s.b, np.float64)
        if i == len(specs) - 1 and wl["margin"] is not None:
            W, b = oracle.fold_margin(W, b, np.asarray(wl["margin"], np.float64))
        layers.append(oracle.Layer("conv", W, b, in_shape=s.in_shape, stride=s.stride, pad=s.pad)
                      if s.kind == "conv" else oracle.Layer("fc", W, b))
    on = oracle.Net(layers)
    if wl.get("ball_eps") is not None:
        from oracle import l2
        lb, ub = l2.ball_ibp_bounds(on, ball_centre(wl).astype(np.float64), np.array([wl["ball_eps"]], np.float64))
    else:
        lb, ub = oracle.ibp_bounds(on, wl["l0"].astype(np.float64), wl["u0"].astype(np.float64))
    lbk, ubk = _outward_f32(np.concatenate([lb[k] for k in range(1, on.n)], axis=1),
                            np.concatenate([ub[k] for k in range(1, on.n)], axis=1))
    amb = np.nonzero((lbk[0] < 0) & (ubk[0] > 0))[0]
    masks = synth.split_masks(lbk.shape[1], wl["B"], amb, wl["depth"], block=wl["rank"])
    return on, lbk, ubk, masks


def oracle_run(on, wl, lbk, ubk, masks):
    import oracle
    if wl.get("ball_eps") is not None:
        c = ball_centre(wl).astype(np.float64)
        out, _, _ = oracle.ld_bound(on, c, c, lbk.astype(np.float64), ubk.astype(np.float64), None, masks, wl["T"],
                                    ball_eps=np.array([wl["ball_eps"]], np.float64))
        return out
    out, _, _ = oracle.ld_bound(on, wl["l0"].astype(np.float64), wl["u0"].astype(np.float64), lbk.astype(np.float64),
                                ubk.astype(np.float64), None, masks, wl["T"])
    return out


def cpu_leg(wl, budget_s, run_gpu=None):
    """The FP64 oracle timed on a bounded sample of the workload (its first
    subdomains, same T), and, with run_gpu, the gap of the library's bounds
    on the same sample and the same oracle-side inputs."""
    on, lbk, ubk, masks = oracle_problem(wl)
    t0 = time.perf_counter()
    oracle_run(on, wl, lbk, ubk, masks[:1])
    per = time.perf_counter() - t0
    n = int(min(wl["B"], max(2, budget_s / max(per, 1e-6))))
    t0 = time.perf_counter()
    ref = oracle_run(on, wl, lbk, ubk, masks[:n])
    dt = time.perf_counter() - t0
    cpu = {"value": n / dt, "unit": "bounds/s", "cores": os.cpu_count(), "kind": "oracle",
           "sample": f"first {n} of {wl['B']} subdomains of the {wl['name']} workload"
                     f"{' over the l2 ball' if wl.get('ball_eps') is not None else ''}, T={wl['T']}, FP64 "
                     f"NumPy/SciPy (dense BLAS may use all {os.cpu_count()} cores; sparse conv products are "
                     "single-threaded)"}
    gaps = None
    if run_gpu is not None:
        gaps = {}
        fin = np.isfinite(ref)
        for prec, got in run_gpu(lbk, ubk, masks[:n]).items():
            assert np.array_equal(np.isfinite(got), fin)
            rel = np.abs(got[fin] - ref[fin]) / np.maximum(np.abs(ref[fin]), 1.0)
            gaps[prec] = {"median": float(np.median(rel)) if rel.size else None,
                          "max": float(rel.max()) if rel.size else None}
        gaps["definition"] = (f"|q_gpu - q_oracle| / max(|q_oracle|, 1) over the first {n} subdomains, same "
                              "oracle-side inputs and T; q_oracle = FP64 oracle (exact passes)")
    return cpu, gaps


# ----------------------------------------------------------------------------- the library's arm

class Bench:
    """One GPU's measurements: the workloads, their nets and the clock sampler."""

    def __init__(self, args, world, rank, dev):
        import torch
        from paper_2104_06718_gb300 import binding as ldb
        self.args, self.world, self.rank, self.dev = args, world, rank, dev
        self.torch, self.ldb = torch, ldb
        self.flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        self.stream = torch.cuda.current_stream()
        self.sampler = ClockSampler(torch.cuda.current_device())
        self.peaks, self.peak_src = measured_peaks()
        self.nets = {}

    def setup(self, name, B=0, T=0):
        """Workload, net (cached per workload) and device inputs."""
        from paper_2104_06718_gb300 import synth
        torch, ldb = self.torch, self.ldb
        wl = make_workload(name, self.rank, B, T)
        if name not in self.nets:
            self.nets[name] = ldb.Net(wl["specs"], margin=wl["margin"])
        net = self.nets[name]
        net.reserve(wl["B"])
        d = dict(wl=wl, net=net)
        d["l0"] = torch.as_tensor(wl["l0"], device=self.dev)
        d["u0"] = torch.as_tensor(wl["u0"], device=self.dev)
        lbk, ubk = ldb.ld_intermediate_bounds(net, d["l0"], d["u0"])
        lb_h, ub_h = lbk.cpu().numpy(), ubk.cpu().numpy()
        amb = np.nonzero((lb_h[0] < 0) & (ub_h[0] > 0))[0]
        d["masks_np"] = synth.split_masks(net.N, wl["B"], amb, wl["depth"], block=self.rank)
        d["masks"] = torch.as_tensor(d["masks_np"], device=self.dev)
        d["ones"] = torch.ones(wl["B"], dtype=torch.float64, device=self.dev)
        return d

    def opts(self, precision):
        a = self.args
        return self.ldb.Options(engine=a.engine, tile=a.tile, cta_threads=a.cta_threads, precision=precision)

    def step_fn(self, d, precision):
        ldb = self.ldb
        net, l0, u0, masks, ones, T = d["net"], d["l0"], d["u0"], d["masks"], d["ones"], d["wl"]["T"]
        opts = self.opts(precision)

        def step():
            lk, uk = ldb.ld_intermediate_bounds(net, l0, u0)
            out, rho = ldb.ld_bound(net, l0, u0, lk, uk, None, masks, n_iters=T, opts=opts, return_rho=True)
            g = ldb.ld_bound_backward(net, l0, u0, lk, uk, rho, grad_out=ones, masks=masks)
            return out, g
        return step

    def timed(self, fn, steps, warmup):
        """Warm-up, then `steps` steps timed with CUDA events on the launch
        stream, L2 flushed before each; returns (per-step ms, host window)."""
        torch = self.torch
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        if self.world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t0 = time.time()
        times = []
        for _ in range(steps):
            self.flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            fn()
            e1.record(self.stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        return times, (t0, time.time())

    def measure(self, d, precision, steps, warmup):
        """bounds/s, per-phase times, roofline and clocks of one workload."""
        ldb = self.ldb
        wl, net = d["wl"], d["net"]
        B, T = wl["B"], wl["T"]
        step = self.step_fn(d, precision)
        for _ in range(warmup):
            step()
        self.torch.cuda.synchronize()
        net.profile(True)
        for ph in ("iter", "final", "init", "ibp", "backward"):
            net.profile_read(ph, reset=True)
        launches0 = ldb.launch_count()
        times, win = self.timed(step, steps, 0)
        launches = ldb.launch_count() - launches0
        ph = {k: net.profile_read(k, reset=True) for k in ("iter", "final", "init", "ibp", "backward")}
        net.profile(False)
        out, _ = step()
        engine, tile, threads = net.tuned(B, precision)
        if self.args.engine != "auto":
            engine, tile, threads = self.args.engine, self.args.tile, self.args.cta_threads
        if precision == "bf16":
            engine = "fused tensor-core bf16" if engine == "fused" else "tensor-core bf16"
            if engine == "fused tensor-core bf16":
                threads = 512
            else:
                tile, threads = 0, 0
        return dict(times=times, window=win, launches=launches, phases=ph, out=out.cpu().numpy(),
                    engine=(engine, tile, threads),
                    roofline=self.roofline(wl, net, precision, ph["iter"], (engine, tile, threads)))

    def roofline(self, wl, net, precision, iter_ph, eng):
        """Roofline of the dominant launch: the Adam iterations of one step
        (the fused engine: one kernel; the layerwise and BF16 engines: one
        graph launch).  Algorithmic work per subdomain-iteration: two linear
        passes of `macs` multiply-adds (2 FLOP each), and, where the dual state
        streams, rho, m, v read and written in FP32 (24 B per ReLU) plus the
        2-bit split mask (0.25 B per ReLU).  The fused engine keeps rho, m, v in
        shared memory for the whole launch, so its bound is the FP32 pipe
        ("alu", peak derived from unit counts and the maximum clock); the other
        engines stream the state through HBM ("hbm", the measured copy
        bandwidth)."""
        B, T = wl["B"], wl["T"]
        iter_ms, iter_n = iter_ph
        avg_launch_s = (iter_ms / max(iter_n, 1)) / 1000.0
        bytes_per_launch = B * T * net.N * 24.25
        achieved_gbs = bytes_per_launch / avg_launch_s / 1e9
        hbm_peak = peak_value(self.peaks, ["hbm_gbs", "hbm_GBs", "hbm"], 6800.0)
        macs = macs_per_pass(wl["specs"])
        flops_per_launch = B * T * 2 * 2 * macs
        achieved_tflops = flops_per_launch / avg_launch_s / 1e12
        sm_count = self.torch.cuda.get_device_properties(self.dev).multi_processor_count
        max_mhz = peak_value(self.peaks, ["sm_max_mhz"], 2070.0)
        alu_peak = sm_count * 128 * 2 * max_mhz * 1e6 / 1e12   # FP32 FMA lanes x 2 FLOP x clock
        bf16_peak = peak_value(self.peaks, ["bf16_tflops"], 1900.0)
        engine, tile, threads = eng
        hbm_obj = {"achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": achieved_gbs / hbm_peak,
                   "peak_source": f"{self.peak_src} copy bandwidth",
                   "work_per_launch": f"{B} subdomains x {T} iterations x {net.N} ReLUs x 24.25 B "
                                      "(rho, m, v read + write FP32; 2-bit mask)"}
        alu_obj = {"achieved": achieved_tflops, "peak": alu_peak, "unit": "TFLOP/s",
                   "frac": achieved_tflops / alu_peak,
                   "peak_source": f"derived: {sm_count} SMs x 128 FP32 FMA/clk x 2 FLOP x {max_mhz:.0f} MHz",
                   "work_per_launch": f"{B} x {T} x 2 passes x {macs} MAC x 2 FLOP"}
        tensor_obj = {"achieved": achieved_tflops, "peak": bf16_peak, "unit": "TFLOP/s",
                      "frac": achieved_tflops / bf16_peak, "peak_source": f"{self.peak_src} bf16 dense (burst)",
                      "work_per_launch": alu_obj["work_per_launch"]}
        resident = engine in ("fused", "fused tensor-core bf16")
        tensor_main = engine == "fused tensor-core bf16"
        main = tensor_obj if tensor_main else (alu_obj if resident else hbm_obj)
        key = (wl["name"], precision, engine, tile, threads, B, T)
        tr = TRAFFIC.get(key)
        traffic = tr[1] if tr is not None and tr[0] == kernel_digest(engine) else None
        other = {"hbm": hbm_obj} if resident else {"alu": alu_obj}
        if tensor_main:
            other["alu"] = alu_obj
        elif precision == "bf16":
            other["tensor"] = tensor_obj
        if tensor_main:
            kernel = (f"fused tensor-core iterations ({tile} subdomains per 512-thread CTA; conv passes as tcgen05 "
                      "BF16 GEMMs from shared-memory shadows, rho, m, v resident in shared memory)")
        elif resident:
            kernel = f"fused iterations (tile {tile}, {threads or 256} threads per CTA; rho, m, v resident in shared memory)"
        else:
            kernel = f"{engine or 'auto'} iterations (one graph launch)"
        return {"bound": "tensor" if tensor_main else ("alu" if resident else "hbm"), "achieved": main["achieved"],
                "peak": main["peak"], "unit": main["unit"], "frac": main["frac"], "traffic": traffic,
                "kernel": kernel,
                "avg_launch_ms": iter_ms / max(iter_n, 1),
                "peak_source": main["peak_source"], "work_per_launch": main["work_per_launch"], "other": other,
                "l2_note": "the dual state of this workload fits in the 129 MB L2" if B * net.N * 24.25 < 100e6
                           else "the dual state exceeds L2 and streams from HBM"}

    def gap_runner(self, d, precisions):
        """GPU bounds of a sample of subdomains on the oracle's own inputs."""
        torch, ldb = self.torch, self.ldb
        net, wl = d["net"], d["wl"]

        def run(lbk, ubk, masks):
            res = {}
            for prec in precisions:
                out = ldb.ld_bound(net, d["l0"], d["u0"], torch.as_tensor(lbk, device=self.dev),
                                   torch.as_tensor(ubk, device=self.dev), None, torch.as_tensor(masks, device=self.dev),
                                   n_iters=wl["T"], opts=self.opts(prec))
                res[prec] = out.cpu().numpy()
            return res
        return run


def measure_ib(bn, args):
    """CROWN / WK layer-wise best intermediate bounds on the Base workload:
    time of the root bounds (one property) and of the bounds recomputed per
    subdomain after its splits (256 subdomains), and the LD bounds after
    T = 100 iterations on IBP root bounds and on the layer-wise best root
    bounds (same masks, drawn from the ReLUs ambiguous under both)."""
    torch, ldb = bn.torch, bn.ldb
    d = bn.setup("base")
    net, l0, u0, masks, wl = d["net"], d["l0"], d["u0"], d["masks"], d["wl"]
    res = {}
    for key, kw, steps in (("root_ms", {}, 20), ("per_subdomain_ms", {"masks": masks}, 3)):
        fn = lambda: ldb.ld_intermediate_bounds_propagated(net, l0, u0, rules="best", **kw)
        times, win = bn.timed(fn, steps, 2)
        res[key] = statistics.median(times)
        res[key.replace("_ms", "_clocks")] = bn.sampler.window(*win)
    lb_i, ub_i = ldb.ld_intermediate_bounds(net, l0, u0)
    lb_b, ub_b = ldb.ld_intermediate_bounds_propagated(net, l0, u0, rules="best")
    both = ((lb_b < 0) & (ub_b > 0))[0].cpu().numpy()
    from paper_2104_06718_gb300 import synth
    m2 = torch.as_tensor(synth.split_masks(net.N, wl["B"], np.nonzero(both)[0], wl["depth"], block=bn.rank),
                         device=bn.dev)
    o_i = ldb.ld_bound(net, l0, u0, lb_i, ub_i, None, m2, n_iters=wl["T"]).cpu().numpy()
    o_b = ldb.ld_bound(net, l0, u0, lb_b, ub_b, None, m2, n_iters=wl["T"]).cpu().numpy()
    fin = np.isfinite(o_i) & np.isfinite(o_b)
    amb = lambda lo, hi: int(((lo < 0) & (hi > 0)).sum().item())
    res.update({"subdomains": wl["B"], "rules": "layer-wise best of CROWN and WK",
                "ambiguous_relus_root": {"ibp": amb(lb_i, ub_i), "best": amb(lb_b, ub_b)},
                "ld_bound_mean_on_ibp": float(o_i[fin].mean()), "ld_bound_mean_on_best": float(o_b[fin].mean()),
                "ld_bound_improved_fraction": float(np.mean(o_b[fin] >= o_i[fin]))})
    return res


def measure_solvers(bn, args):
    """The three dual solvers on the Base workload with the layer-wise best
    CROWN/WK root bounds, at the iteration counts Sec. 8.2 tunes to roughly
    equal time (supergradient 160, proximal 100 with eta = 100 and no
    momentum, DSG+ 260): time per call (256 subdomains), bounds/s and the mean
    bound (the FP64 bound at the final duals; for DSG+ also its own d_O)."""
    ldb = bn.ldb
    d = bn.setup("base")
    net, l0, u0, masks = d["net"], d["l0"], d["u0"], d["masks"]
    lk, uk = ldb.ld_intermediate_bounds_propagated(net, l0, u0, rules="best")
    B = d["wl"]["B"]
    runs = {
        "supergradient_T160": lambda: ldb.ld_bound(net, l0, u0, lk, uk, None, masks, n_iters=160),
        "proximal_T100": lambda: ldb.ld_bound_proximal(net, l0, u0, lk, uk, None, masks, n_iters=100,
                                                       opts=ldb.ProxOptions(eta0=100.0, eta_end=100.0, mu=0.0)),
        "dsg_T260": lambda: ldb.ld_bound_dsg(net, l0, u0, lk, uk, None, masks, n_iters=260),
    }
    res = {"subdomains": B, "intermediate_bounds": "layer-wise best of CROWN and WK at the root"}
    for key, fn in runs.items():
        times, win = bn.timed(fn, 3, 1)
        out = fn()
        ms = statistics.median(times)
        entry = {"ms_per_call": ms, "bounds_per_s": B / (ms / 1000.0), "clocks": bn.sampler.window(*win)}
        if key.startswith("dsg"):
            dec, dd = (x.cpu().numpy() for x in out)
            fin = np.isfinite(dec)
            entry.update({"mean_bound_dec_dsg": float(dec[fin].mean()), "mean_bound_dsg": float(dd[fin].mean())})
        else:
            o = out.cpu().numpy()
            entry["mean_bound"] = float(o[np.isfinite(o)].mean())
        res[key] = entry
    return res


def measure_ball(bn, args, eps=0.1):
    """The Base workload over an l2 ball (Sec. 3.2.1) instead of the box:
    radius eps around the box centre, interval bounds over the ball, 256
    subdomains, T = 100, FP32 layer-wise iterations and the FP64 final bound
    (ld_bound_ball); time per call, bounds/s, and, in the CPU leg, the gap to
    the FP64 oracle on its own inputs."""
    torch, ldb = bn.torch, bn.ldb
    from paper_2104_06718_gb300 import synth
    d = bn.setup("base")
    net, wl = d["net"], dict(d["wl"], ball_eps=eps)
    c = torch.as_tensor(ball_centre(wl), device=bn.dev)
    e = torch.tensor([eps], dtype=torch.float32, device=bn.dev)
    lbk, ubk = ldb.ld_intermediate_bounds_ball(net, c, e)
    lb_h, ub_h = lbk.cpu().numpy(), ubk.cpu().numpy()
    amb = np.nonzero((lb_h[0] < 0) & (ub_h[0] > 0))[0]
    masks = torch.as_tensor(synth.split_masks(net.N, wl["B"], amb, wl["depth"], block=bn.rank), device=bn.dev)
    fn = lambda: ldb.ld_bound_ball(net, c, e, lbk, ubk, None, masks, n_iters=wl["T"])
    times, win = bn.timed(fn, 5, 2)
    ms = statistics.median(times)
    out = fn().cpu().numpy()
    res = {"subdomains": wl["B"], "iterations": wl["T"], "radius": eps, "ms_per_call": ms,
           "bounds_per_s": wl["B"] / (ms / 1000.0), "clocks": bn.sampler.window(*win),
           "ambiguous_relus_root": int(amb.size), "mean_bound": float(out[np.isfinite(out)].mean()),
           "engine": dict(zip(("engine", "tile", "cta_threads"), net.tuned(wl["B"], "fp32")))}
    if not args.no_cpu_baseline:
        def run(lbk_o, ubk_o, masks_o):
            got = ldb.ld_bound_ball(net, c, e, torch.as_tensor(lbk_o, device=bn.dev),
                                    torch.as_tensor(ubk_o, device=bn.dev), None,
                                    torch.as_tensor(masks_o, device=bn.dev), n_iters=wl["T"])
            return {"fp32": got.cpu().numpy()}
        res["cpu_baseline"], res["gap_vs_fp64_oracle"] = cpu_leg(wl, 3.0, run)
    return res


def measure_branching(bn, args):
    """Branching decisions for the 256 Base subdomains (SR, mSR, FSB: time per
    call) and one batched branch and bound run on a Base property (CROWN/WK
    root bounds, T = 50 per bound, 128 subdomains per step, a budget of 4096
    subdomains): status, subdomains bounded and their rate."""
    ldb = bn.ldb
    from paper_2104_06718_gb300 import bab
    d = bn.setup("base")
    net, l0, u0, masks = d["net"], d["l0"], d["u0"], d["masks"]
    lk, uk = ldb.ld_intermediate_bounds_propagated(net, l0, u0, rules="best")
    res = {"subdomains": d["wl"]["B"]}
    for rule in ("sr", "msr", "fsb"):
        fn = lambda: ldb.ld_branch(net, l0, u0, lk, uk, None, masks, rule=rule)
        times, _ = bn.timed(fn, 5, 1)
        res[f"{rule}_ms_per_call"] = statistics.median(times)
    # the synthetic margin property is false at the root of this random net
    # (an upper bound below zero); shift the folded output by delta so that
    # the root lower bound is below zero and the root upper bound above it,
    # and let branch and bound decide the shifted property
    from paper_2104_06718_gb300 import synth
    import torch
    specs, margin = d["wl"]["specs"], np.asarray(d["wl"]["margin"], np.float64)
    last = specs[-1]
    Wf = (margin @ np.asarray(last.W, np.float64))[None, :]
    bf = np.array([margin @ np.asarray(last.b, np.float64)])
    folded = list(specs[:-1]) + [synth.LayerSpec("fc", Wf.astype(np.float32), bf.astype(np.float32), last.in_shape)]
    one = torch.zeros((1, net.N), dtype=torch.int8, device=l0.device)
    fnet = ldb.Net(folded)
    lo, rho = ldb.ld_bound(fnet, l0, u0, lk, uk, None, one, n_iters=50, return_rho=True)
    ub = float(ldb.ld_upper_bound(fnet, l0, u0, lk, uk, rho, masks=one).min().item())
    lo = float(lo.min().item())
    delta = -lo - 0.25 * (ub - lo)
    shifted = list(specs[:-1]) + [synth.LayerSpec("fc", Wf.astype(np.float32), (bf + delta).astype(np.float32),
                                                  last.in_shape)]
    snet = ldb.Net(shifted)
    t0 = time.perf_counter()
    r = bab.verify(snet, d["wl"]["l0"][0], d["wl"]["u0"][0], lk, uk, T=50, batch=128, max_nodes=4096)
    dt = time.perf_counter() - t0
    res["bab"] = {"status": r.status, "subdomains_bounded": r.nodes, "branching_steps": r.iterations,
                  "lower": r.lower, "upper": r.upper, "seconds": dt, "subdomains_per_s": r.nodes / dt,
                  "root": {"lower": lo, "upper": ub, "delta": delta},
                  "setting": "FSB, T = 50 per bound (fused engine), 128 subdomains per step, budget 4096; "
                             "the margin property shifted by delta = -(lower + (upper - lower) / 4) at the root"}
    return res


def summarise(m, B, world):
    t = sum(m["times"]) / 1000.0
    ph = m["phases"]
    n = len(m["times"])
    return {"value": B * n * world / t, "unit": "bounds/s", "ms_per_step": 1000 * t / n, "steps": n,
            "phases_ms_per_step": {k: v[0] / n for k, v in ph.items()},
            "engine": {"engine": m["engine"][0], "tile": m["engine"][1], "cta_threads": m["engine"][2]},
            "gpu_launches": int(m["launches"]), "roofline": m["roofline"]}


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
    dev = torch.device("cuda", torch.cuda.current_device())
    bn = Bench(args, world, rank, dev)
    bn.sampler.start()
    d = bn.setup(args.workload, args.subdomains, args.iters)
    wl, net = d["wl"], d["net"]
    B, T = wl["B"], wl["T"]
    # ---- the headline workload, device-resident inputs
    m = bn.measure(d, args.precision, args.steps, args.warmup)
    clocks = bn.sampler.window(*m["window"])
    t_local = sum(m["times"]) / 1000.0
    # ---- end to end through the C ABI with host buffers
    h_l0 = torch.as_tensor(wl["l0"]).pin_memory()
    h_u0 = torch.as_tensor(wl["u0"]).pin_memory()
    h_masks = torch.as_tensor(d["masks_np"]).pin_memory()
    h_out = torch.empty(B, dtype=torch.float64).pin_memory()
    h_gW = torch.empty(net.n_weights, dtype=torch.float32).pin_memory()
    h2d = h_l0.numel() * 4 + h_u0.numel() * 4 + h_masks.numel()
    d2h = B * 8 + net.n_weights * 4
    opts = bn.opts(args.precision)

    def e2e_step():
        d_l0 = h_l0.to(dev, non_blocking=True)
        d_u0 = h_u0.to(dev, non_blocking=True)
        d_m = h_masks.to(dev, non_blocking=True)
        lk, uk = ldb.ld_intermediate_bounds(net, d_l0, d_u0)
        out, rho = ldb.ld_bound(net, d_l0, d_u0, lk, uk, None, d_m, n_iters=T, opts=opts, return_rho=True)
        gg = ldb.ld_bound_backward(net, d_l0, d_u0, lk, uk, rho, grad_out=d["ones"], masks=d_m)
        h_out.copy_(out, non_blocking=True)
        h_gW.copy_(gg["gW"], non_blocking=True)

    te_local = float("nan")
    if not args.no_e2e:
        etimes, _ = bn.timed(e2e_step, args.steps, 1)
        te_local = sum(etimes) / 1000.0
    if world > 1:
        from paper_2104_06718_gb300.replicas import max_over_ranks
        t_all, te_all = max_over_ranks([t_local, te_local], device=dev)
        torch.distributed.barrier()
    else:
        t_all, te_all = t_local, te_local
    total_bounds = B * args.steps * world
    # ---- the metric's other configurations (rank 0 of a single-GPU run)
    configs = None
    if not args.no_configs and world == 1:
        configs = {}
        for key, (name, prec) in CONFIGS.items():
            dc = bn.setup(name)
            mc = bn.measure(dc, prec, args.config_steps, max(args.warmup, 2))
            entry = summarise(mc, dc["wl"]["B"], 1)
            entry.update({"precision": prec, "clocks": bn.sampler.window(*mc["window"]),
                          "config": workload_config(dc["wl"], dc["net"].N, 1, prec)})
            if not args.no_cpu_baseline:
                cpu, gaps = cpu_leg(dc["wl"], 3.0, bn.gap_runner(dc, [prec]))
                entry["cpu_baseline"] = cpu
                entry["gap_vs_fp64_oracle"] = gaps
            configs[key] = entry
            if prec == "bf16":
                # the same workload's FP32 run for the BF16-vs-FP32 gap over the whole batch
                f32 = bn.measure(dc, "fp32", 1, 0)["out"]
                a16 = mc["out"]
                fin = np.isfinite(f32) & np.isfinite(a16)
                rel = np.abs(a16[fin] - f32[fin]) / np.maximum(np.abs(f32[fin]), 1.0)
                entry["gap_vs_fp32_gpu"] = {"median": float(np.median(rel)), "p99": float(np.percentile(rel, 99)),
                                            "max": float(rel.max()),
                                            "definition": "|q_bf16 - q_fp32| / max(|q_fp32|, 1) per subdomain, "
                                                          "same inputs and T, whole batch"}
        configs["intermediate_bounds_base256"] = measure_ib(bn, args)
        configs["solvers_base256"] = measure_solvers(bn, args)
        configs["branching_base256"] = measure_branching(bn, args)
        configs["l2_ball_base256"] = measure_ball(bn, args)
    bn.sampler.stop()
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0
    head = summarise(m, B, world)
    line = {
        "metric": METRIC, "value": total_bounds / t_all, "unit": "bounds/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * t_all / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16" if args.precision == "bf16" else "f32",
        "data": "synthetic",
        "config": {**workload_config(wl, net.N, world, args.precision),
                   "precision": ("bf16 GEMM operands, fp32 accumulation and dual state" if args.precision == "bf16"
                                 else "fp32") + " iterations, fp64 final",
                   "l2": "flushed between steps (512 MB write)"},
        "clocks": clocks,
        "e2e": {"value": total_bounds / te_all, "unit": "bounds/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": head["gpu_launches"],
        "roofline": head["roofline"],
        "phases_ms_per_step": head["phases_ms_per_step"],
        "engine": head["engine"],
        "configs": configs,
        "peaks_source": bn.peak_src,
        "kernel_digest": kernel_digest(),
    }
    if not args.no_cpu_baseline:
        cpu, gaps = cpu_leg(wl, 15.0, bn.gap_runner(d, [args.precision]))
        line["cpu_baseline"] = cpu
        line["gap_vs_fp64_oracle"] = gaps
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# ----------------------------------------------------------------------------- the reference arm

def run_reference(args):
    """The reference arm: the FP64 CPU oracle, as it stands, on the host cores,
    each step a bounded sample of the headline workload."""
    world, rank, local = dist_env()
    if rank != 0:
        return 0
    wl = make_workload(args.workload, 0, args.subdomains, args.iters)
    on, lbk, ubk, masks = oracle_problem(wl)
    t0 = time.perf_counter()
    oracle_run(on, wl, lbk, ubk, masks[:2])
    per = (time.perf_counter() - t0) / 2
    budget_total = 120.0
    S = int(min(wl["B"], max(2, budget_total / max(per, 1e-6) / max(args.steps + args.warmup, 1))))
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle_run(on, wl, lbk, ubk, masks[:S])
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = S * len(times) / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "bounds/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / max(len(times), 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {**workload_config(wl, lbk.shape[1], args.gpus, args.precision),
                       "precision": "fp64 oracle (iterations and final bound)",
                       "oracle_sample": f"first {S} of {wl['B']} subdomains per step (the bound only: no IBP or "
                                        "backward in the timed region)"},
            "cpu_baseline": {"value": value, "unit": "bounds/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"first {S} of {wl['B']} subdomains per step, T={wl['T']}, FP64 NumPy/SciPy"},
            "e2e": {"value": value, "unit": "bounds/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
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
                res[prec] = (B / (statistics.median(times) / 1000.0), out.cpu().numpy(), net.tuned(B, prec))
            a32, a16 = res["fp32"][1], res["bf16"][1]
            fin = np.isfinite(a32) & np.isfinite(a16)
            rel = np.abs(a16[fin] - a32[fin]) / np.maximum(np.abs(a32[fin]), 1.0)
            print(json.dumps({"sweep": "deep", "subdomains": B, "iterations": T, "properties": n_props,
                              "fp32_bounds_per_s": res["fp32"][0], "bf16_bounds_per_s": res["bf16"][0],
                              "bf16_speedup": res["bf16"][0] / res["fp32"][0],
                              "fp32_engine": list(res["fp32"][2]), "bf16_engine": list(res["bf16"][2]),
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
