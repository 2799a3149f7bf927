"""Thin ctypes binding of libld's C ABI (include/ld.h).

Argument marshalling only: every step of the bound runs in libld's CUDA
kernels.  Tensors are torch CUDA tensors (device memory and streams come
from PyTorch); calls are ordered on torch's current CUDA stream.  If the
library is missing or no GPU is present, the calls raise: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libld.so")

LD_OK, LD_ERR_ARG, LD_ERR_SHAPE, LD_ERR_CUDA, LD_ERR_NOMEM, LD_ERR_TIMEOUT, LD_ERR_NONFINITE, LD_ERR_UNSUPPORTED = range(8)
LD_LAYER_FC, LD_LAYER_CONV = 0, 1
LD_INIT_ZERO, LD_INIT_CROWN, LD_INIT_GIVEN = 0, 1, 2
LD_PREC_FP32, LD_PREC_BF16 = 0, 1
LD_ENGINE_AUTO, LD_ENGINE_LAYERWISE, LD_ENGINE_FUSED = 0, 1, 2
LD_IB_CROWN, LD_IB_WK = 1, 2
LD_BRANCH_SR, LD_BRANCH_MSR, LD_BRANCH_FSB = 0, 1, 2
BRANCH_RULES = {"sr": LD_BRANCH_SR, "msr": LD_BRANCH_MSR, "fsb": LD_BRANCH_FSB}
IB_RULES = {"crown": LD_IB_CROWN, "wk": LD_IB_WK, "best": LD_IB_CROWN | LD_IB_WK}

EXPORTED = [
    "ld_opts_default", "ld_status_str", "ld_net_create", "ld_net_destroy", "ld_net_sizes", "ld_net_reserve",
    "ld_net_sync_status", "ld_selftest_wait_timeout", "ld_intermediate_bounds", "ld_intermediate_bounds_split",
    "ld_bound", "ld_dual_supergradient", "ld_bound_backward",
    "ld_net_profile", "ld_net_profile_read", "ld_launch_count", "ld_net_tuned", "ld_final_bound_noalloc",
    "ld_test_inject_alloc_failure", "ld_intermediate_bounds_propagated", "ld_prox_opts_default", "ld_bound_proximal",
    "ld_branching_scores", "ld_branch", "ld_upper_bound", "ld_bound_dsg", "ld_test_fused_tc_plan",
    "ld_intermediate_bounds_ball", "ld_bound_ball", "ld_bound_trace",
]
PHASES = {"iter": 0, "final": 1, "init": 2, "ibp": 3, "backward": 4}


class LDError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {status_str(code)} (status {code})")


class LayerDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("cin", C.c_int32), ("h", C.c_int32), ("w", C.c_int32),
                ("cout", C.c_int32), ("kh", C.c_int32), ("kw", C.c_int32), ("stride", C.c_int32),
                ("pad", C.c_int32), ("W", C.c_void_p), ("b", C.c_void_p)]


class Opts(C.Structure):
    _fields_ = [("alpha0", C.c_float), ("alpha_end", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float),
                ("eps", C.c_float), ("init", C.c_int32), ("precision", C.c_int32), ("fp64_final", C.c_int32),
                ("t_offset", C.c_int32), ("t_total", C.c_int32), ("engine", C.c_int32), ("tile", C.c_int32),
                ("cta_threads", C.c_int32)]


class ProxOpts(C.Structure):
    _fields_ = [("eta0", C.c_float), ("eta_end", C.c_float), ("mu", C.c_float), ("J", C.c_int32),
                ("init", C.c_int32), ("fp64_final", C.c_int32)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libld.so (built in-tree by paper_2104_06718_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libld.so not found at {path}: run `python -m paper_2104_06718_gb300.build` "
                           "(nvcc, sm_103a) first; there is no CPU fallback")
    lib = C.CDLL(path)
    vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
    lib.ld_opts_default.argtypes = [C.POINTER(Opts)]
    lib.ld_opts_default.restype = None
    lib.ld_status_str.argtypes = [C.c_int]
    lib.ld_status_str.restype = C.c_char_p
    lib.ld_net_create.argtypes = [C.POINTER(LayerDesc), i32, vp, C.POINTER(vp), vp]
    lib.ld_net_destroy.argtypes = [vp]
    lib.ld_net_sizes.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i32), C.POINTER(i64), C.POINTER(i64)]
    lib.ld_net_reserve.argtypes = [vp, i32]
    lib.ld_net_sync_status.argtypes = [vp, vp]
    lib.ld_intermediate_bounds.argtypes = [vp, vp, vp, i32, vp, vp, vp, vp]
    lib.ld_intermediate_bounds_split.argtypes = [vp, vp, vp, i32, vp, vp, i32, vp, vp, vp]
    lib.ld_bound.argtypes = [vp, vp, vp, vp, vp, i32, vp, vp, i32, i32, C.POINTER(Opts), vp, vp, vp, vp, vp]
    lib.ld_bound_trace.argtypes = [vp, vp, vp, vp, vp, i32, vp, vp, i32, i32, C.POINTER(Opts), vp, vp, vp, vp, vp,
                                   vp]
    lib.ld_bound_ball.argtypes = [vp, vp, vp, vp, vp, i32, vp, vp, i32, i32, C.POINTER(Opts), vp, vp, vp, vp, vp]
    lib.ld_intermediate_bounds_ball.argtypes = [vp, vp, vp, i32, vp, vp, vp, vp]
    lib.ld_dual_supergradient.argtypes = [vp, vp, vp, vp, vp, i32, vp, vp, i32, vp, vp, vp, vp, vp]
    lib.ld_bound_backward.argtypes = [vp, vp, vp, vp, vp, i32, vp, vp, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.ld_selftest_wait_timeout.argtypes = [vp, vp]
    lib.ld_net_profile.argtypes = [vp, i32]
    lib.ld_net_profile_read.argtypes = [vp, i32, C.POINTER(C.c_double), C.POINTER(i64), i32]
    lib.ld_launch_count.argtypes = [C.POINTER(i64)]
    lib.ld_net_tuned.argtypes = [vp, i32, i32, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]
    lib.ld_final_bound_noalloc.argtypes = [vp, vp, vp, vp, vp, i32, vp, vp, i32, vp, vp, vp]
    lib.ld_test_inject_alloc_failure.argtypes = [i32, i32]
    lib.ld_intermediate_bounds_propagated.argtypes = [vp, vp, vp, i32, vp, vp, i32, i32, vp, vp, vp]
    lib.ld_prox_opts_default.argtypes = [C.POINTER(ProxOpts)]
    lib.ld_prox_opts_default.restype = None
    lib.ld_bound_proximal.argtypes = [vp, vp, vp, vp, vp, i32, vp, vp, i32, i32, C.POINTER(ProxOpts), vp, vp, vp, vp]
    lib.ld_branching_scores.argtypes = [vp, vp, vp, i32, vp, vp, i32, vp, vp, vp, vp]
    lib.ld_branch.argtypes = [vp, vp, vp, vp, vp, i32, vp, vp, i32, i32, C.c_float, vp, vp, vp]
    lib.ld_upper_bound.argtypes = [vp, vp, vp, vp, vp, i32, vp, vp, i32, vp, vp, vp, vp]
    lib.ld_bound_dsg.argtypes = [vp, vp, vp, vp, vp, i32, vp, vp, i32, i32, C.POINTER(Opts), vp, vp, vp, vp, vp, vp, vp]
    for name in EXPORTED:
        if name not in ("ld_opts_default", "ld_status_str", "ld_prox_opts_default"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def status_str(code: int) -> str:
    try:
        return load_library().ld_status_str(int(code)).decode()
    except RuntimeError:
        return "unknown"


def _check(code, where):
    if code != LD_OK:
        raise LDError(code, where)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("libld takes CUDA tensors")
    if not t.is_contiguous():
        raise ValueError("libld takes contiguous tensors")
    return C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(x, dtype):
    if isinstance(x, torch.Tensor):
        t = x.to(device="cuda", dtype=dtype)
    else:
        t = torch.as_tensor(np.asarray(x), dtype=dtype, device="cuda")
    return t.contiguous()


@dataclass
class Options:
    """Solver options (ld_opts): step size alpha0 -> alpha_end decayed
    linearly (Sec. 7.2), Adam moments, initialisation (Prop. 3 CROWN by
    default), FP64 final bound."""
    alpha0: float = 1e-2
    alpha_end: float = 1e-4
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    init: str = "crown"          # "zero" | "crown" | "given"
    precision: str = "fp32"      # "fp32" | "bf16"
    fp64_final: bool = True
    t_offset: int = 0
    t_total: int = 0
    engine: str = "auto"         # "auto" | "layerwise" | "fused"
    tile: int = 0                # fused engine: subdomains per CTA (0 = auto, 1, 2, 4)
    cta_threads: int = 0         # fused engine: threads per CTA (0 = auto, 256, 512 with tile 1 or 2)

    def to_c(self) -> Opts:
        return Opts(self.alpha0, self.alpha_end, self.beta1, self.beta2, self.eps,
                    {"zero": LD_INIT_ZERO, "crown": LD_INIT_CROWN, "given": LD_INIT_GIVEN}[self.init],
                    {"fp32": LD_PREC_FP32, "bf16": LD_PREC_BF16}[self.precision],
                    int(self.fp64_final), self.t_offset, self.t_total,
                    {"auto": LD_ENGINE_AUTO, "layerwise": LD_ENGINE_LAYERWISE, "fused": LD_ENGINE_FUSED}[self.engine],
                    int(self.tile), int(self.cta_threads))


@dataclass
class ProxOptions:
    """Proximal-solver options (ld_prox_opts): eta increased linearly from
    eta0 to eta_end, momentum mu, J Frank-Wolfe sweeps (Sec. 7.2 defaults;
    the branch-and-bound setting of Sec. 8.2 is eta0 = eta_end = 100, mu = 0)."""
    eta0: float = 1e1
    eta_end: float = 5e2
    mu: float = 0.3
    J: int = 2
    init: str = "crown"
    fp64_final: bool = True

    def to_c(self) -> ProxOpts:
        return ProxOpts(self.eta0, self.eta_end, self.mu, int(self.J),
                        {"zero": LD_INIT_ZERO, "crown": LD_INIT_CROWN, "given": LD_INIT_GIVEN}[self.init],
                        int(self.fp64_final))


def layer_descs(specs):
    """ld_layer_desc array of layer specs, and the arrays it points into."""
    keep = []
    descs = (LayerDesc * len(specs))()
    for d, s in zip(descs, specs):
        W = np.ascontiguousarray(np.asarray(s.W, dtype=np.float32))
        b = np.ascontiguousarray(np.asarray(s.b, dtype=np.float32))
        keep += [W, b]
        if s.kind == "fc":
            d.kind, d.cin, d.h, d.w = LD_LAYER_FC, W.shape[1], 1, 1
            d.cout, d.kh, d.kw, d.stride, d.pad = W.shape[0], 1, 1, 1, 0
        else:
            c, h, w = s.in_shape
            d.kind, d.cin, d.h, d.w = LD_LAYER_CONV, c, h, w
            d.cout, d.kh, d.kw, d.stride, d.pad = W.shape[0], W.shape[2], W.shape[3], s.stride, s.pad
        d.W = W.ctypes.data
        d.b = b.ctypes.data
    return descs, keep


class Net:
    """An ld_net handle: device copies of a ReLU net in canonical form.

    specs: sequence of layer specs with attributes kind ('fc'|'conv'), W, b,
    in_shape, stride, pad (see paper_2104_06718_gb300.synth.LayerSpec).
    margin: None, or the property vector c folded into the last layer.
    """

    def __init__(self, specs, margin=None):
        lib = load_library()
        descs, self._keep = layer_descs(specs)
        mptr = None
        if margin is not None:
            m = np.ascontiguousarray(np.asarray(margin, dtype=np.float32))
            self._keep.append(m)
            mptr = C.c_void_p(m.ctypes.data)
        h = C.c_void_p()
        torch.cuda.init()
        _check(lib.ld_net_create(descs, len(specs), mptr, C.byref(h), _stream()), "ld_net_create")
        self._h = h
        self._lib = lib
        n0, N, nl, nw, nb = C.c_int64(), C.c_int64(), C.c_int32(), C.c_int64(), C.c_int64()
        _check(lib.ld_net_sizes(h, C.byref(n0), C.byref(N), C.byref(nl), C.byref(nw), C.byref(nb)), "ld_net_sizes")
        self.n0, self.N, self.n_layers, self.n_weights, self.n_biases = n0.value, N.value, nl.value, nw.value, nb.value
        self.specs = list(specs)
        self.margin = None if margin is None else np.asarray(margin, np.float32)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.ld_net_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def reserve(self, B: int):
        _check(self._lib.ld_net_reserve(self._h, int(B)), "ld_net_reserve")

    def sync_status(self):
        return self._lib.ld_net_sync_status(self._h, _stream())

    def selftest_wait_timeout(self):
        """Launch the bounded-wait self-test (a wait nothing completes); the
        status word then reads LD_ERR_TIMEOUT."""
        _check(self._lib.ld_selftest_wait_timeout(self._h, _stream()), "ld_selftest_wait_timeout")

    def profile(self, enable: bool = True):
        """Record CUDA events around each phase of every call."""
        _check(self._lib.ld_net_profile(self._h, int(enable)), "ld_net_profile")

    def profile_read(self, phase: str, reset: bool = False):
        """(total ms, instances) of a phase since the last reset."""
        ms, n = C.c_double(), C.c_int64()
        _check(self._lib.ld_net_profile_read(self._h, PHASES[phase], C.byref(ms), C.byref(n), int(reset)),
               "ld_net_profile_read")
        return ms.value, n.value

    def tuned(self, B: int, precision: str = "fp32"):
        """(engine, tile, threads per CTA) chosen by the autotuner for batch
        size B and the iterations' precision, or (None, 0, 0).  For "bf16",
        "layerwise" is the layer-wise tensor-core engine and "fused" the
        fused tensor-core engine."""
        e, t, n = C.c_int32(), C.c_int32(), C.c_int32()
        prec = {"fp32": LD_PREC_FP32, "bf16": LD_PREC_BF16}[precision]
        _check(self._lib.ld_net_tuned(self._h, prec, int(B), C.byref(e), C.byref(t), C.byref(n)), "ld_net_tuned")
        names = {LD_ENGINE_LAYERWISE: "layerwise", LD_ENGINE_FUSED: "fused"}
        return names.get(e.value), t.value, n.value


def inject_alloc_failure(after: int, code: int = LD_ERR_NOMEM):
    """Arm a host-side failure of libld's device allocations: after `after`
    more allocations succeed, the next one fails with `code` (LD_ERR_NOMEM or
    LD_ERR_CUDA) without calling the CUDA allocator; after < 0 disarms."""
    _check(load_library().ld_test_inject_alloc_failure(int(after), int(code)), "ld_test_inject_alloc_failure")


def fused_tc_plan(specs, S: int, smem_limit: int = 232448):
    """Host-only layout check of the fused tensor-core engine for S
    subdomains per CTA (no GPU needed): None when the net has no plan within
    smem_limit bytes, else the plan's figures."""
    descs, keep = layer_descs(specs)
    info = (C.c_int64 * 7)()
    st = load_library().ld_test_fused_tc_plan(descs, len(specs), int(S), C.c_int64(smem_limit), info)
    if st == LD_ERR_UNSUPPORTED:
        return None
    _check(st, "ld_test_fused_tc_plan")
    keys = ("smem_bytes", "tmem_cols", "mmas_per_iteration", "shadow_bytes", "weight_tile_bytes", "passes",
            "half_tile_mmas")
    return dict(zip(keys, (int(v) for v in info)))


def launch_count() -> int:
    """Kernels launched by libld in this process so far."""
    n = C.c_int64()
    _check(load_library().ld_launch_count(C.byref(n)), "ld_launch_count")
    return n.value


def ld_intermediate_bounds(net: Net, lb0, ub0, want_output_lb: bool = False):
    """IBP bounds of layers 1..n-1 ([P, N] each, outward rounded) and,
    optionally, the IBP lower bound of the output ([P] float64)."""
    lb0 = _dev(lb0, torch.float32)
    ub0 = _dev(ub0, torch.float32)
    if lb0.dim() == 1:
        lb0, ub0 = lb0[None], ub0[None]
    P = lb0.shape[0]
    lbk = torch.empty((P, net.N), dtype=torch.float32, device="cuda")
    ubk = torch.empty_like(lbk)
    out_lb = torch.empty(P, dtype=torch.float64, device="cuda") if want_output_lb else None
    _check(net._lib.ld_intermediate_bounds(net.handle, _ptr(lb0), _ptr(ub0), P, _ptr(lbk), _ptr(ubk), _ptr(out_lb),
                                           _stream()), "ld_intermediate_bounds")
    return (lbk, ubk, out_lb) if want_output_lb else (lbk, ubk)


def ld_intermediate_bounds_ball(net: Net, center, eps, want_output_lb: bool = False):
    """Interval bounds of layers 1..n-1 over l2 balls ||x0 - center[p]|| <=
    eps[p] (Sec. 3.2.1): layer 1 exact up to outward rounding, the rest by
    interval propagation; optionally the output's lower bound ([P] float64)."""
    center = _dev(center, torch.float32)
    if center.dim() == 1:
        center = center[None]
    P = center.shape[0]
    eps = _dev(eps, torch.float32).reshape(-1)
    if eps.numel() != P:
        raise ValueError("eps needs one radius per centre")
    lbk = torch.empty((P, net.N), dtype=torch.float32, device="cuda")
    ubk = torch.empty_like(lbk)
    out_lb = torch.empty(P, dtype=torch.float64, device="cuda") if want_output_lb else None
    _check(net._lib.ld_intermediate_bounds_ball(net.handle, _ptr(center), _ptr(eps), P, _ptr(lbk), _ptr(ubk),
                                                _ptr(out_lb), _stream()), "ld_intermediate_bounds_ball")
    return (lbk, ubk, out_lb) if want_output_lb else (lbk, ubk)


def ld_intermediate_bounds_split(net: Net, lb0, ub0, masks, prop=None):
    """Interval bounds recomputed per subdomain after its splits: ([B, N],
    [B, N]) float32, outward rounded and already clamped by the masks.
    To bound with them, pass n_props = B: ld_bound(net, lb0[prop], ub0[prop],
    lbk, ubk, prop=arange(B), masks=masks, ...)."""
    lb0 = _dev(lb0, torch.float32)
    ub0 = _dev(ub0, torch.float32)
    if lb0.dim() == 1:
        lb0, ub0 = lb0[None], ub0[None]
    masks = _dev(masks, torch.int8)
    B = masks.shape[0]
    prop = None if prop is None else _dev(prop, torch.int32)
    lbk = torch.empty((B, net.N), dtype=torch.float32, device="cuda")
    ubk = torch.empty_like(lbk)
    _check(net._lib.ld_intermediate_bounds_split(net.handle, _ptr(lb0), _ptr(ub0), lb0.shape[0], _ptr(prop),
                                                 _ptr(masks), B, _ptr(lbk), _ptr(ubk), _stream()),
           "ld_intermediate_bounds_split")
    return lbk, ubk


def ld_intermediate_bounds_propagated(net: Net, lb0, ub0, rules: str = "best", masks=None, prop=None,
                                      n_rows: int | None = None):
    """CROWN / WK / layer-wise best ("best") intermediate bounds ([R, N],
    [R, N]) float32, outward rounded.  Without masks and prop: one row per
    box (root bounds).  With masks [B, N] (and prop [B] when there are several
    boxes): bounds recomputed per subdomain after its splits, already clamped."""
    lb0 = _dev(lb0, torch.float32)
    ub0 = _dev(ub0, torch.float32)
    if lb0.dim() == 1:
        lb0, ub0 = lb0[None], ub0[None]
    masks = None if masks is None else _dev(masks, torch.int8)
    prop = None if prop is None else _dev(prop, torch.int32)
    if n_rows is None:
        n_rows = masks.shape[0] if masks is not None else (prop.shape[0] if prop is not None else lb0.shape[0])
    lbk = torch.empty((n_rows, net.N), dtype=torch.float32, device="cuda")
    ubk = torch.empty_like(lbk)
    _check(net._lib.ld_intermediate_bounds_propagated(net.handle, _ptr(lb0), _ptr(ub0), lb0.shape[0], _ptr(prop),
                                                      _ptr(masks), int(n_rows), IB_RULES[rules], _ptr(lbk), _ptr(ubk),
                                                      _stream()), "ld_intermediate_bounds_propagated")
    return lbk, ubk


def _problem(lb0, ub0, lbk, ubk, prop, masks, B):
    lb0 = _dev(lb0, torch.float32)
    ub0 = _dev(ub0, torch.float32)
    if lb0.dim() == 1:
        lb0, ub0 = lb0[None], ub0[None]
    lbk = _dev(lbk, torch.float32)
    ubk = _dev(ubk, torch.float32)
    if lbk.dim() == 1:
        lbk, ubk = lbk[None], ubk[None]
    prop = None if prop is None else _dev(prop, torch.int32)
    masks = None if masks is None else _dev(masks, torch.int8)
    if B is None:
        B = masks.shape[0] if masks is not None else (prop.shape[0] if prop is not None else 1)
    return lb0, ub0, lbk, ubk, prop, masks, int(B)


def ld_bound(net: Net, lb0, ub0, lbk, ubk, prop=None, masks=None, n_iters: int = 100, opts: Options | None = None,
             rho_in=None, B: int | None = None, return_rho: bool = False, adam_mv=None):
    """Lower bounds [B] (float64) after n_iters Adam iterations (Algorithm 1).
    With return_rho, also returns rho_T [B, N] (float32)."""
    lb0, ub0, lbk, ubk, prop, masks, B = _problem(lb0, ub0, lbk, ubk, prop, masks, B)
    o = (opts or Options())
    if rho_in is not None and o.init != "given":
        o = Options(**{**o.__dict__, "init": "given"})
    rho_in = None if rho_in is None else _dev(rho_in, torch.float32)
    out = torch.empty(B, dtype=torch.float64, device="cuda")
    rho_out = torch.empty((B, net.N), dtype=torch.float32, device="cuda") if return_rho else None
    oc = o.to_c()
    _check(net._lib.ld_bound(net.handle, _ptr(lb0), _ptr(ub0), _ptr(lbk), _ptr(ubk), lbk.shape[0], _ptr(prop),
                             _ptr(masks), B, int(n_iters), C.byref(oc), _ptr(rho_in), _ptr(rho_out), _ptr(adam_mv),
                             _ptr(out), _stream()), "ld_bound")
    return (out, rho_out) if return_rho else out


def ld_bound_trace(net: Net, lb0, ub0, lbk, ubk, prop=None, masks=None, n_iters: int = 100,
                   opts: Options | None = None, rho_in=None, B: int | None = None, adam_mv=None):
    """(bounds [B] float64, q trace [n_iters, B] float64): ld_bound on the
    FP32 layer-wise engine with q(rho_t) recorded before every update."""
    lb0, ub0, lbk, ubk, prop, masks, B = _problem(lb0, ub0, lbk, ubk, prop, masks, B)
    o = (opts or Options())
    if rho_in is not None and o.init != "given":
        o = Options(**{**o.__dict__, "init": "given"})
    rho_in = None if rho_in is None else _dev(rho_in, torch.float32)
    out = torch.empty(B, dtype=torch.float64, device="cuda")
    trace = torch.empty((int(n_iters), B), dtype=torch.float64, device="cuda")
    oc = o.to_c()
    _check(net._lib.ld_bound_trace(net.handle, _ptr(lb0), _ptr(ub0), _ptr(lbk), _ptr(ubk), lbk.shape[0], _ptr(prop),
                                   _ptr(masks), B, int(n_iters), C.byref(oc), _ptr(rho_in), None, _ptr(adam_mv),
                                   _ptr(out), _ptr(trace) if trace.numel() else None, _stream()), "ld_bound_trace")
    return out, trace


def ld_bound_ball(net: Net, center, eps, lbk, ubk, prop=None, masks=None, n_iters: int = 100,
                  opts: Options | None = None, rho_in=None, B: int | None = None, return_rho: bool = False,
                  adam_mv=None):
    """Lower bounds [B] (float64) over l2-ball input domains (Sec. 3.2.1)
    after n_iters Adam iterations; arguments as ld_bound with the boxes
    replaced by centres [P, n0] and radii [P]."""
    center, _, lbk, ubk, prop, masks, B = _problem(center, center, lbk, ubk, prop, masks, B)
    eps = _dev(eps, torch.float32).reshape(-1)
    if eps.numel() != center.shape[0]:
        raise ValueError("eps needs one radius per centre")
    o = (opts or Options())
    if rho_in is not None and o.init != "given":
        o = Options(**{**o.__dict__, "init": "given"})
    rho_in = None if rho_in is None else _dev(rho_in, torch.float32)
    out = torch.empty(B, dtype=torch.float64, device="cuda")
    rho_out = torch.empty((B, net.N), dtype=torch.float32, device="cuda") if return_rho else None
    oc = o.to_c()
    _check(net._lib.ld_bound_ball(net.handle, _ptr(center), _ptr(eps), _ptr(lbk), _ptr(ubk), lbk.shape[0],
                                  _ptr(prop), _ptr(masks), B, int(n_iters), C.byref(oc), _ptr(rho_in),
                                  _ptr(rho_out), _ptr(adam_mv), _ptr(out), _stream()), "ld_bound_ball")
    return (out, rho_out) if return_rho else out


def ld_bound_proximal(net: Net, lb0, ub0, lbk, ubk, prop=None, masks=None, n_iters: int = 100,
                      opts: ProxOptions | None = None, rho_in=None, B: int | None = None, return_rho: bool = False):
    """Lower bounds [B] (float64) after n_iters iterations of the proximal
    solver (Algorithm 2).  With return_rho, also the final duals [B, N]."""
    lb0, ub0, lbk, ubk, prop, masks, B = _problem(lb0, ub0, lbk, ubk, prop, masks, B)
    o = opts or ProxOptions()
    if rho_in is not None and o.init != "given":
        o = ProxOptions(**{**o.__dict__, "init": "given"})
    rho_in = None if rho_in is None else _dev(rho_in, torch.float32)
    out = torch.empty(B, dtype=torch.float64, device="cuda")
    rho_out = torch.empty((B, net.N), dtype=torch.float32, device="cuda") if return_rho else None
    oc = o.to_c()
    _check(net._lib.ld_bound_proximal(net.handle, _ptr(lb0), _ptr(ub0), _ptr(lbk), _ptr(ubk), lbk.shape[0],
                                      _ptr(prop), _ptr(masks), B, int(n_iters), C.byref(oc), _ptr(rho_in),
                                      _ptr(rho_out), _ptr(out), _stream()), "ld_bound_proximal")
    return (out, rho_out) if return_rho else out


def ld_bound_dsg(net: Net, lb0, ub0, lbk, ubk, prop=None, masks=None, n_iters: int = 100,
                 opts: Options | None = None, mu_in=None, lam_in=None, B: int | None = None,
                 return_duals: bool = False):
    """DSG+ (Sec. 2.2.2): (Dec-DSG+ bound q(mu_T) [B] float64, sound; DSG+'s own
    d_O(mu_T, lambda_T) [B] float64); with return_duals also (mu_T, lambda_T)."""
    lb0, ub0, lbk, ubk, prop, masks, B = _problem(lb0, ub0, lbk, ubk, prop, masks, B)
    o = opts or Options()
    if mu_in is not None and o.init != "given":
        o = Options(**{**o.__dict__, "init": "given"})
    mu_in = None if mu_in is None else _dev(mu_in, torch.float32)
    lam_in = None if lam_in is None else _dev(lam_in, torch.float32)
    dec = torch.empty(B, dtype=torch.float64, device="cuda")
    dsg = torch.empty(B, dtype=torch.float64, device="cuda")
    f = (lambda: torch.empty((B, net.N), dtype=torch.float32, device="cuda")) if return_duals else (lambda: None)
    mu_out, lam_out = f(), f()
    oc = o.to_c()
    _check(net._lib.ld_bound_dsg(net.handle, _ptr(lb0), _ptr(ub0), _ptr(lbk), _ptr(ubk), lbk.shape[0], _ptr(prop),
                                 _ptr(masks), B, int(n_iters), C.byref(oc), _ptr(mu_in), _ptr(lam_in), _ptr(mu_out),
                                 _ptr(lam_out), _ptr(dec), _ptr(dsg), _stream()), "ld_bound_dsg")
    return (dec, dsg, mu_out, lam_out) if return_duals else (dec, dsg)


def ld_branching_scores(net: Net, lbk, ubk, prop=None, masks=None, B: int | None = None):
    """(s_SR, s_FSB, t_SR) [B, N] float32 branching scores (Sec. 4)."""
    lbk = _dev(lbk, torch.float32)
    ubk = _dev(ubk, torch.float32)
    if lbk.dim() == 1:
        lbk, ubk = lbk[None], ubk[None]
    prop = None if prop is None else _dev(prop, torch.int32)
    masks = None if masks is None else _dev(masks, torch.int8)
    if B is None:
        B = masks.shape[0] if masks is not None else (prop.shape[0] if prop is not None else 1)
    f = lambda: torch.empty((B, net.N), dtype=torch.float32, device="cuda")
    s_sr, s_fsb, t_sr = f(), f(), f()
    _check(net._lib.ld_branching_scores(net.handle, _ptr(lbk), _ptr(ubk), lbk.shape[0], _ptr(prop), _ptr(masks), int(B),
                                        _ptr(s_sr), _ptr(s_fsb), _ptr(t_sr), _stream()), "ld_branching_scores")
    return s_sr, s_fsb, t_sr


def ld_branch(net: Net, lb0, ub0, lbk, ubk, prop=None, masks=None, rule: str = "fsb", threshold: float = 0.0,
              B: int | None = None, return_child_bounds: bool = False):
    """Branching decision per subdomain [B] int32 (flat ReLU index, -1 when
    none is ambiguous); with return_child_bounds (FSB), also the candidates'
    children bounds [B, 2(n-1), 2] float64."""
    lb0, ub0, lbk, ubk, prop, masks, B = _problem(lb0, ub0, lbk, ubk, prop, masks, B)
    dec = torch.empty(B, dtype=torch.int32, device="cuda")
    child = torch.empty((B, 2 * (net.n_layers - 1), 2), dtype=torch.float64, device="cuda") \
        if return_child_bounds else None
    _check(net._lib.ld_branch(net.handle, _ptr(lb0), _ptr(ub0), _ptr(lbk), _ptr(ubk), lbk.shape[0], _ptr(prop),
                              _ptr(masks), B, BRANCH_RULES[rule], float(threshold), _ptr(dec), _ptr(child),
                              _stream()), "ld_branch")
    return (dec, child) if return_child_bounds else dec


def ld_upper_bound(net: Net, lb0, ub0, lbk, ubk, rho, prop=None, masks=None, return_x0: bool = False):
    """Network output [B] (float64) at the inner minimiser's input point x0* of
    q(rho), an upper bound on the minimum (Sec. 5.1.3); optionally x0* [B, n0]."""
    rho = _dev(rho, torch.float32)
    lb0, ub0, lbk, ubk, prop, masks, B = _problem(lb0, ub0, lbk, ubk, prop, masks, rho.shape[0])
    ub = torch.empty(B, dtype=torch.float64, device="cuda")
    x0 = torch.empty((B, net.n0), dtype=torch.float32, device="cuda") if return_x0 else None
    _check(net._lib.ld_upper_bound(net.handle, _ptr(lb0), _ptr(ub0), _ptr(lbk), _ptr(ubk), lbk.shape[0], _ptr(prop),
                                   _ptr(masks), B, _ptr(rho), _ptr(ub), _ptr(x0), _stream()), "ld_upper_bound")
    return (ub, x0) if return_x0 else ub


def ld_dual_supergradient(net: Net, lb0, ub0, lbk, ubk, rho, prop=None, masks=None):
    """q(rho) [B] float64, supergradient [B, N] float32 and vertex codes [B, N]
    int8 at a given rho, in FP32 (no update)."""
    rho = _dev(rho, torch.float32)
    lb0, ub0, lbk, ubk, prop, masks, B = _problem(lb0, ub0, lbk, ubk, prop, masks, rho.shape[0])
    q = torch.empty(B, dtype=torch.float64, device="cuda")
    sg = torch.empty((B, net.N), dtype=torch.float32, device="cuda")
    vtx = torch.empty((B, net.N), dtype=torch.int8, device="cuda")
    _check(net._lib.ld_dual_supergradient(net.handle, _ptr(lb0), _ptr(ub0), _ptr(lbk), _ptr(ubk), lbk.shape[0],
                                          _ptr(prop), _ptr(masks), B, _ptr(rho), _ptr(q), _ptr(sg), _ptr(vtx),
                                          _stream()), "ld_dual_supergradient")
    return q, sg, vtx


def ld_bound_backward(net: Net, lb0, ub0, lbk, ubk, rho, grad_out=None, prop=None, masks=None):
    """Danskin gradients at fixed rho: dict with gW (packed), gb, glb0, gub0,
    glbk, gubk (float32 device tensors)."""
    rho = _dev(rho, torch.float32)
    lb0, ub0, lbk, ubk, prop, masks, B = _problem(lb0, ub0, lbk, ubk, prop, masks, rho.shape[0])
    P = lbk.shape[0]
    go = None if grad_out is None else _dev(grad_out, torch.float64)
    f = lambda *shape: torch.empty(shape, dtype=torch.float32, device="cuda")
    out = {"gW": f(net.n_weights), "gb": f(net.n_biases), "glb0": f(P, net.n0), "gub0": f(P, net.n0),
           "glbk": f(P, net.N), "gubk": f(P, net.N)}
    _check(net._lib.ld_bound_backward(net.handle, _ptr(lb0), _ptr(ub0), _ptr(lbk), _ptr(ubk), P, _ptr(prop),
                                      _ptr(masks), B, _ptr(rho), _ptr(go), _ptr(out["gW"]), _ptr(out["gb"]),
                                      _ptr(out["glb0"]), _ptr(out["gub0"]), _ptr(out["glbk"]), _ptr(out["gubk"]),
                                      _stream()), "ld_bound_backward")
    return out


def ld_final_bound_noalloc(net: Net, lb0, ub0, lbk, ubk, rho, prop=None, masks=None, out=None):
    """Sound FP64 bound q(rho) [B] at a given rho without any device allocation
    inside the library (its scratch is a fixed array compiled into libld).
    For callers that cannot allocate device memory when they need a bound.
    Pass `out` (a float64 CUDA tensor [B]) to keep this call allocation-free
    on the Python side too."""
    rho = _dev(rho, torch.float32)
    lb0, ub0, lbk, ubk, prop, masks, B = _problem(lb0, ub0, lbk, ubk, prop, masks, rho.shape[0])
    if out is None:
        out = torch.empty(B, dtype=torch.float64, device="cuda")
    _check(net._lib.ld_final_bound_noalloc(net.handle, _ptr(lb0), _ptr(ub0), _ptr(lbk), _ptr(ubk), lbk.shape[0],
                                           _ptr(prop), _ptr(masks), B, _ptr(rho), _ptr(out), _stream()),
           "ld_final_bound_noalloc")
    return out
