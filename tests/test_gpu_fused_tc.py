"""GPU: the fused tensor-core engine (precision "bf16", engine "fused").

All iterations of a call in one launch with the dual state resident in
shared memory, the conv passes as tcgen05 GEMMs over BF16 shadow planes
(FP32 accumulation in TMEM), the FC passes with BF16-rounded operands: the
same operand rounding as the layer-wise tensor-core engine, so the same
oracle (oracle.BF16Passes: BF16 weights and operands, exact sums).

Checks, for 1 and 2 subdomains per CTA where the net has a plan:
  * short runs against the BF16 oracle                              1e-5
  * long runs against the BF16 oracle and the FP32 iterations      FP32 chaos floor / 1e-3 gap
  * the two BF16 engines against each other after 1 and 3 steps     1e-5
  * a ragged last CTA, an empty subdomain, bitwise resume, a given start
  * the full-size Base call (256 subdomains, T = 100): sampled rows
    against the BF16 and FP64 oracles, the gap to FP32 over the batch
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2104_06718_gb300 import binding as ldb
from helpers import conv_problem

pytestmark = pytest.mark.gpu

FULL_RUN_MAX = 1e-3
FULL_RUN_MEDIAN = 3e-4
GAP_MAX = 1e-3
SHAPES = [("base", 1), ("base", 2), ("wide", 1), ("deep", 1)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_06718_gb300 import build
    build.build()
    ldb.load_library()


def fused(S, **kw):
    return ldb.Options(precision="bf16", engine="fused", tile=S, **kw)


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b) / np.maximum(np.abs(b), 1.0)


def args_of(pb):
    return (pb["l0"], pb["u0"], pb["lbk"], pb["ubk"], pb["prop"], pb["masks"])


def run_gpu(pb, T, opts, net=None):
    net = net or ldb.Net(pb["specs"])
    return ldb.ld_bound(net, *args_of(pb), n_iters=T, opts=opts).cpu().numpy()


def run_oracle(pb, T, operands="bf16", rows=None):
    prop = pb["prop"] if rows is None else pb["prop"][rows]
    masks = pb["masks"] if rows is None else pb["masks"][rows]
    ref, _, _ = oracle.ld_bound(pb["net"], pb["l0"].astype(np.float64), pb["u0"].astype(np.float64),
                                pb["lbk"].astype(np.float64), pb["ubk"].astype(np.float64), prop, masks, T,
                                operands=operands)
    return ref


@pytest.mark.parametrize("name,S", SHAPES)
@pytest.mark.parametrize("T", [1, 3])
def test_short_runs_match_bf16_oracle(name, S, T):
    pb = conv_problem(name, 15, depth=(0, 8), block=8)   # 15: a ragged last CTA for S = 2
    net = ldb.Net(pb["specs"])
    out = run_gpu(pb, T, fused(S), net)
    ref = run_oracle(pb, T)
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(out), fin)
    assert np.max(rel(out[fin], ref[fin])) < 1e-5
    lay = run_gpu(pb, T, ldb.Options(precision="bf16", engine="layerwise"), net)
    assert np.max(rel(out[fin], lay[fin])) < 1e-5


@pytest.mark.parametrize("name,S,B,T", [("base", 2, 24, 100), ("base", 1, 12, 100), ("deep", 1, 12, 100),
                                        ("wide", 1, 8, 60)])
def test_long_runs_match_bf16_oracle_and_fp32(name, S, B, T):
    pb = conv_problem(name, B, depth=(0, 8), block=5)
    out = run_gpu(pb, T, fused(S))
    ref = run_oracle(pb, T)
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(out), fin)
    r = rel(out[fin], ref[fin])
    assert np.max(r) < FULL_RUN_MAX and np.median(r) < FULL_RUN_MEDIAN
    f32 = run_gpu(pb, T, ldb.Options(engine="layerwise"))
    assert np.max(rel(out[fin], f32[fin])) < GAP_MAX


@pytest.mark.parametrize("S", [1, 2])
def test_empty_subdomain_ragged_batch_and_resume(S):
    pb = conv_problem("base", 15, depth=(0, 8), block=1)
    masks = pb["masks"].copy()
    blk = np.nonzero(pb["ubk"][0] < 0)[0]
    masks[3, blk[0]] = 1          # forced passing on a blocking ReLU: empty
    pb = dict(pb, masks=masks)
    net = ldb.Net(pb["specs"])
    args = args_of(pb)
    out_a, rho_a = ldb.ld_bound(net, *args, n_iters=20, return_rho=True, opts=fused(S))
    assert np.isinf(out_a[3].item()) and np.isfinite(np.delete(out_a.cpu().numpy(), 3)).all()
    B, N = pb["B"], pb["lbk"].shape[1]
    mv = torch.zeros((2, B, N), dtype=torch.float32, device="cuda")
    _, rho_1 = ldb.ld_bound(net, *args, n_iters=12, opts=fused(S, t_offset=0, t_total=20), return_rho=True,
                            adam_mv=mv)
    out_b, rho_b = ldb.ld_bound(net, *args, n_iters=8, opts=fused(S, t_offset=12, t_total=20, init="given"),
                                rho_in=rho_1, return_rho=True, adam_mv=mv)
    assert torch.equal(rho_a, rho_b)
    assert torch.equal(out_a, out_b)


@pytest.mark.parametrize("S", [1, 2])
def test_given_start_matches_the_layerwise_engine(S):
    pb = conv_problem("base", 16, depth=(0, 8), block=3)
    net = ldb.Net(pb["specs"])
    args = args_of(pb)
    _, rho0 = ldb.ld_bound(net, *args, n_iters=5, return_rho=True)      # an FP32 start
    a = ldb.ld_bound(net, *args, n_iters=3, opts=fused(S, init="given"), rho_in=rho0).cpu().numpy()
    b = ldb.ld_bound(net, *args, n_iters=3, opts=ldb.Options(precision="bf16", engine="layerwise", init="given"),
                     rho_in=rho0).cpu().numpy()
    fin = np.isfinite(b)
    assert np.array_equal(np.isfinite(a), fin)
    assert np.max(rel(a[fin], b[fin])) < 1e-5


def test_full_size_base_call():
    """The Base call of the benchmark (256 subdomains, split depth 0-8, 100
    iterations) on the fused tensor-core engine: sampled subdomains against
    the BF16 oracle and the FP64 oracle, the gap to the FP32 engine over the
    whole batch."""
    pb = conv_problem("base", 256, depth=(0, 8), block=0)
    out = run_gpu(pb, 100, fused(2))
    rows = np.array([0, 1, 128, 255])
    ref = run_oracle(pb, 100, rows=rows)
    fin = np.isfinite(ref)
    assert np.max(rel(out[rows][fin], ref[fin])) < FULL_RUN_MAX
    exact = run_oracle(pb, 100, operands="fp64", rows=rows)
    assert np.max(rel(out[rows][fin], exact[fin])) < GAP_MAX
    f32 = run_gpu(pb, 100, ldb.Options())
    both = np.isfinite(out) & np.isfinite(f32)
    gap = rel(out[both], f32[both])
    assert np.median(gap) < FULL_RUN_MEDIAN and gap.max() < GAP_MAX


def test_autotuner_reports_the_bf16_engine():
    """LD_ENGINE_AUTO with BF16 iterations times the layer-wise and the fused
    tensor-core engines and caches its choice per batch size; ld_net_tuned
    reports it (FP32 and BF16 choices are kept apart)."""
    pb = conv_problem("base", 32, depth=(0, 8), block=4)
    net = ldb.Net(pb["specs"])
    assert net.tuned(32, "bf16") == (None, 0, 0)
    run_gpu(pb, 4, ldb.Options(precision="bf16"), net)
    eng, tile, threads = net.tuned(32, "bf16")
    assert (eng, threads) in (("layerwise", 0), ("fused", 512))
    assert eng != "fused" or tile in (1, 2)
    assert net.tuned(32, "fp32") == (None, 0, 0)
    run_gpu(pb, 4, ldb.Options(), net)
    assert net.tuned(32, "fp32")[0] in ("layerwise", "fused")
