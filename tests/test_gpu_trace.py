"""GPU: the per-iterate dual values (ld_bound_trace).

Algorithm 1 evaluates q(rho_t) at every iterate before its update; the
trace [T, B] records it.  Against the FP64 oracle's own trace (AdamResult
.q_trace): after 1-3 steps within 1e-5, along 100 steps within the FP32
floor of the trajectory; row 0 equals the bound at the start and row T the
bound after T steps; the returned bounds and moments are bitwise those of
ld_bound on the layer-wise engine (the evaluation leaves the iteration's
state alone); empty subdomains are +inf.
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
MID_RUN_MAX = 5e-3        # 2.5x the mid-run FP32 floor


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_06718_gb300 import build
    build.build()
    ldb.load_library()


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b) / np.maximum(np.abs(b), 1.0)


def args_of(pb):
    return (pb["l0"], pb["u0"], pb["lbk"], pb["ubk"], pb["prop"], pb["masks"])


def oracle_trace(pb, T):
    out, res, keep = oracle.ld_bound(pb["net"], pb["l0"].astype(np.float64), pb["u0"].astype(np.float64),
                                     pb["lbk"].astype(np.float64), pb["ubk"].astype(np.float64), pb["prop"],
                                     pb["masks"], T)
    return out, res.q_trace, keep


@pytest.mark.parametrize("name", ["base", "deep"])
def test_short_trace_matches_the_oracle(name):
    pb = conv_problem(name, 7, depth=(0, 8), block=3)
    net = ldb.Net(pb["specs"])
    out, tr = ldb.ld_bound_trace(net, *args_of(pb), n_iters=3)
    ref_out, ref_tr, keep = oracle_trace(pb, 3)
    tr = tr.cpu().numpy()
    assert tr.shape == (3, pb["B"])
    assert np.max(rel(tr[:, keep], ref_tr)) < 1e-5
    assert np.max(rel(out.cpu().numpy()[keep], ref_out[keep])) < 1e-5
    # row 0 is q at the CROWN start: the FP64 bound of a zero-step call
    start = ldb.ld_bound(net, *args_of(pb), n_iters=0).cpu().numpy()
    assert np.max(rel(tr[0, keep], start[keep])) < 1e-6


def test_trace_leaves_the_iterations_unchanged():
    pb = conv_problem("base", 9, depth=(0, 8), block=2)
    masks = pb["masks"].copy()
    blk = np.nonzero(pb["ubk"][0] < 0)[0]
    masks[4, blk[0]] = 1          # forced passing on a blocking ReLU: empty
    pb = dict(pb, masks=masks)
    net = ldb.Net(pb["specs"])
    B, N = pb["B"], pb["lbk"].shape[1]
    mv_a = torch.zeros((2, B, N), dtype=torch.float32, device="cuda")
    mv_b = torch.zeros_like(mv_a)
    # 25 steps of a 26-step schedule, so that a 26-step trace continues them
    a, tr = ldb.ld_bound_trace(net, *args_of(pb), n_iters=25, adam_mv=mv_a, opts=ldb.Options(t_total=26))
    b = ldb.ld_bound(net, *args_of(pb), n_iters=25, opts=ldb.Options(engine="layerwise", t_total=26), adam_mv=mv_b)
    assert torch.equal(a, b) and torch.equal(mv_a, mv_b)
    tr = tr.cpu().numpy()
    assert np.all(np.isinf(tr[:, 4])) and np.isinf(a[4].item())
    assert np.all(np.isfinite(np.delete(tr, 4, axis=1)))
    # the next row is q(rho_25), the value the 25-step call bounded in FP64
    _, tr26 = ldb.ld_bound_trace(net, *args_of(pb), n_iters=26)
    tr26 = tr26.cpu().numpy()
    assert np.array_equal(tr26[:25], tr)
    fin = np.isfinite(a.cpu().numpy())
    assert np.max(rel(tr26[25, fin], a.cpu().numpy()[fin])) < 1e-6


def test_long_trace_within_the_fp32_floor():
    pb = conv_problem("base", 8, depth=(0, 8), block=5)
    net = ldb.Net(pb["specs"])
    _, tr = ldb.ld_bound_trace(net, *args_of(pb), n_iters=100)
    _, ref_tr, keep = oracle_trace(pb, 100)
    r = rel(tr.cpu().numpy()[:, keep], ref_tr)
    # the first steps to 1e-5; mid-run the FP32 floor of the trajectory (up
    # to ~2e-3 for single subdomains, tests/test_oracle_fp32_floor.py); the
    # last iterates to the long-run tolerances
    assert np.max(r[:3]) < 1e-5
    assert np.max(r) < MID_RUN_MAX and np.median(r) < FULL_RUN_MEDIAN
    assert np.max(r[-1]) < FULL_RUN_MAX


def test_bf16_trace_is_refused():
    pb = conv_problem("base", 2, depth=(0, 8), block=1)
    net = ldb.Net(pb["specs"])
    with pytest.raises(ldb.LDError):
        ldb.ld_bound_trace(net, *args_of(pb), n_iters=2, opts=ldb.Options(precision="bf16"))
