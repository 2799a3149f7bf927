"""GPU: propagation-based intermediate bounds (CROWN, WK, layer-wise best;
Sec. 2.2.1, Sec. 2.2.3, Sec. 7.2) against oracle/intermediate.py.

The device bounds are rounded outward (every FP32 pass's rounding error is
bounded a priori and subtracted), so they must contain the oracle's FP64
bounds, and lie within 1e-4 of them relative to max(|l|, |u|) + 1:
  * root bounds of two properties on the Base, Wide and Deep convnets
    (layer-wise best), and CROWN-only and WK-only on Base and the tiny MLPs;
  * bounds recomputed per subdomain after its splits (Base, Deep): the split
    clamp enters every later layer; without splits they equal the root
    bounds of each subdomain's property bitwise;
  * LD bounds on top of them match the oracle after 3 iterations (1e-5).
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import intermediate as ib
from paper_2104_06718_gb300 import binding as ldb
from paper_2104_06718_gb300 import synth
from helpers import conv_problem, outward_f32, tiny_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_06718_gb300 import build
    build.build()
    ldb.load_library()


def flat(net, lst):
    return np.concatenate([lst[k] for k in range(1, net.n)], axis=1)


def check_outward(gl, gu, fl, fu, tol=1e-4):
    gl = np.asarray(gl, np.float64)
    gu = np.asarray(gu, np.float64)
    scale = np.maximum(np.abs(fl), np.abs(fu)) + 1.0
    assert np.all(gl <= fl + 1e-12 * scale), ("lower bound not outward", np.max((gl - fl) / scale))
    assert np.all(gu >= fu - 1e-12 * scale), ("upper bound not outward", np.max((fu - gu) / scale))
    assert np.max((fl - gl) / scale) < tol and np.max((gu - fu) / scale) < tol, \
        (np.max((fl - gl) / scale), np.max((gu - fu) / scale))


@pytest.mark.parametrize("name", ["base", "wide", "deep"])
def test_root_layerwise_best_contains_oracle(name):
    pb = conv_problem(name, 1, props=(0, 1))
    net = ldb.Net(pb["specs"])
    on = pb["net"]
    lbk, ubk = ldb.ld_intermediate_bounds_propagated(net, pb["l0"], pb["u0"], rules="best")
    fl, fu = ib.crown_wk_bounds(on, pb["l0"], pb["u0"])
    check_outward(lbk.cpu().numpy(), ubk.cpu().numpy(), flat(on, fl), flat(on, fu))


@pytest.mark.parametrize("rule", ["crown", "wk"])
def test_single_rule_bounds_contain_oracle(rule):
    pb = conv_problem("base", 1, props=(2,))
    net = ldb.Net(pb["specs"])
    on = pb["net"]
    lbk, ubk = ldb.ld_intermediate_bounds_propagated(net, pb["l0"], pb["u0"], rules=rule)
    fl, fu = ib.crown_wk_bounds(on, pb["l0"], pb["u0"], rules=(rule,))
    check_outward(lbk.cpu().numpy(), ubk.cpu().numpy(), flat(on, fl), flat(on, fu))
    for i in range(6):
        specs, tn, l0, u0, _, _ = tiny_problem(i)
        tnet = ldb.Net(specs)
        gl, gu = ldb.ld_intermediate_bounds_propagated(tnet, l0.astype(np.float32), u0.astype(np.float32), rules=rule)
        fl, fu = ib.crown_wk_bounds(tn, l0, u0, rules=(rule,))
        check_outward(gl.cpu().numpy(), gu.cpu().numpy(), flat(tn, fl), flat(tn, fu))


def _split_problem(name, B, block):
    """Masks over ReLUs ambiguous under the oracle's root layer-wise best bounds."""
    pb = conv_problem(name, B, depth=(0, 3), props=(0, 1), block=block)
    on = pb["net"]
    fl, fu = ib.crown_wk_bounds(on, pb["l0"][:1], pb["u0"][:1])
    l, u = flat(on, fl)[0], flat(on, fu)[0]
    amb = np.nonzero((l < 0) & (u > 0))[0]
    pb["masks"] = synth.split_masks(l.size, B, amb, (0, 3), block=block)
    return pb


@pytest.mark.parametrize("name,B", [("base", 5), ("deep", 3)])
def test_per_subdomain_bounds_after_splits_contain_oracle(name, B):
    pb = _split_problem(name, B, block=17)
    net = ldb.Net(pb["specs"])
    on = pb["net"]
    lbk, ubk = ldb.ld_intermediate_bounds_propagated(net, pb["l0"], pb["u0"], rules="best", masks=pb["masks"],
                                                     prop=pb["prop"])
    ls, us, empty = ib.crown_wk_bounds_split(on, pb["l0"], pb["u0"], pb["masks"], pb["prop"])
    gl, gu = lbk.cpu().numpy(), ubk.cpu().numpy()
    fl, fu = flat(on, ls), flat(on, us)
    ok = ~empty
    assert ok.sum() >= 2
    check_outward(gl[ok], gu[ok], fl[ok], fu[ok])
    # without splits each subdomain gets its property's root bounds, bitwise
    zero = np.zeros_like(pb["masks"])
    l2, u2 = ldb.ld_intermediate_bounds_propagated(net, pb["l0"], pb["u0"], rules="best", masks=zero,
                                                   prop=pb["prop"])
    lr, ur = ldb.ld_intermediate_bounds_propagated(net, pb["l0"], pb["u0"], rules="best")
    idx = torch.as_tensor(pb["prop"].astype(np.int64), device="cuda")
    assert torch.equal(l2, lr[idx]) and torch.equal(u2, ur[idx])


def test_ld_bound_on_propagated_bounds_matches_oracle():
    """ld_bound with the layer-wise best root bounds as its intermediate bounds,
    against the oracle given the oracle's own best bounds (outward-rounded to
    float32 the same way), after 3 iterations."""
    pb = conv_problem("base", 12, depth=(0, 0), block=21)
    on = pb["net"]
    fl, fu = ib.crown_wk_bounds(on, pb["l0"], pb["u0"])
    lbk, ubk = outward_f32(flat(on, fl), flat(on, fu))
    amb = np.nonzero((lbk[0] < 0) & (ubk[0] > 0))[0]
    masks = synth.split_masks(lbk.shape[1], pb["B"], amb, (0, 6), block=21)
    net = ldb.Net(pb["specs"])
    out = ldb.ld_bound(net, pb["l0"], pb["u0"], lbk, ubk, pb["prop"], masks, n_iters=3).cpu().numpy()
    ref, _, _ = oracle.ld_bound(on, pb["l0"].astype(np.float64), pb["u0"].astype(np.float64),
                                lbk.astype(np.float64), ubk.astype(np.float64), pb["prop"], masks, 3)
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(out), fin)
    rel = np.abs(out[fin] - ref[fin]) / np.maximum(np.abs(ref[fin]), 1.0)
    assert rel.max() < 1e-5
    # the device's own propagated bounds give the same bounds to within their rounding
    gl, gu = ldb.ld_intermediate_bounds_propagated(net, pb["l0"], pb["u0"], rules="best")
    out2 = ldb.ld_bound(net, pb["l0"], pb["u0"], gl, gu, pb["prop"], masks, n_iters=3).cpu().numpy()
    assert np.array_equal(np.isfinite(out2), fin)
    assert np.max(np.abs(out2[fin] - out[fin]) / np.maximum(np.abs(out[fin]), 1.0)) < 1e-3


def test_propagated_bounds_argument_errors():
    pb = conv_problem("base", 1, props=(0, 1))
    net = ldb.Net(pb["specs"])
    with pytest.raises(ldb.LDError) as e:
        ldb.ld_intermediate_bounds_propagated(net, pb["l0"], pb["u0"], n_rows=3)  # no map for 2 boxes
    assert e.value.code == ldb.LD_ERR_ARG
    lib = ldb.load_library()
    assert lib.ld_intermediate_bounds_propagated(net.handle, None, None, 1, None, None, 1, 3, None, None,
                                                 None) == ldb.LD_ERR_ARG
    l0 = torch.as_tensor(pb["l0"], device="cuda")
    out = torch.empty((2, net.N), device="cuda")
    assert lib.ld_intermediate_bounds_propagated(net.handle, l0.data_ptr(), l0.data_ptr(), 2, None, None, 2, 4,
                                                 out.data_ptr(), out.data_ptr(), None) == ldb.LD_ERR_ARG
