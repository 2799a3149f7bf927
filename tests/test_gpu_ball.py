"""GPU: l2-ball input domains (Sec. 3.2.1) through the C ABI.

ld_intermediate_bounds_ball (layer 1 exact over the ball up to outward
rounding, then interval propagation) and ld_bound_ball (the LD dual with P0
minimised over the ball: x0* = c + eps g0/||g0||, value -g0.c - eps||g0||)
against the FP64 oracle (oracle.l2 and oracle.ld_bound with ball_eps):

  * interval bounds: contain the oracle's exact ones; layer 1 within 1e-6,
    the propagated layers within the 1e-4 of the box interval tests
  * short runs (T = 1, 3): within 1e-5 of the oracle (FP32 iterations)
  * long runs (T = 100): the FP32 chaos floor of the box tests
  * the FP64 final bound at the returned rho: at or below the oracle's q at
    that rho, within 1e-9 of it
  * a net affine over the ball (every ReLU passing): the CROWN start gives
    the exact minimum -a.c - eps||a|| + b
  * weak duality against sampled points of the ball; a zero radius equals
    the degenerate box [c, c]; radii that are negative or NaN set the status
    word; BF16 iterations are refused
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import l2
from paper_2104_06718_gb300 import binding as ldb
from paper_2104_06718_gb300 import synth
from helpers import folded_specs, oracle_net, outward_f32

pytestmark = pytest.mark.gpu

FULL_RUN_MAX = 1e-3
FULL_RUN_MEDIAN = 3e-4


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


def flat(net, lst):
    return np.concatenate([lst[k] for k in range(1, net.n)], axis=1)


def ball_problem(name, B, eps, depth=(0, 8), block=0):
    """Convnet of the benchmark family, the ball of radius eps around the
    centre of property 0's image box, oracle interval bounds over the ball
    rounded outward to FP32, split masks over the root-ambiguous ReLUs."""
    specs = synth.make_convnet(name)
    l0, u0, margin = synth.image_property(0)
    fspecs = folded_specs(specs, margin)
    net = oracle_net(fspecs)
    c = ((l0.astype(np.float64) + u0.astype(np.float64)) / 2).astype(np.float32)[None]
    e = np.array([eps], np.float32)
    lb, ub = l2.ball_ibp_bounds(net, c.astype(np.float64), e.astype(np.float64))
    lbk, ubk = outward_f32(flat(net, lb), flat(net, ub))
    amb = np.nonzero((lbk[0] < 0) & (ubk[0] > 0))[0]
    masks = synth.split_masks(lbk.shape[1], B, amb, depth, block=block)
    prop = np.zeros(B, np.int32)
    return dict(specs=fspecs, net=net, c=c, eps=e, lbk=lbk, ubk=ubk, prop=prop, masks=masks, B=B)


def run_gpu(pb, T, opts=None, net=None, **kw):
    net = net or ldb.Net(pb["specs"])
    return ldb.ld_bound_ball(net, pb["c"], pb["eps"], pb["lbk"], pb["ubk"], pb["prop"], pb["masks"], n_iters=T,
                             opts=opts, **kw)


def run_oracle(pb, T, rows=None, **kw):
    prop = pb["prop"] if rows is None else pb["prop"][rows]
    masks = pb["masks"] if rows is None else pb["masks"][rows]
    c = pb["c"].astype(np.float64)
    out, _, _ = oracle.ld_bound(pb["net"], c, c, pb["lbk"].astype(np.float64), pb["ubk"].astype(np.float64), prop,
                                masks, T, ball_eps=pb["eps"].astype(np.float64), **kw)
    return out


@pytest.mark.parametrize("name,eps", [("base", 0.1), ("wide", 0.05), ("deep", 0.05), ("base", 0.0)])
def test_intermediate_bounds_contain_the_exact_ones(name, eps):
    pb = ball_problem(name, 1, eps)
    on = pb["net"]
    net = ldb.Net(pb["specs"])
    lbk, ubk, out_lb = ldb.ld_intermediate_bounds_ball(net, pb["c"], pb["eps"], want_output_lb=True)
    assert net.sync_status() == ldb.LD_OK
    lbk, ubk = lbk.cpu().numpy()[0].astype(np.float64), ubk.cpu().numpy()[0].astype(np.float64)
    lb, ub = l2.ball_ibp_bounds(on, pb["c"].astype(np.float64), pb["eps"].astype(np.float64))
    el, eu = flat(on, lb)[0], flat(on, ub)[0]
    scale = np.maximum(np.maximum(np.abs(el), np.abs(eu)), 1.0)
    assert np.all(lbk <= el + 1e-12 * scale) and np.all(ubk >= eu - 1e-12 * scale)
    # layer 1: FP64 up to one outward FP32 rounding; above it the outward FP32
    # interval propagation of the box tests (same 1e-4)
    n1 = on.L(1).n_out
    assert np.max(rel(lbk[:n1], el[:n1])) < 1e-6 and np.max(rel(ubk[:n1], eu[:n1])) < 1e-6
    assert np.max(rel(lbk, el)) < 1e-4 and np.max(rel(ubk, eu)) < 1e-4
    assert out_lb.item() <= lb[on.n][0, 0] + 1e-9 * max(1.0, abs(lb[on.n][0, 0]))
    assert rel(out_lb.item(), lb[on.n][0, 0]) < 1e-4


def test_intermediate_bounds_on_a_fully_connected_first_layer():
    specs = synth.tiny_mlp(0)
    on = oracle_net(specs)
    c = (synth.tiny_box(0)[0][0].astype(np.float64) + 0.1).astype(np.float32)
    eps = np.array([0.3, 0.0, 1.5], np.float32)
    cs = np.stack([c, c - 0.2, c + 0.3]).astype(np.float32)
    net = ldb.Net(specs)
    lbk, ubk = ldb.ld_intermediate_bounds_ball(net, cs, eps)
    lb, ub = l2.ball_ibp_bounds(on, cs.astype(np.float64), eps.astype(np.float64))
    el, eu = flat(on, lb), flat(on, ub)
    g, h = lbk.cpu().numpy().astype(np.float64), ubk.cpu().numpy().astype(np.float64)
    scale = np.maximum(np.maximum(np.abs(el), np.abs(eu)), 1.0)
    assert np.all(g <= el + 1e-12 * scale) and np.all(h >= eu - 1e-12 * scale)
    n1 = on.L(1).n_out
    assert np.max(rel(g[:, :n1], el[:, :n1])) < 1e-6 and np.max(rel(h[:, :n1], eu[:, :n1])) < 1e-6
    assert np.max(rel(g, el)) < 1e-4 and np.max(rel(h, eu)) < 1e-4


@pytest.mark.parametrize("name", ["base", "deep"])
@pytest.mark.parametrize("T", [1, 3])
def test_short_runs_match_the_oracle(name, T):
    pb = ball_problem(name, 6, 0.1 if name == "base" else 0.05, block=2)
    out = run_gpu(pb, T).cpu().numpy()
    ref = run_oracle(pb, T)
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(out), fin)
    assert np.max(rel(out[fin], ref[fin])) < 1e-5


def test_long_runs_match_the_oracle():
    pb = ball_problem("base", 8, 0.1, block=5)
    out = run_gpu(pb, 100).cpu().numpy()
    ref = run_oracle(pb, 100)
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(out), fin)
    r = rel(out[fin], ref[fin])
    assert np.max(r) < FULL_RUN_MAX and np.median(r) < FULL_RUN_MEDIAN


def test_fp64_final_bound_at_the_returned_rho():
    """The FP64 final bound at rho_T is a lower bound of the exact q(rho_T)
    (the oracle's value at the same FP32 rho) and close to it."""
    pb = ball_problem("base", 8, 0.1, block=4)
    on = pb["net"]
    out, rho = run_gpu(pb, 20, return_rho=True)
    out, rho = out.cpu().numpy(), rho.cpu().numpy().astype(np.float64)
    c = pb["c"].astype(np.float64)
    lb = oracle.layer_lists(on, pb["lbk"][pb["prop"]].astype(np.float64))
    ub = oracle.layer_lists(on, pb["ubk"][pb["prop"]].astype(np.float64))
    lb, ub, empty = oracle.apply_masks(on, lb, ub, pb["masks"])
    keep = np.nonzero(~empty)[0]
    sel = lambda lst: [None] + [lst[k][keep] for k in range(1, on.n)]
    q = oracle.dual_value(on, c[pb["prop"][keep]], c[pb["prop"][keep]], sel(lb), sel(ub),
                          sel(oracle.layer_lists(on, rho)), ball_eps=pb["eps"][pb["prop"][keep]].astype(np.float64))
    mag = np.maximum(np.abs(q), 1.0)
    assert np.all(out[keep] <= q + 1e-12 * mag)
    assert np.max((q - out[keep]) / mag) < 1e-9
    assert np.all(np.isinf(out[empty]))


def _affine_specs():
    """The tiny MLP with each hidden layer's biases raised, layer by layer,
    until its interval lower bound over the ball (radius 0.25 around c) is at
    least 1: every ReLU passes there and the net is affine over the ball."""
    specs = list(synth.tiny_mlp(2))
    c = np.linspace(-0.5, 0.5, specs[0].W.shape[1]).astype(np.float32)
    eps = np.float32(0.25)
    for k in range(len(specs) - 1):
        lb, _ = l2.ball_ibp_bounds(oracle_net(specs), c[None].astype(np.float64), np.array([float(eps)]))
        shift = np.float32(max(0.0, 1.0 - lb[k + 1].min()))
        s = specs[k]
        specs[k] = synth.LayerSpec(s.kind, s.W, (s.b + shift).astype(np.float32), s.in_shape)
    return specs, c, eps


def test_affine_net_gives_the_exact_minimum():
    specs, c, eps = _affine_specs()
    on = oracle_net(specs)
    net = ldb.Net(specs)
    lbk, ubk = ldb.ld_intermediate_bounds_ball(net, c[None], np.array([eps]))
    assert float(lbk.min()) > 0.0
    out = ldb.ld_bound_ball(net, c[None], np.array([eps]), lbk, ubk, B=1, n_iters=0).item()
    # over the ball the net is x -> a.x + beta (every ReLU the identity)
    a = np.asarray(on.L(on.n).mat, np.float64)
    for k in range(on.n - 1, 0, -1):
        a = a @ np.asarray(on.L(k).mat, np.float64)
    a = a[0]
    c64 = c.astype(np.float64)
    exact = on.evaluate(c64[None])[0] - float(eps) * np.linalg.norm(a)
    assert out <= exact + 1e-12 * max(1.0, abs(exact))
    assert rel(out, exact) < 1e-6
    # later iterates stay below the minimum (weak duality)
    assert ldb.ld_bound_ball(net, c[None], np.array([eps]), lbk, ubk, B=1, n_iters=20).item() <= exact + 1e-9


def test_weak_duality_against_points_of_the_ball():
    pb = ball_problem("base", 1, 0.1)
    out = run_gpu(pb, 60).item()
    pts = l2.ball_points(pb["c"][0].astype(np.float64), float(pb["eps"][0]), 256, seed=5)
    vals = pb["net"].evaluate(pts)
    assert np.all(out <= vals)


def test_zero_radius_is_the_degenerate_box():
    pb = ball_problem("base", 4, 0.0, block=1)
    net = ldb.Net(pb["specs"])
    a = run_gpu(pb, 10, net=net).cpu().numpy()
    b = ldb.ld_bound(net, pb["c"], pb["c"], pb["lbk"], pb["ubk"], pb["prop"], pb["masks"], n_iters=10,
                     opts=ldb.Options(engine="layerwise")).cpu().numpy()
    c = pb["c"].astype(np.float64)
    ref, _, _ = oracle.ld_bound(pb["net"], c, c, pb["lbk"].astype(np.float64), pb["ubk"].astype(np.float64),
                                pb["prop"], pb["masks"], 10)
    assert np.max(rel(a, ref)) < 1e-5 and np.max(rel(b, ref)) < 1e-5


def test_bad_radii_set_the_status_and_bf16_is_refused():
    pb = ball_problem("base", 2, 0.1)
    net = ldb.Net(pb["specs"])
    for bad in (-0.1, np.nan):
        ldb.ld_bound_ball(net, pb["c"], np.array([bad], np.float32), pb["lbk"], pb["ubk"], pb["prop"], pb["masks"],
                          n_iters=2)
        assert net.sync_status() == ldb.LD_ERR_NONFINITE
        ldb.ld_intermediate_bounds_ball(net, pb["c"], np.array([bad], np.float32))
        assert net.sync_status() == ldb.LD_ERR_NONFINITE
    run_gpu(pb, 2, net=net)
    assert net.sync_status() == ldb.LD_OK
    with pytest.raises(ldb.LDError):
        run_gpu(pb, 2, opts=ldb.Options(precision="bf16"), net=net)
    with pytest.raises(ldb.LDError):
        run_gpu(pb, 2, opts=ldb.Options(fp64_final=False), net=net)


# ------------------------------------------------------------------ the fused FP32 engine

def fused(S):
    return ldb.Options(engine="fused", tile=S)


def tiny_ball_problem(B, eps=0.5, block=0):
    """The tiny MLP (a fully connected first layer) over a ball around its box
    centre, with the same construction as ball_problem."""
    specs = synth.tiny_mlp(1)
    net = oracle_net(specs)
    l0, u0 = synth.tiny_box(1)
    c = ((l0.astype(np.float64) + u0.astype(np.float64)) / 2).astype(np.float32).reshape(1, -1)
    e = np.array([eps], np.float32)
    lb, ub = l2.ball_ibp_bounds(net, c.astype(np.float64), e.astype(np.float64))
    lbk, ubk = outward_f32(flat(net, lb), flat(net, ub))
    amb = np.nonzero((lbk[0] < 0) & (ubk[0] > 0))[0]
    masks = synth.split_masks(lbk.shape[1], B, amb, (0, 3), block=block)
    return dict(specs=specs, net=net, c=c, eps=e, lbk=lbk, ubk=ubk, prop=np.zeros(B, np.int32), masks=masks, B=B)


@pytest.mark.parametrize("name,S", [("base", 1), ("base", 2), ("deep", 1), ("tiny", 1)])
@pytest.mark.parametrize("T", [1, 3])
def test_fused_engine_short_runs_match_the_oracle(name, S, T):
    pb = tiny_ball_problem(5) if name == "tiny" else \
        ball_problem(name, 7, 0.1 if name == "base" else 0.05, block=3)   # 7: a ragged last CTA for S = 2
    net = ldb.Net(pb["specs"])
    out = run_gpu(pb, T, opts=fused(S), net=net).cpu().numpy()
    ref = run_oracle(pb, T)
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(out), fin)
    assert np.max(rel(out[fin], ref[fin])) < 1e-5
    lay = run_gpu(pb, T, opts=ldb.Options(engine="layerwise"), net=net).cpu().numpy()
    assert np.max(rel(out[fin], lay[fin])) < 1e-5


@pytest.mark.parametrize("S", [1, 2])
def test_fused_engine_long_runs_and_repeatability(S):
    pb = ball_problem("base", 9, 0.1, block=5)
    net = ldb.Net(pb["specs"])
    out, rho = run_gpu(pb, 100, opts=fused(S), net=net, return_rho=True)
    ref = run_oracle(pb, 100)
    o = out.cpu().numpy()
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(o), fin)
    r = rel(o[fin], ref[fin])
    assert np.max(r) < FULL_RUN_MAX and np.median(r) < FULL_RUN_MEDIAN
    # the norm is reduced in a fixed order: a second run is bitwise the same
    out2, rho2 = run_gpu(pb, 100, opts=fused(S), net=net, return_rho=True)
    assert torch.equal(rho, rho2) and torch.equal(out, out2)
