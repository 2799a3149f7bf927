"""Oracle pins for l2-ball input domains (Sec. 3.2.1), CPU only.

The P0 minimiser and value over the ball are pinned to a generic constrained
solver and to sampled points; the first layer's interval bounds over the
ball to sampled points and to the points that attain them; the LD bound over
the ball to weak duality (never above the net at sampled points of the
ball), to an exact closed form on nets that are affine over the ball (every
ReLU passing), and to the value at the centre when the radius is zero.
"""
import numpy as np
import pytest
from scipy.optimize import minimize

import oracle
from oracle import l2
from helpers import oracle_net
from paper_2104_06718_gb300 import synth


def test_ball_argmin_is_the_minimum_of_the_linear_cost():
    rng = np.random.default_rng(1)
    B, n = 4, 10
    g = rng.standard_normal((B, n))
    c = rng.standard_normal((B, n))
    eps = rng.uniform(0.05, 1.0, B)
    x = l2.ball_argmin(g, c, eps)
    v = l2.ball_min(g, c, eps)
    assert np.allclose(-np.sum(g * x, axis=1), v, rtol=0, atol=1e-12)
    assert np.allclose(np.linalg.norm(x - c, axis=1), eps, rtol=1e-12)
    for b in range(B):
        res = minimize(lambda z: -g[b] @ z, c[b], jac=lambda z: -g[b], method="SLSQP",
                       constraints=[{"type": "ineq", "fun": lambda z: eps[b] ** 2 - np.sum((z - c[b]) ** 2),
                                     "jac": lambda z: -2 * (z - c[b])}], options={"ftol": 1e-12, "maxiter": 500})
        assert res.fun == pytest.approx(v[b], abs=1e-7)
        pts = l2.ball_points(c[b], eps[b], 2000, seed=b)
        assert np.all(-(pts @ g[b]) >= v[b] - 1e-12)
    # g = 0: every point is a minimiser; the centre is returned
    assert np.array_equal(l2.ball_argmin(np.zeros((1, n)), c[:1], eps[:1]), c[:1])


@pytest.mark.parametrize("which", ["tiny", "base"])
def test_first_layer_bounds_are_the_exact_range(which):
    if which == "tiny":
        net = oracle_net(synth.tiny_mlp(0))
        c = synth.tiny_box(0)[0][0].astype(np.float64) + 0.1
    else:
        l0, _, margin = synth.image_property(0)
        net = oracle_net(synth.make_convnet("base"), margin)
        c = l0.reshape(-1).astype(np.float64)
    eps = np.array([0.3 if which == "tiny" else 0.05])
    lo, hi = l2.ball_first_layer_bounds(net, c[None], eps)
    pts = l2.ball_points(c, eps[0], 500, seed=3)
    vals = net.L(1).forward(pts)
    assert np.all(vals >= lo - 1e-12) and np.all(vals <= hi + 1e-12)
    # attained: c -+ eps w_j / ||w_j|| for a few neurons
    W = net.L(1).mat
    for j in (0, 7, lo.shape[1] - 1):
        w = np.asarray(W[j].todense()).reshape(-1) if hasattr(W, "todense") else W[j]
        d = w / np.linalg.norm(w)
        assert net.L(1).forward((c - eps[0] * d)[None])[0, j] == pytest.approx(lo[0, j], abs=1e-12)
        assert net.L(1).forward((c + eps[0] * d)[None])[0, j] == pytest.approx(hi[0, j], abs=1e-12)


def _tiny_ball(i, eps):
    net = oracle_net(synth.tiny_mlp(i))
    c = (synth.tiny_box(i)[0][0].astype(np.float64) + synth.tiny_box(i)[1][0].astype(np.float64)) / 2
    lb, ub = l2.ball_ibp_bounds(net, c[None], np.array([eps]))
    return net, c, lb, ub


@pytest.mark.parametrize("i", range(4))
def test_weak_duality_over_the_ball(i):
    net, c, lb, ub = _tiny_ball(i, 0.4)
    B = 1
    C = c[None]
    e = np.array([0.4])
    f_min = net.evaluate(l2.ball_points(c, 0.4, 4000, seed=10 + i)).min()
    rng = np.random.default_rng(i)
    rhos = [[None] + [np.zeros((B, lb[k].shape[1])) for k in range(1, net.n)],
            [None] + [rng.standard_normal((B, lb[k].shape[1])) for k in range(1, net.n)],
            oracle.crown_init(net, lb, ub)[0]]
    for rho in rhos:
        assert oracle.dual_value(net, C, C, lb, ub, rho, ball_eps=e)[0] <= f_min + 1e-9
    res = oracle.supergradient_adam(net, C, C, lb, ub, rhos[2], 50, ball_eps=e)
    assert np.all(res.q_trace <= f_min + 1e-9) and res.q_final[0] <= f_min + 1e-9


def _affine_net():
    """A tiny net whose every ReLU is passing over the ball (each hidden
    layer's biases shifted, layer by layer, until its lower bound is positive):
    (net, centre, radius, lb, ub)."""
    specs = [synth.LayerSpec(s.kind, np.asarray(s.W, np.float64), np.asarray(s.b, np.float64), s.in_shape)
             for s in synth.tiny_mlp(2)]
    c = np.linspace(-0.5, 0.5, specs[0].W.shape[1])
    eps = 0.25
    for k in range(len(specs) - 1):
        lb, _ = l2.ball_ibp_bounds(oracle_net(specs), c[None], np.array([eps]))
        shift = max(0.0, 1.0 - lb[k + 1].min())
        s = specs[k]
        specs[k] = synth.LayerSpec(s.kind, s.W, s.b + shift, s.in_shape)
    net = oracle_net(specs)
    lb, ub = l2.ball_ibp_bounds(net, c[None], np.array([eps]))
    return net, c, eps, lb, ub


def test_net_affine_over_the_ball_is_bounded_exactly():
    """With every ReLU passing over the whole ball the net is affine there:
    min = w^T c + b - eps ||w||, which the LD bound at the CROWN start (rho = g
    exactly for passing ReLUs) meets, and no later iterate exceeds."""
    net, c, eps, lb, ub = _affine_net()
    assert all(np.all(lb[k] > 0) for k in range(1, net.n))
    w = np.asarray(net.L(net.n).mat, np.float64)
    for k in range(net.n - 1, 0, -1):
        w = w @ (net.L(k).mat.toarray() if hasattr(net.L(k).mat, "toarray") else net.L(k).mat)
    exact = net.evaluate(c[None])[0] - eps * np.linalg.norm(w)
    rho0, _ = oracle.crown_init(net, lb, ub)
    q0 = oracle.dual_value(net, c[None], c[None], lb, ub, rho0, ball_eps=np.array([eps]))[0]
    assert q0 == pytest.approx(exact, abs=1e-9)
    res = oracle.supergradient_adam(net, c[None], c[None], lb, ub, rho0, 20, ball_eps=np.array([eps]))
    assert np.all(res.q_trace <= exact + 1e-9)


@pytest.mark.parametrize("i", range(3))
def test_zero_radius_gives_the_value_at_the_centre(i):
    net, c, lb, ub = _tiny_ball(i, 0.0)
    rho0, _ = oracle.crown_init(net, lb, ub)
    q = oracle.dual_value(net, c[None], c[None], lb, ub, rho0, ball_eps=np.array([0.0]))[0]
    assert q == pytest.approx(net.evaluate(c[None])[0], abs=1e-9)


def test_ld_bound_driver_takes_the_ball_per_property():
    net, c, lb, ub = _tiny_ball(1, 0.3)
    flat_l = np.concatenate([lb[k] for k in range(1, net.n)], axis=1)
    flat_u = np.concatenate([ub[k] for k in range(1, net.n)], axis=1)
    masks = np.zeros((2, flat_l.shape[1]), np.int8)
    out, res, keep = oracle.ld_bound(net, c[None], c[None], flat_l, flat_u, None, masks, 10,
                                     ball_eps=np.array([0.3]))
    direct = oracle.supergradient_adam(net, np.repeat(c[None], 2, 0), np.repeat(c[None], 2, 0),
                                       [None] + [np.repeat(lb[k], 2, 0) for k in range(1, net.n)],
                                       [None] + [np.repeat(ub[k], 2, 0) for k in range(1, net.n)],
                                       oracle.crown_init(net, [None] + [np.repeat(lb[k], 2, 0) for k in range(1, net.n)],
                                                         [None] + [np.repeat(ub[k], 2, 0) for k in range(1, net.n)])[0],
                                       10, ball_eps=np.array([0.3, 0.3]))
    assert np.allclose(out, direct.q_final, rtol=0, atol=1e-12)


def test_planted_sign_error_in_the_ball_term_is_caught(monkeypatch):
    """The exact closed form on the affine net sees a wrong sign of the
    eps ||g|| term, and so does weak duality."""
    import oracle.l2 as l2mod
    net, c, eps, lb, ub = _affine_net()
    f_min = net.evaluate(l2.ball_points(c, eps, 4000, seed=10)).min()
    rho, _ = oracle.crown_init(net, lb, ub)
    good = oracle.dual_value(net, c[None], c[None], lb, ub, rho, ball_eps=np.array([eps]))[0]
    assert good <= f_min + 1e-9
    monkeypatch.setattr(l2mod, "ball_min",
                        lambda g, cc, e: -np.sum(g * cc, axis=1) + np.asarray(e).reshape(-1) * np.linalg.norm(g, axis=1))
    bad = oracle.dual_value(net, c[None], c[None], lb, ub, rho, ball_eps=np.array([eps]))[0]
    assert bad > f_min
