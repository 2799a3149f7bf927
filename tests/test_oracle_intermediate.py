"""Pins of the oracle's CROWN / WK intermediate bounds (Sec. 2.2.3, Sec. 7.2)
to things other than the oracle itself: exact ranges by corner enumeration,
network values at sampled inputs, the Planet LP and exact minima on tiny
nets, and Prop. 3 at the network output (the LD dual at the CROWN start is
the CROWN bound)."""
import itertools

import numpy as np
import pytest

import oracle
from oracle import intermediate as ib
from oracle import lp
from helpers import conv_problem, tiny_problem


def pre_activations(net, x0):
    """x_hat_k for k = 1..n at inputs x0 [M, n_0] (the network itself)."""
    out, x = [None], x0
    for k in range(1, net.n + 1):
        xh = net.L(k).forward(x)
        out.append(xh)
        x = np.maximum(xh, 0.0)
    return out


def corners(l0, u0):
    """All 2^n0 vertices of the box [l0, u0] (l0, u0: [n0])."""
    n0 = l0.shape[0]
    bits = np.array(list(itertools.product([0.0, 1.0], repeat=n0)))
    return l0[None, :] + bits * (u0 - l0)[None, :]


def shifted(net, delta):
    """The same net with delta added to the biases of its hidden layers."""
    layers = []
    for k in range(1, net.n + 1):
        lay = net.L(k)
        b = lay.b + (delta if k < net.n else 0.0)
        layers.append(oracle.Layer(lay.kind, lay.W, b, lay.in_shape, lay.stride, lay.pad))
    return oracle.Net(layers)


def truncated(net, k, j, sign=1.0):
    """Layers 1..k-1 and the scalar objective sign * x_hat_k[j]."""
    lay = net.L(k)
    top = oracle.Layer("fc", sign * np.asarray(lay.mat[j:j + 1].todense() if hasattr(lay.mat, "todense")
                                               else lay.mat[j:j + 1]),
                       sign * lay.bias_vector()[j:j + 1])
    return oracle.Net([net.L(i) for i in range(1, k)] + [top])


@pytest.mark.parametrize("i", range(6))
def test_first_layer_is_the_exact_range_of_an_affine_map(i):
    _, net, l0, u0, _, _ = tiny_problem(i)
    vals = pre_activations(net, corners(l0[0], u0[0]))[1]
    for rule in ib.RULES:
        lo, up = ib.layer_bounds(net, 1, l0, u0, [None], [None], rule)
        assert np.allclose(lo[0], vals.min(axis=0), rtol=0, atol=1e-12)
        assert np.allclose(up[0], vals.max(axis=0), rtol=0, atol=1e-12)


@pytest.mark.parametrize("i", range(3))
def test_affine_regime_is_exact_and_blocking_regime_is_constant(i):
    """Every hidden ReLU passing: the net is affine on the box, and both
    relaxations are the identity, so every bound is the exact range (attained
    at a corner).  Every ReLU blocking: x_hat_k = b_k for k >= 2."""
    _, net, l0, u0, _, _ = tiny_problem(i)
    up_net = shifted(net, 100.0)
    pts = pre_activations(up_net, corners(l0[0], u0[0]))
    lb, ub = ib.crown_wk_bounds(up_net, l0, u0, include_output=True)
    for k in range(1, up_net.n + 1):
        assert np.allclose(lb[k][0], pts[k].min(axis=0), rtol=1e-12, atol=1e-9)
        assert np.allclose(ub[k][0], pts[k].max(axis=0), rtol=1e-12, atol=1e-9)
    down_net = shifted(net, -100.0)
    lb, ub = ib.crown_wk_bounds(down_net, l0, u0, include_output=True)
    for k in range(2, down_net.n + 1):
        b = down_net.L(k).bias_vector()
        assert np.array_equal(lb[k][0], b) and np.array_equal(ub[k][0], b)


def _check_contains(net, l0, u0, lb, ub, x, last):
    pts = pre_activations(net, x)
    for k in range(1, last + 1):
        scale = np.maximum(np.abs(lb[k]), np.abs(ub[k])) + 1.0
        assert np.all(pts[k] >= lb[k] - 1e-9 * scale), f"layer {k} lower bound cut off a value"
        assert np.all(pts[k] <= ub[k] + 1e-9 * scale), f"layer {k} upper bound cut off a value"


@pytest.mark.parametrize("i", range(6))
def test_bounds_contain_the_values_at_sampled_inputs_tiny(i):
    _, net, l0, u0, _, _ = tiny_problem(i)
    rng = np.random.default_rng(10 + i)
    x = np.concatenate([corners(l0[0], u0[0]),
                        l0 + rng.uniform(size=(2000, l0.shape[1])) * (u0 - l0)])
    for rules in [("crown",), ("wk",), ib.RULES]:
        lb, ub = ib.crown_wk_bounds(net, l0, u0, rules=rules, include_output=True)
        _check_contains(net, l0, u0, [None] + [a[0] for a in lb[1:]], [None] + [a[0] for a in ub[1:]], x, net.n)


@pytest.mark.parametrize("name", ["base", "deep"])
def test_bounds_contain_the_values_at_sampled_inputs_convnet(name):
    pb = conv_problem(name, 1)
    net = pb["net"]
    l0, u0 = pb["l0"].astype(np.float64), pb["u0"].astype(np.float64)
    rng = np.random.default_rng(7)
    # box corners at random and interior points
    x = np.concatenate([np.where(rng.uniform(size=(200, l0.shape[1])) < 0.5, l0, u0),
                        l0 + rng.uniform(size=(200, l0.shape[1])) * (u0 - l0)])
    lb, ub = ib.crown_wk_bounds(net, l0, u0)
    _check_contains(net, l0, u0, [None] + [a[0] for a in lb[1:]], [None] + [a[0] for a in ub[1:]], x, net.n - 1)
    # the layer-wise best is tighter than interval propagation on these nets
    ilb, iub = oracle.ibp_bounds(net, l0, u0)
    for k in range(2, net.n):
        assert np.mean(ub[k] - lb[k]) < np.mean(iub[k] - ilb[k])


@pytest.mark.parametrize("i", range(4))
def test_propagation_bounds_are_below_the_lp_and_the_exact_minimum(i):
    """For every neuron of layer 2 and for the output: CROWN and WK lower
    bounds <= the Planet LP optimum over the same subnetwork and earlier
    bounds (the convex hull is the tightest relaxation of each ReLU) <= the
    exact minimum (activation-pattern enumeration)."""
    _, net, l0, u0, _, _ = tiny_problem(i)
    lb, ub = ib.crown_wk_bounds(net, l0, u0, include_output=True)
    for k in (2, net.n):
        lows = {r: ib.layer_bounds(net, k, l0, u0, lb, ub, r) for r in ib.RULES}
        for j in range(net.L(k).n_out):
            for sign in (1.0, -1.0):
                sub = truncated(net, k, j, sign)
                L = [None] + [lb[m][0] for m in range(1, k)]
                U = [None] + [ub[m][0] for m in range(1, k)]
                p = lp.planet_lp(sub, l0[0], u0[0], L, U)
                assert p.status == 0
                for r in ib.RULES:
                    bound = lows[r][0][0, j] if sign > 0 else -lows[r][1][0, j]
                    assert bound <= p.p_star + 1e-7 * max(1.0, abs(p.p_star)), (k, j, sign, r)
                try:
                    exact = lp.exact_min_enumeration(sub, l0[0], u0[0], L, U, max_ambiguous=8)
                except ValueError:
                    continue  # too many ambiguous ReLUs to enumerate quickly
                assert p.p_star <= exact + 1e-7 * max(1.0, abs(exact))


@pytest.mark.parametrize("i", range(6))
def test_crown_bound_of_the_output_is_the_dual_at_the_crown_start(i):
    """Prop. 3: with the same intermediate bounds, the LD dual value at the
    CROWN initial duals (and the closed-form propagation bound at them) is
    the CROWN bound obtained here by direct substitution."""
    _, net, l0, u0, _, _ = tiny_problem(i)
    lb, ub = ib.crown_wk_bounds(net, l0, u0)
    low, _ = ib.layer_bounds(net, net.n, l0, u0, lb, ub, "crown")
    rho, lam = oracle.crown_init(net, lb, ub)
    q = oracle.dual_value(net, l0, u0, lb, ub, rho)
    pb = oracle.propagation_bound(net, l0, u0, lb, ub, rho, lam)
    assert np.allclose(low[:, 0], q, rtol=1e-10, atol=1e-10)
    assert np.allclose(low[:, 0], pb, rtol=1e-10, atol=1e-10)


def test_rules_differ_only_in_the_ambiguous_lower_slope():
    l = np.array([[-2.0, -1.0, 0.5, -3.0, -1.0]])
    u = np.array([[1.0, 3.0, 2.0, -0.5, 1.0]])
    lo_c, bar_c, bb_c = ib.relaxation(l, u, "crown")
    lo_w, bar_w, bb_w = ib.relaxation(l, u, "wk")
    assert np.array_equal(bar_c, bar_w) and np.array_equal(bb_c, bb_w)
    # ambiguous (-2, 1): CROWN lower slope 0 (u < -l), WK u/(u-l) = 1/3
    assert lo_c[0, 0] == 0.0 and lo_w[0, 0] == pytest.approx(1.0 / 3.0)
    # ambiguous (-1, 3): CROWN 1 (u >= -l), WK 3/4; upper slope 3/4, intercept 3/4
    assert lo_c[0, 1] == 1.0 and lo_w[0, 1] == pytest.approx(0.75)
    assert bar_c[0, 1] == pytest.approx(0.75) and bb_c[0, 1] == pytest.approx(0.75)
    # passing (0.5, 2): identity; blocking (-3, -0.5): zero
    assert lo_c[0, 2] == lo_w[0, 2] == bar_c[0, 2] == 1.0 and bb_c[0, 2] == 0.0
    assert lo_c[0, 3] == lo_w[0, 3] == bar_c[0, 3] == 0.0 and bb_c[0, 3] == 0.0
    # u == -l: CROWN takes slope 1 (the footnote's u >= -l)
    assert lo_c[0, 4] == 1.0


# ------------------------------------------------------------------ per-subdomain recomputation after splits

def _split_masks(net, lb, ub, rng, n_sub, l0=None, u0=None):
    """Subdomain 0 unsplit; the others split 1-3 root-ambiguous units of layer 1
    or 2.  Phases at random, or (with the box given) the phases of a random
    input's own pre-activations, so that the subdomain contains that input."""
    offs = oracle.split_offsets(net)
    amb = [j for k in (1, 2) for j in range(offs[k - 1], offs[k])
           if lb[k][0, j - offs[k - 1]] < 0 < ub[k][0, j - offs[k - 1]]]
    masks = np.zeros((n_sub, offs[-1]), np.int8)
    for b in range(1, n_sub):
        units = rng.choice(amb, size=rng.integers(1, 4), replace=False)
        if l0 is None:
            masks[b, units] = rng.choice([-1, 1], size=len(units))
        else:
            x = l0 + rng.uniform(size=l0.shape) * (u0 - l0)
            pts = pre_activations(net, x)
            flat = np.concatenate([pts[k] for k in range(1, net.n)], axis=1)[0]
            masks[b, units] = np.where(flat[units] >= 0, 1, -1)
    return masks


@pytest.mark.parametrize("i", range(4))
def test_split_bounds_contain_every_sampled_input_that_meets_the_splits(i):
    _, net, l0, u0, _, _ = tiny_problem(i)
    rlb, rub = ib.crown_wk_bounds(net, l0, u0)
    rng = np.random.default_rng(100 + i)
    masks = _split_masks(net, rlb, rub, rng, 12)
    lb, ub, empty = ib.crown_wk_bounds_split(net, l0, u0, masks)
    # no splits: the root bounds; every split unit clamped to its phase
    for k in range(1, net.n):
        assert np.array_equal(lb[k][0], rlb[k][0]) and np.array_equal(ub[k][0], rub[k][0])
    offs = oracle.split_offsets(net)
    for k in range(1, net.n):
        m = masks[:, offs[k - 1]:offs[k]]
        assert np.all(lb[k][m > 0] >= 0.0) and np.all(ub[k][m < 0] <= 0.0)
    x = l0 + rng.uniform(size=(20000, l0.shape[1])) * (u0 - l0)
    pts = pre_activations(net, x)
    flat = np.concatenate([pts[k] for k in range(1, net.n)], axis=1)
    checked = 0
    for b in range(masks.shape[0]):
        ok = np.all(np.where(masks[b] > 0, flat >= 0, True) & np.where(masks[b] < 0, flat <= 0, True), axis=1)
        if not ok.any():
            continue
        assert not empty[b]
        for k in range(1, net.n):
            scale = np.maximum(np.abs(lb[k][b]), np.abs(ub[k][b])) + 1.0
            assert np.all(pts[k][ok] >= lb[k][b] - 1e-9 * scale)
            assert np.all(pts[k][ok] <= ub[k][b] + 1e-9 * scale)
        checked += 1
    assert checked >= 6


@pytest.mark.parametrize("i", range(2))
def test_split_bounds_are_below_the_lp_of_the_subdomain(i):
    """With a subdomain's clamped bounds of layer 1, the Planet LP over them is
    a relaxation of that subdomain; the CROWN/WK bounds of every neuron of
    layer 2 of the subdomain lie below its optimum (above, for upper bounds)."""
    _, net, l0, u0, _, _ = tiny_problem(i)
    rlb, rub = ib.crown_wk_bounds(net, l0, u0)
    masks = _split_masks(net, rlb, rub, np.random.default_rng(200 + i), 5, l0, u0)
    lb, ub, empty = ib.crown_wk_bounds_split(net, l0, u0, masks)
    assert not empty.any()  # every subdomain contains the input its phases came from
    for b in range(1, masks.shape[0]):
        L = [lb[0][b:b + 1]] + [lb[1][b:b + 1]]
        U = [ub[0][b:b + 1]] + [ub[1][b:b + 1]]
        lows = {r: ib.layer_bounds(net, 2, L[0], U[0], L, U, r) for r in ib.RULES}
        for j in range(net.L(2).n_out):
            for sign in (1.0, -1.0):
                p = lp.planet_lp(truncated(net, 2, j, sign), l0[0], u0[0], [None, lb[1][b]], [None, ub[1][b]])
                assert p.status == 0
                for r in ib.RULES:
                    bound = lows[r][0][0, j] if sign > 0 else -lows[r][1][0, j]
                    assert bound <= p.p_star + 1e-7 * max(1.0, abs(p.p_star)), (b, j, sign, r)
            # the recomputed (clamped) best bound of the unit is one of them, clamped
            assert lb[2][b, j] >= min(lows[r][0][0, j] for r in ib.RULES) - 1e-12


def test_split_against_a_unit_that_cannot_pass_is_empty():
    _, net, l0, u0, _, _ = tiny_problem(0)
    rlb, rub = ib.crown_wk_bounds(net, l0, u0)
    dead = np.nonzero(rub[1][0] < 0)[0]
    live = np.nonzero(rlb[1][0] > 0)[0]
    assert dead.size and live.size
    masks = np.zeros((3, oracle.split_offsets(net)[-1]), np.int8)
    masks[1, dead[0]] = 1      # force a blocked unit to pass: l = 0 > u
    masks[2, live[0]] = -1     # force a passing unit to block: u = 0 < l
    _, _, empty = ib.crown_wk_bounds_split(net, l0, u0, masks)
    assert empty.tolist() == [False, True, True]


# ------------------------------------------------------------------ planted mistakes

def _pins_hold(i=1):
    """The sampled-value and Prop. 3 pins on tiny problem i; False if one fails."""
    try:
        test_bounds_contain_the_values_at_sampled_inputs_tiny(i)
        test_crown_bound_of_the_output_is_the_dual_at_the_crown_start(i)
        test_affine_regime_is_exact_and_blocking_regime_is_constant(i)
    except AssertionError:
        return False
    return True


def test_planted_mistakes_in_the_relaxation_are_caught(monkeypatch):
    good = ib.relaxation
    assert _pins_hold()

    def no_intercept(l, u, rule):
        a_low, a_bar, b_bar = good(l, u, rule)
        return a_low, a_bar, np.zeros_like(b_bar)

    def swapped(l, u, rule):
        a_low, a_bar, b_bar = good(l, u, rule)
        return a_bar, a_low, b_bar

    def crown_threshold_flipped(l, u, rule):
        a_low, a_bar, b_bar = good(l, u, rule)
        if rule == "crown":
            amb = oracle.classify(l, u) == 2
            a_low = np.where(amb, 1.0 - a_low, a_low)
        return a_low, a_bar, b_bar

    for bad in (no_intercept, swapped, crown_threshold_flipped):
        monkeypatch.setattr(ib, "relaxation", bad)
        assert not all(_pins_hold(i) for i in range(3)), f"{bad.__name__} passed every pin"
    monkeypatch.setattr(ib, "relaxation", good)
