"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every check uses a library
routine (torch conv2d, SciPy HiGHS LP/MILP, torch.optim.Adam), a closed form,
brute force, or an identity the paper proves.
"""
import os

import numpy as np
import pytest
import torch

import oracle
from oracle import lp
from paper_2104_06718_gb300 import synth
from helpers import oracle_net, tiny_problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def lists(net, lb, ub):
    L = [None] + [lb[k] for k in range(1, net.n)]
    U = [None] + [ub[k] for k in range(1, net.n)]
    return L, U


def row(lst, i):
    return [None] + [x[i] for x in lst[1:]]


def zeros_like_rho(L):
    return [None] + [np.zeros_like(x) for x in L[1:]]


# ---------------------------------------------------------------- layers

@pytest.mark.parametrize("cin,cout,k,s,p,h", [(3, 8, 4, 2, 1, 32), (8, 16, 4, 2, 1, 16), (8, 8, 3, 1, 1, 16), (2, 3, 3, 2, 0, 7)])
def test_conv_matrix_matches_torch_conv(cin, cout, k, s, p, h):
    rng = np.random.default_rng(0)
    W = rng.normal(size=(cout, cin, k, k))
    b = rng.normal(size=cout)
    lay = oracle.Layer("conv", W, b, in_shape=(cin, h, h), stride=s, pad=p)
    x = rng.normal(size=(2, cin, h, h))
    ref = torch.nn.functional.conv2d(torch.tensor(x), torch.tensor(W), torch.tensor(b), stride=s, padding=p)
    got = lay.forward(x.reshape(2, -1))
    np.testing.assert_allclose(got, ref.reshape(2, -1).numpy(), rtol=1e-12, atol=1e-12)
    # transposed pass = adjoint of the conv (torch conv_transpose2d)
    r = rng.normal(size=ref.shape)
    out_pad = h - ((ref.shape[-1] - 1) * s - 2 * p + k)
    reft = torch.nn.functional.conv_transpose2d(torch.tensor(r), torch.tensor(W), stride=s, padding=p,
                                                output_padding=out_pad)
    np.testing.assert_allclose(lay.transposed(r.reshape(2, -1)), reft.reshape(2, -1).numpy(), rtol=1e-12, atol=1e-12)


def test_fold_margin_is_logit_difference():
    rng = np.random.default_rng(1)
    W = rng.normal(size=(10, 7))
    b = rng.normal(size=10)
    c = np.zeros(10)
    c[3], c[8] = 1.0, -1.0
    Wf, bf = oracle.fold_margin(W, b, c)
    x = rng.normal(size=7)
    z = W @ x + b
    assert abs((Wf @ x + bf)[0] - (z[3] - z[8])) < 1e-12


# ---------------------------------------------------------------- IBP

def test_ibp_single_layer_is_exact_range():
    """For one affine layer the interval bound is the exact range over the box:
    the minimum of each row is attained at a box corner (brute force)."""
    rng = np.random.default_rng(2)
    W = rng.normal(size=(4, 3))
    b = rng.normal(size=4)
    net = oracle.Net([oracle.Layer("fc", W, b), oracle.Layer("fc", rng.normal(size=(1, 4)), np.zeros(1))])
    l0 = rng.uniform(-1, 0, size=(1, 3))
    u0 = rng.uniform(0, 1, size=(1, 3))
    lb, ub = oracle.ibp_bounds(net, l0, u0)
    corners = np.array([[l0[0, j] if (m >> j) & 1 == 0 else u0[0, j] for j in range(3)] for m in range(8)])
    vals = corners @ W.T + b
    np.testing.assert_allclose(lb[1][0], vals.min(axis=0), atol=1e-12)
    np.testing.assert_allclose(ub[1][0], vals.max(axis=0), atol=1e-12)


def test_ibp_is_sound_on_samples():
    specs, net, l0, u0, lb, ub = tiny_problem(0)
    xs = synth.random_box_points(l0[0], u0[0], 4000, seed=7)
    x = xs
    for k in range(1, net.n + 1):
        xh = net.L(k).forward(x)
        assert np.all(xh >= lb[k] - 1e-12) and np.all(xh <= ub[k] + 1e-12)
        x = np.maximum(xh, 0)


# ---------------------------------------------------------------- per-subdomain IBP after splits

def test_split_ibp_hand_worked_chain():
    """x0 in [-1, 1], x_hat_1 = x0, x_hat_2 = 2 relu(x_hat_1) + 1 (worked by hand).
    Root IBP: x_hat_2 in [1, 3].  Split -1 on neuron 1 fixes relu(x_hat_1) = 0,
    so the recomputed bound of x_hat_2 is [1, 1]; split +1 keeps x_hat_1 in
    [0, 1] and x_hat_2 in [1, 3]."""
    net = oracle.Net([oracle.Layer("fc", np.array([[1.0]]), np.zeros(1)),
                      oracle.Layer("fc", np.array([[2.0]]), np.array([1.0])),
                      oracle.Layer("fc", np.array([[1.0]]), np.zeros(1))])
    l0, u0 = np.array([[-1.0]]), np.array([[1.0]])
    masks = np.array([[0, 0], [-1, 0], [1, 0]], dtype=np.int8)
    lb, ub, empty = oracle.ibp_bounds_split(net, l0, u0, masks)
    np.testing.assert_array_equal(lb[1][:, 0], [-1.0, -1.0, 0.0])
    np.testing.assert_array_equal(ub[1][:, 0], [1.0, 0.0, 1.0])
    np.testing.assert_array_equal(lb[2][:, 0], [1.0, 1.0, 1.0])
    np.testing.assert_array_equal(ub[2][:, 0], [3.0, 1.0, 3.0])
    assert not empty.any()


def _split_problem(i, B=24, depth=(0, 4)):
    specs, net, l0, u0, lb, ub = tiny_problem(i)
    Lr = np.concatenate([lb[k] for k in range(1, net.n)], axis=1)
    Ur = np.concatenate([ub[k] for k in range(1, net.n)], axis=1)
    amb = np.nonzero((Lr[0] < 0) & (Ur[0] > 0))[0]
    masks = synth.split_masks(Lr.shape[1], B, amb, depth, block=40 + i)
    return net, l0, u0, lb, ub, masks


@pytest.mark.parametrize("i", range(3))
def test_split_ibp_without_splits_is_root_ibp(i):
    net, l0, u0, lb, ub, masks = _split_problem(i)
    masks[:] = 0
    ls, us, empty = oracle.ibp_bounds_split(net, l0, u0, masks)
    for k in range(1, net.n):
        np.testing.assert_allclose(ls[k], np.broadcast_to(lb[k], ls[k].shape), rtol=0, atol=1e-12)
        np.testing.assert_allclose(us[k], np.broadcast_to(ub[k], us[k].shape), rtol=0, atol=1e-12)
    assert not empty.any()


@pytest.mark.parametrize("i", range(3))
def test_split_ibp_is_tighter_than_root_clamp(i):
    """IBP is monotone in its input intervals, so recomputing after the clamp
    can only tighten the root bounds clamped by the same masks."""
    net, l0, u0, lb, ub, masks = _split_problem(i)
    ls, us, _ = oracle.ibp_bounds_split(net, l0, u0, masks)
    lc, uc, _ = oracle.apply_masks(net, [None] + [np.broadcast_to(lb[k], ls[k].shape) for k in range(1, net.n)],
                                   [None] + [np.broadcast_to(ub[k], us[k].shape) for k in range(1, net.n)], masks)
    strict = False
    for k in range(1, net.n):
        assert np.all(ls[k] >= lc[k] - 1e-12) and np.all(us[k] <= uc[k] + 1e-12)
        strict |= bool(np.any(ls[k] > lc[k] + 1e-9) or np.any(us[k] < uc[k] - 1e-9))
    assert strict  # splits on layer 1 do tighten layer 2 here


@pytest.mark.parametrize("i", range(3))
def test_split_ibp_is_sound_on_samples(i):
    """Every sampled input whose pre-activations satisfy a subdomain's splits
    has pre-activations inside that subdomain's recomputed bounds."""
    net, l0, u0, lb, ub, masks = _split_problem(i, B=8, depth=(1, 3))
    offs = oracle.split_offsets(net)
    xs = synth.random_box_points(l0[0], u0[0], 20000, seed=11 + i)
    pre = []
    x = xs
    for k in range(1, net.n):
        xh = net.L(k).forward(x)
        pre.append(xh)
        x = np.maximum(xh, 0)
    flat = np.concatenate(pre, axis=1)
    ls, us, _ = oracle.ibp_bounds_split(net, l0, u0, masks)
    checked = 0
    for b in range(masks.shape[0]):
        m = masks[b]
        ok = np.all((m <= 0) | (flat >= 0), axis=1) & np.all((m >= 0) | (flat <= 0), axis=1)
        pts = flat[ok]
        checked += len(pts)
        for k in range(1, net.n):
            seg = pts[:, offs[k - 1]:offs[k]]
            assert np.all(seg >= ls[k][b] - 1e-9) and np.all(seg <= us[k][b] + 1e-9)
    assert checked > 1000


# ---------------------------------------------------------------- identities of the paper

@pytest.mark.parametrize("i", range(4))
def test_zero_dual_equals_ibp(i):
    """Sec. 7.2: IBP corresponds to all duals set to zero."""
    specs, net, l0, u0, lb, ub = tiny_problem(i)
    L, U = lists(net, lb, ub)
    q0 = oracle.dual_value(net, l0, u0, L, U, zeros_like_rho(L))
    assert abs(q0[0] - lb[net.n][0, 0]) < 1e-12


@pytest.mark.parametrize("i", range(4))
def test_crown_init_equals_propagation_bound(i):
    """Prop. 3: q at rho = mu_bar of Eq. (salman-assignment) equals the closed
    form Eq. (bounds-propagation)."""
    specs, net, l0, u0, lb, ub = tiny_problem(i)
    L, U = lists(net, lb, ub)
    rho, lam = oracle.crown_init(net, L, U)
    q = oracle.dual_value(net, l0, u0, L, U, rho)
    d = oracle.propagation_bound(net, l0, u0, L, U, rho, lam)
    assert abs(q[0] - d[0]) < 1e-12


def crown_backsubstitution(net, l0, u0, L, U):
    """Textbook CROWN lower bound by explicit back-substitution of linear
    relaxations: keep x_hat_n >= a^T x_k + c and replace x_k by its lower or
    upper linear relaxation according to the sign of a (written independently
    of the dual assignment)."""
    n = net.n
    a = np.asarray(net.L(n).mat, dtype=np.float64)[0].copy()
    c = net.L(n).bias_vector()[0]
    for k in range(n - 1, 0, -1):
        l, u = L[k][0], U[k][0]
        # relaxation of x_k = relu(x_hat_k): upper  a_up*x_hat + b_up, lower a_lo*x_hat
        a_up = np.zeros_like(l)
        b_up = np.zeros_like(l)
        a_lo = np.zeros_like(l)
        pas = l >= 0
        blk = u <= 0
        amb = ~pas & ~blk
        a_up[pas] = 1.0
        a_lo[pas] = 1.0
        a_up[amb] = u[amb] / (u[amb] - l[amb])
        b_up[amb] = -l[amb] * u[amb] / (u[amb] - l[amb])
        a_lo[amb] = (u[amb] >= -l[amb]).astype(float)
        pos = a >= 0
        slope = np.where(pos, a_lo, a_up)
        c = c + np.sum(np.where(pos, 0.0, a * b_up))
        a = a * slope                      # coefficient on x_hat_k
        Wk = net.L(k).mat
        Wk = Wk.toarray() if hasattr(Wk, "toarray") else Wk
        c = c + a @ net.L(k).bias_vector()
        a = a @ Wk                         # coefficient on x_{k-1}
    return c + np.sum(np.minimum(a * l0[0], a * u0[0]))


@pytest.mark.parametrize("i", range(4))
def test_crown_matches_textbook_backsubstitution(i):
    specs, net, l0, u0, lb, ub = tiny_problem(i)
    L, U = lists(net, lb, ub)
    rho, lam = oracle.crown_init(net, L, U)
    q = oracle.dual_value(net, l0, u0, L, U, rho)
    assert abs(q[0] - crown_backsubstitution(net, l0, u0, L, U)) < 1e-12


@pytest.mark.parametrize("i", range(4))
def test_weak_duality_random_duals(i):
    """Any rho gives a valid lower bound (Sec. 3.1): q(rho) <= f(x) on samples
    and <= the exact minimum (MILP)."""
    specs, net, l0, u0, lb, ub = tiny_problem(i)
    L, U = lists(net, lb, ub)
    xs = synth.random_box_points(l0[0], u0[0], 2000, seed=11 + i)
    fmin = net.evaluate(xs).min()
    exact = lp.exact_min_milp(net, l0[0], u0[0], row(L, 0), row(U, 0))
    assert exact <= fmin + 1e-9
    for s in range(5):
        rho = [None] + [r.astype(np.float64) for r in synth.random_duals([L[1].shape[1], L[2].shape[1]], 1, seed=100 + s, scale=0.5)]
        q = oracle.dual_value(net, l0, u0, L, U, rho)[0]
        assert q <= exact + 1e-9


@pytest.mark.parametrize("i", range(4))
def test_strong_duality_lp_multipliers(i):
    """Prop. 1: max q = optimum of the Planet LP.  q at the LP's agreement-row
    multipliers equals p*; every Adam iterate stays at or below p*; p* is at
    or below the exact minimum."""
    specs, net, l0, u0, lb, ub = tiny_problem(i)
    L, U = lists(net, lb, ub)
    res = lp.planet_lp(net, l0[0], u0[0], row(L, 0), row(U, 0))
    assert res.status == 0
    rho = [None] + [r[None, :] for r in res.rho[1:]]
    q = oracle.dual_value(net, l0, u0, L, U, rho)[0]
    assert abs(q - res.p_star) <= 1e-6 * max(1.0, abs(res.p_star))
    rho0, _ = oracle.crown_init(net, L, U)
    run = oracle.supergradient_adam(net, l0, u0, L, U, rho0, 200)
    assert np.all(run.q_trace <= res.p_star + 1e-9)
    assert run.q_final[0] <= res.p_star + 1e-9
    exact = lp.exact_min_milp(net, l0[0], u0[0], row(L, 0), row(U, 0))
    assert res.p_star <= exact + 1e-9


def test_long_run_approaches_lp_optimum():
    """Prop. 1 in practice: a long decaying-step run closes most of the gap."""
    specs, net, l0, u0, lb, ub = tiny_problem(1)
    L, U = lists(net, lb, ub)
    res = lp.planet_lp(net, l0[0], u0[0], row(L, 0), row(U, 0))
    rho0, _ = oracle.crown_init(net, L, U)
    q_init = oracle.dual_value(net, l0, u0, L, U, rho0)[0]
    run = oracle.supergradient_adam(net, l0, u0, L, U, rho0, 3000,
                                    oracle.AdamSettings(alpha0=1e-2, alpha_end=1e-5))
    gap0 = res.p_star - q_init
    gap = res.p_star - run.q_final[0]
    assert 0 <= gap < 0.05 * gap0


@pytest.mark.parametrize("i", range(3))
def test_exact_min_enumeration_matches_milp(i):
    """Two independent exact solvers of Eq. (noncvx_pb) agree (small nets)."""
    specs = synth.make_mlp([4, 6, 5, 1], seed=500 + i)
    net = oracle_net(specs)
    l0 = np.full((1, 4), -0.5)
    u0 = np.full((1, 4), 0.5)
    lb, ub = oracle.ibp_bounds(net, l0, u0)
    L, U = lists(net, lb, ub)
    e1 = lp.exact_min_enumeration(net, l0[0], u0[0], row(L, 0), row(U, 0))
    e2 = lp.exact_min_milp(net, l0[0], u0[0], row(L, 0), row(U, 0))
    assert abs(e1 - e2) < 1e-7
    xs = synth.random_box_points(l0[0], u0[0], 5000, seed=3)
    assert e1 <= net.evaluate(xs).min() + 1e-9


# ---------------------------------------------------------------- closed forms

def read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split("=")
                vals[k.strip()] = float(v)
    return vals


def single_relu_net(w, b, c, d):
    return oracle.Net([oracle.Layer("fc", np.array([[w]]), np.array([b])),
                       oracle.Layer("fc", np.array([[c]]), np.array([d]))])


@pytest.mark.parametrize("case", ["single_relu_neg.txt", "single_relu_pos.txt"])
def test_single_relu_closed_form(case):
    """One ambiguous ReLU: the Planet hull of Eq. (planet-relu-hull) is exact
    for a monotone objective, so LP = exact min = d + c*relu(l) (c >= 0) or
    d + c*relu(u) (c < 0).  Values worked by hand in tests/golden."""
    g = read_golden(case)
    net = single_relu_net(g["w"], g["b"], g["c"], g["d"])
    l0 = np.array([[g["l0"]]])
    u0 = np.array([[g["u0"]]])
    lb, ub = oracle.ibp_bounds(net, l0, u0)
    assert abs(lb[1][0, 0] - g["lhat"]) < 1e-12 and abs(ub[1][0, 0] - g["uhat"]) < 1e-12
    L, U = lists(net, lb, ub)
    res = lp.planet_lp(net, l0[0], u0[0], row(L, 0), row(U, 0))
    assert abs(res.p_star - g["min"]) < 1e-9
    q = oracle.dual_value(net, l0, u0, L, U, [None, res.rho[1][None, :]])[0]
    assert abs(q - g["min"]) < 1e-9
    # the dual at a hand-picked rho from the golden file
    q_r = oracle.dual_value(net, l0, u0, L, U, [None, np.array([[g["rho"]]])])[0]
    assert abs(q_r - g["q_at_rho"]) < 1e-12
    run = oracle.supergradient_adam(net, l0, u0, L, U, [None, np.zeros((1, 1))], 400,
                                    oracle.AdamSettings(alpha0=0.1, alpha_end=1e-3))
    assert run.q_final[0] <= g["min"] + 1e-12
    assert g["min"] - run.q_final[0] < 1e-2


# ---------------------------------------------------------------- Adam = library Adam

def test_adam_step_matches_torch_adam():
    """The ascent update is Adam (Kingma & Ba) with the linear step decay of
    Sec. 7.2: torch.optim.Adam(maximize=True) fed the oracle's supergradients
    reproduces the oracle's rho trajectory."""
    specs, net, l0, u0, lb, ub = tiny_problem(2)
    L, U = lists(net, lb, ub)
    rho0, _ = oracle.crown_init(net, L, U)
    T = 25
    s = oracle.AdamSettings()
    run = oracle.supergradient_adam(net, l0, u0, L, U, rho0, T, s)
    params = [torch.tensor(rho0[k], dtype=torch.float64, requires_grad=True) for k in (1, 2)]
    opt = torch.optim.Adam(params, lr=s.alpha0, betas=(s.beta1, s.beta2), eps=s.eps, maximize=True)
    for t in range(T):
        rho = [None] + [p.detach().numpy().copy() for p in params]
        sol = oracle.inner_minimisation(net, l0, u0, L, U, rho)
        sg = oracle.supergradient(sol)
        for p, k in zip(params, (1, 2)):
            p.grad = torch.tensor(sg[k])
        for gr in opt.param_groups:
            gr["lr"] = oracle.step_size(t, T, s)
        opt.step()
    for p, k in zip(params, (1, 2)):
        np.testing.assert_allclose(p.detach().numpy(), run.rho[k], rtol=1e-12, atol=1e-14)


def test_step_size_schedule_endpoints():
    s = oracle.AdamSettings(alpha0=1e-2, alpha_end=1e-4)
    assert oracle.step_size(0, 100, s) == 1e-2
    assert abs(oracle.step_size(99, 100, s) - 1e-4) < 1e-18
    assert oracle.step_size(0, 1, s) == 1e-2


# ---------------------------------------------------------------- masks

def test_infeasible_mask_gives_inf():
    specs, net, l0, u0, lb, ub = tiny_problem(0)
    offs = oracle.split_offsets(net)
    flat_l = np.concatenate([lb[k] for k in range(1, net.n)], axis=1)
    flat_u = np.concatenate([ub[k] for k in range(1, net.n)], axis=1)
    blocking = np.nonzero(flat_u[0] < 0)[0]
    passing = np.nonzero(flat_l[0] > 0)[0]
    masks = np.zeros((3, flat_l.shape[1]), np.int8)
    masks[1, blocking[0]] = 1     # force a blocking ReLU on: empty domain
    if passing.size:
        masks[2, passing[0]] = -1  # force a passing ReLU off: empty domain
    out, _, _ = oracle.ld_bound(net, l0, u0, flat_l, flat_u, None, masks, 5)
    assert np.isfinite(out[0]) and out[1] == np.inf
    if passing.size:
        assert out[2] == np.inf


def test_splits_tighten_lp_and_cover_exact_min():
    """Sec. 2.3.2: splitting an ambiguous ReLU into its two phases.  The LP of
    each child is at least the parent's, and the smaller child LP is still at
    or below the exact minimum (the two children cover the domain)."""
    specs, net, l0, u0, lb, ub = tiny_problem(0)
    L, U = lists(net, lb, ub)
    flat_l = np.concatenate([L[k] for k in range(1, net.n)], axis=1)
    flat_u = np.concatenate([U[k] for k in range(1, net.n)], axis=1)
    amb = np.nonzero((flat_l[0] < 0) & (flat_u[0] > 0))[0]
    parent = lp.planet_lp(net, l0[0], u0[0], row(L, 0), row(U, 0)).p_star
    exact = lp.exact_min_milp(net, l0[0], u0[0], row(L, 0), row(U, 0))
    for j in amb[:4]:
        kids = []
        for sgn in (1, -1):
            m = np.zeros((1, flat_l.shape[1]), np.int8)
            m[0, j] = sgn
            Lc, Uc, empty = oracle.apply_masks(net, oracle.layer_lists(net, flat_l), oracle.layer_lists(net, flat_u), m)
            assert not empty[0]
            kids.append(lp.planet_lp(net, l0[0], u0[0], row(Lc, 0), row(Uc, 0)).p_star)
        assert min(kids) >= parent - 1e-9
        assert min(kids) <= exact + 1e-9


def test_all_ambiguous_split_closes_gap():
    """With every ambiguous ReLU split, the hull is exact: the LP of the
    subdomain equals the exact minimum of that activation pattern."""
    specs = synth.make_mlp([3, 4, 3, 1], seed=77)
    net = oracle_net(specs)
    l0 = np.full((1, 3), -1.0)
    u0 = np.full((1, 3), 1.0)
    lb, ub = oracle.ibp_bounds(net, l0, u0)
    L, U = lists(net, lb, ub)
    flat_l = np.concatenate([L[k] for k in range(1, net.n)], axis=1)
    flat_u = np.concatenate([U[k] for k in range(1, net.n)], axis=1)
    amb = np.nonzero((flat_l[0] < 0) & (flat_u[0] > 0))[0]
    rng = np.random.default_rng(5)
    m = np.zeros((1, flat_l.shape[1]), np.int8)
    m[0, amb] = rng.choice([-1, 1], size=amb.size)
    Lc, Uc, empty = oracle.apply_masks(net, oracle.layer_lists(net, flat_l), oracle.layer_lists(net, flat_u), m)
    p = lp.planet_lp(net, l0[0], u0[0], row(Lc, 0), row(Uc, 0))
    if p.status != 0:
        pytest.skip("pattern infeasible for this draw")
    ex = lp.exact_min_enumeration(net, l0[0], u0[0], row(Lc, 0), row(Uc, 0))
    assert abs(p.p_star - ex) < 1e-7


# ---------------------------------------------------------------- Danskin gradients

def test_danskin_gradients_match_finite_differences():
    specs, net, l0, u0, lb, ub = tiny_problem(3)
    L, U = lists(net, lb, ub)
    rho0, _ = oracle.crown_init(net, L, U)
    run = oracle.supergradient_adam(net, l0, u0, L, U, rho0, 30)
    rho = run.rho
    info = [None] + [(np.zeros_like(L[k], bool), np.zeros_like(L[k], bool)) for k in range(1, net.n)]
    g = oracle.danskin_gradients(net, l0, u0, L, U, info, rho, np.ones(1))
    h = 1e-6

    def q_with(mod):
        layers = []
        for k in range(1, net.n + 1):
            lay = net.L(k)
            W, b = lay.W.copy(), lay.b.copy()
            W, b = mod(k, W, b)
            layers.append(oracle.Layer("fc", W, b))
        return oracle.dual_value(oracle.Net(layers), l0, u0, L, U, rho)[0]

    rng = np.random.default_rng(9)
    for k in range(1, net.n + 1):
        for _ in range(4):
            i = rng.integers(net.L(k).W.shape[0])
            j = rng.integers(net.L(k).W.shape[1])

            def modW(kk, W, b, s):
                if kk == k:
                    W[i, j] += s
                return W, b
            fd = (q_with(lambda kk, W, b: modW(kk, W, b, h)) - q_with(lambda kk, W, b: modW(kk, W, b, -h))) / (2 * h)
            assert abs(fd - g.gW[k][i, j]) < 1e-6

            def modb(kk, W, b, s):
                if kk == k:
                    b[i] += s
                return W, b
            fd = (q_with(lambda kk, W, b: modb(kk, W, b, h)) - q_with(lambda kk, W, b: modb(kk, W, b, -h))) / (2 * h)
            assert abs(fd - g.gb[k][i]) < 1e-6
    for j in range(l0.shape[1]):
        for arr, gr in ((l0, g.gl0), (u0, g.gu0)):
            a1, a2 = arr.copy(), arr.copy()
            a1[0, j] += h
            a2[0, j] -= h
            if arr is l0:
                fd = (oracle.dual_value(net, a1, u0, L, U, rho) - oracle.dual_value(net, a2, u0, L, U, rho))[0] / (2 * h)
            else:
                fd = (oracle.dual_value(net, l0, a1, L, U, rho) - oracle.dual_value(net, l0, a2, L, U, rho))[0] / (2 * h)
            assert abs(fd - gr[0, j]) < 1e-6
    for k in range(1, net.n):
        for j in range(L[k].shape[1]):
            for which in ("l", "u"):
                A1 = [None] + [x.copy() for x in (L if which == "l" else U)[1:]]
                A2 = [None] + [x.copy() for x in (L if which == "l" else U)[1:]]
                A1[k][0, j] += h
                A2[k][0, j] -= h
                if which == "l":
                    fd = (oracle.dual_value(net, l0, u0, A1, U, rho) - oracle.dual_value(net, l0, u0, A2, U, rho))[0] / (2 * h)
                    assert abs(fd - g.glb[k][0, j]) < 1e-6
                else:
                    fd = (oracle.dual_value(net, l0, u0, L, A1, rho) - oracle.dual_value(net, l0, u0, L, A2, rho))[0] / (2 * h)
                    assert abs(fd - g.gub[k][0, j]) < 1e-6


def test_danskin_bias_gradient_closed_form():
    """dq/db_k = -rho_k (rho_n = -1): q is affine in the biases at fixed argmins."""
    specs, net, l0, u0, lb, ub = tiny_problem(1)
    L, U = lists(net, lb, ub)
    rho, _ = oracle.crown_init(net, L, U)
    info = [None] + [(np.zeros_like(L[k], bool), np.zeros_like(L[k], bool)) for k in range(1, net.n)]
    g = oracle.danskin_gradients(net, l0, u0, L, U, info, rho, np.ones(1))
    for k in range(1, net.n):
        np.testing.assert_allclose(g.gb[k], -rho[k][0], atol=0)
    assert g.gb[net.n][0] == 1.0


def test_conv_weight_gradient_matches_torch_autograd():
    """The conv weight gradient of the Danskin adjoint is the usual conv
    weight-gradient (torch autograd of conv2d)."""
    rng = np.random.default_rng(4)
    W = rng.normal(size=(4, 3, 4, 4))
    lay = oracle.Layer("conv", W, np.zeros(4), in_shape=(3, 8, 8), stride=2, pad=1)
    x = rng.normal(size=(2, 3 * 64))
    og = rng.normal(size=(2, lay.n_out))
    G = oracle.conv_weight_grad(lay, og, x)
    Wt = torch.tensor(W, requires_grad=True)
    y = torch.nn.functional.conv2d(torch.tensor(x.reshape(2, 3, 8, 8)), Wt, stride=2, padding=1)
    (y.reshape(2, -1) * torch.tensor(og)).sum().backward()
    np.testing.assert_allclose(G, Wt.grad.numpy(), rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------- pins have teeth

def test_planted_vertex_sign_error_is_caught(monkeypatch):
    """Plant a plausible mistake in the oracle ((u,u) vertex value with the
    wrong sign of g) and check that the strong-duality pin fails."""
    specs, net, l0, u0, lb, ub = tiny_problem(0)
    L, U = lists(net, lb, ub)
    res = lp.planet_lp(net, l0[0], u0[0], row(L, 0), row(U, 0))
    rho = [None] + [r[None, :] for r in res.rho[1:]]
    good = oracle.dual_value(net, l0, u0, L, U, rho)[0]
    orig = oracle.ld_oracle.inner_minimisation

    def bad(net_, l0_, u0_, lb_, ub_, rho_, ball_eps=None):
        rho2 = [None] + [r for r in rho_[1:]]
        sol = orig(net_, l0_, u0_, lb_, ub_, rho2)
        # recompute with the transposed pass negated (a transposed-operand slip)
        sol2 = orig(net_, l0_, u0_, lb_, ub_, [None] + [-r for r in rho2[1:]])
        return sol2
    monkeypatch.setattr(oracle.ld_oracle, "inner_minimisation", bad)
    wrong = oracle.ld_oracle.dual_value(net, l0, u0, L, U, rho)[0]
    assert abs(good - res.p_star) < 1e-6
    assert abs(wrong - res.p_star) > 1e-3


def test_planted_dropped_term_is_caught(monkeypatch):
    """Dropping the rho^T (x_hat_B - x_hat_A) term of one layer breaks Prop. 3."""
    specs, net, l0, u0, lb, ub = tiny_problem(1)
    L, U = lists(net, lb, ub)
    rho, lam = oracle.crown_init(net, L, U)
    sol = oracle.inner_minimisation(net, l0, u0, L, U, rho)
    q_drop = sol.xA[net.n][:, 0] + np.sum(rho[2] * (sol.xB[2] - sol.xA[2]), axis=1)
    d = oracle.propagation_bound(net, l0, u0, L, U, rho, lam)
    assert abs(sol.q[0] - d[0]) < 1e-12
    assert abs(q_drop[0] - d[0]) > 1e-6


@pytest.mark.parametrize("i", range(3))
def test_dual_value_is_the_exact_minimum(i):
    """q is read from the exact per-subproblem minima; the Lagrangian at the
    returned (tie-margin) point is never below it, exceeds it by at most the
    margins, and at random duals (no near-ties) equals it."""
    specs, net, l0, u0, lb, ub = tiny_problem(i)
    L, U = lists(net, lb, ub)
    rho, _ = oracle.crown_init(net, L, U)
    sol = oracle.inner_minimisation(net, l0, u0, L, U, rho)
    slack = sum(np.sum(oracle.TIE_REL * (np.abs(rho[k]) + np.abs(sol.g[k]))
                       * np.maximum(np.abs(L[k]), np.abs(U[k]))) for k in range(1, net.n))
    assert sol.q_point[0] >= sol.q[0] - 1e-12
    assert sol.q_point[0] - sol.q[0] <= slack + 1e-12
    rr = [None] + [r.astype(np.float64) for r in synth.random_duals([L[1].shape[1], L[2].shape[1]], 1, seed=3)]
    s2 = oracle.inner_minimisation(net, l0, u0, L, U, rr)
    assert abs(s2.q_point[0] - s2.q[0]) < 1e-12


# --------------------------------------------------------------------------
# BF16 operand emulation (the precision of the tensor-core passes)
# --------------------------------------------------------------------------

def test_round_bf16_matches_torch_bfloat16():
    """round_bf16 is round-to-nearest-even to bfloat16 (the library conversion)."""
    rng = np.random.default_rng(11)
    a = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-6, 6, 20000),
                        [0.0, -0.0, 1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 65504.0, 1e-30]])
    a = a.astype(np.float32).astype(np.float64)
    ref = torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).double().numpy()
    assert np.array_equal(oracle.round_bf16(a), ref)


def _bf16_exact_net():
    """A small conv + FC net whose weights are exactly representable in bf16."""
    rng = np.random.default_rng(5)
    Wc = rng.integers(-4, 5, size=(4, 2, 3, 3)) / 8.0
    bc = rng.integers(-4, 5, size=4) / 16.0
    conv = oracle.Layer("conv", Wc, bc, (2, 6, 6), 2, 1)
    Wf = rng.integers(-4, 5, size=(5, conv.n_out)) / 4.0
    fc = oracle.Layer("fc", Wf, rng.integers(-3, 4, size=5) / 8.0)
    top = oracle.Layer("fc", rng.integers(-3, 4, size=(1, 5)) / 2.0, np.array([0.25]))
    return oracle.Net([conv, fc, top])


def test_bf16_passes_equal_exact_passes_on_representable_values():
    """With bf16-representable weights, duals, activations and box offsets the
    BF16 passes are the exact passes (rounding is the only difference)."""
    net = _bf16_exact_net()
    rng = np.random.default_rng(6)
    B = 3
    l0 = rng.integers(0, 8, size=(B, net.widths[0])) / 8.0
    u0 = l0 + rng.integers(1, 4, size=l0.shape) / 16.0
    ps, ex = oracle.BF16Passes(net, l0, u0), oracle.ExactPasses(net)
    for k in (1, 2):
        r = rng.integers(-8, 9, size=(B, net.widths[k])) / 16.0
        assert np.allclose(ps.transposed(k, r), ex.transposed(k, r), rtol=0, atol=1e-12)
    x0 = np.where(rng.random(l0.shape) < 0.5, l0, u0)
    assert np.allclose(ps.forward(1, x0), ex.forward(1, x0), rtol=0, atol=1e-12)
    x1 = rng.integers(0, 8, size=(B, net.widths[1])) / 4.0
    assert np.allclose(ps.forward(2, x1), ex.forward(2, x1), rtol=0, atol=1e-12)


def test_bf16_passes_round_what_they_should():
    """Off the bf16 grid, the forward pass of layer 1 keeps the box centre
    exact (only x0 - c0 is rounded) and hidden layers round weights and
    inputs; the top layer is untouched."""
    net = _bf16_exact_net()
    rng = np.random.default_rng(7)
    l0 = rng.random((2, net.widths[0])) + 100.0       # pixel values far above the box width
    u0 = l0 + 1e-3
    ps, ex = oracle.BF16Passes(net, l0, u0), oracle.ExactPasses(net)
    x0 = np.where(rng.random(l0.shape) < 0.5, l0, u0)
    # exact weights and a box offset +-5e-4 (rounded by ~2^-9 relative): the
    # error is that of the offset, not of the pixel values near 100
    err = np.abs(ps.forward(1, x0) - ex.forward(1, x0))
    scale = np.abs(net.L(1).W).sum() * 5e-4
    assert err.max() < 2 ** -8 * scale
    r = rng.standard_normal((2, 1))
    assert np.array_equal(ps.transposed(3, r), ex.transposed(3, r))
    x1 = rng.standard_normal((2, net.widths[1])) * 3
    assert np.allclose(ps.forward(2, x1), ex.forward(2, oracle.round_bf16(x1)), rtol=0, atol=1e-12)
