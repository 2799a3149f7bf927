"""Pins of the proximal-solver oracle (Sec. 3.3, Algorithm 2, Eq.
(optimal-gamma-gauss), App. D) against things other than itself.

  * gamma_k^* equals the minimiser over [0, 1] of the Augmented Lagrangian
    along the Frank-Wolfe segment, found from values of L alone (L is
    quadratic in gamma: three values fix the parabola) and by a dense grid;
  * every block step never increases the Augmented Lagrangian (the segment
    contains gamma = 0);
  * the conditional gradient of block k is the inner minimisation of the
    supergradient method at the Augmented Lagrangian's duals (Sec. 3.3.2);
  * every iterate q(lambda^t) stays at or below the Planet LP optimum (weak
    duality, Sec. 3.1, Prop. 1) and after 1000 iterations the bound is within
    1e-3 of it, on the tiny MLPs, in both settings of the paper;
  * the dual update is Eq. (lambda_updates) with mu = 0 and accumulates the
    momentum of Eq. (momentum_updates) with mu > 0;
  * planted mistakes (the step's sign, a dropped curvature term, a block
    dual without its Augmented-Lagrangian part) make a pin fail;
  * (a measurement) the method's sensitivity to rounding: a relative
    perturbation of 1e-7 of the CROWN start moves the bound after 50
    iterations on the Deep convnet by more than 1e-3 -- far more than the
    supergradient method's ~3e-4 -- which sets the tolerance of the device's
    long runs (tests/test_gpu_proximal.py).
"""
import numpy as np
import pytest

import oracle
from oracle import lp
from oracle import proximal as px
from helpers import conv_problem, oracle_lists, tiny_problem


def _tiny(i):
    specs, on, l0, u0, lb, ub = tiny_problem(i)
    return on, l0, u0, [None] + lb[1:on.n], [None] + ub[1:on.n]


def _base(B=4):
    pb = conv_problem("base", B, depth=(0, 6), block=33)
    on = pb["net"]
    L0, U0, lbs, ubs, empty = oracle_lists(on, pb)
    keep = ~empty
    sel = lambda l: [None] + [x[keep] for x in l[1:]]
    return on, L0[keep], U0[keep], sel(lbs), sel(ubs)


def _states(on, l0, u0, lb, ub):
    """(lambda, primal) at the start of Algorithm 2 and after 7 outer iterations."""
    r0 = px.proximal_solver(on, l0, u0, lb, ub, 0)
    r7 = px.proximal_solver(on, l0, u0, lb, ub, 7)
    return [(r0.lam, r0.primal, 10.0), (r7.lam, r7.primal, px.eta_at(7, 20, px.ProxSettings()))]


def _moved(P, k, gam, zB, zA):
    Q = P.copy()
    g = np.asarray(gam)[:, None]
    if k >= 1:
        Q.xB[k] = g * zB + (1.0 - g) * Q.xB[k]
    Q.xA[k + 1] = g * zA + (1.0 - g) * Q.xA[k + 1]
    return Q


def check_steps(on, l0, u0, lb, ub, lam, P, eta):
    """Block by block, in the sweep order: gamma* against the segment's
    minimiser from values of L only, and L never increasing."""
    P = P.copy()
    for k in range(on.n):
        lp_k, lp_k1 = px.block_duals(on, P, lam, eta, k)
        zB, zA = px.conditional_gradient(on, k, lp_k, lp_k1, l0, u0, lb, ub)
        gam = px.optimal_step(on, k, P, lp_k, lp_k1, zB, zA, eta)
        L = lambda g: px.augmented_lagrangian(on, _moved(P, k, np.full(gam.shape, g), zB, zA), lam, eta)
        f0, fh, f1 = L(0.0), L(0.5), L(1.0)
        # parabola through (0, f0), (1/2, fh), (1, f1): f = a g^2 + b g + f0
        a = 2.0 * (f1 - 2.0 * fh + f0)
        b = f1 - f0 - a
        scale = 1.0 + np.abs(f0) + np.abs(f1) + np.abs(fh)
        flat = np.abs(a) <= 1e-12 * scale
        g_par = np.where(flat, np.where(b < 0, 1.0, 0.0), np.clip(-b / np.where(flat, 1.0, 2.0 * a), 0.0, 1.0))
        fg = L(gam)
        grid = np.linspace(0.0, 1.0, 401)
        vals = np.stack([L(g) for g in grid])
        assert np.all(fg <= vals.min(axis=0) + 1e-10 * scale), f"gamma* is not the segment's minimiser (block {k})"
        # where the parabola is strictly convex its minimiser is unique: gamma* equals it
        curved = a > 1e-8 * scale
        assert np.all(np.abs(gam - g_par)[curved] <= 1e-6), (k, np.max(np.abs(gam - g_par)[curved], initial=0))
        assert np.all(fg <= f0 + 1e-12 * scale), f"block {k} increased the Augmented Lagrangian"
        P = _moved(P, k, gam, zB, zA)
    return P


@pytest.mark.parametrize("case", ["tiny", "base"])
def test_optimal_step_is_the_segment_minimiser_and_never_ascends(case):
    cases = [_tiny(i) for i in range(6)] if case == "tiny" else [_base()]
    for on, l0, u0, lb, ub in cases:
        for lam, P, eta in _states(on, l0, u0, lb, ub):
            P1 = check_steps(on, l0, u0, lb, ub, lam, P, eta)
            check_steps(on, l0, u0, lb, ub, lam, P1, eta)   # a second sweep from the moved blocks


def test_conditional_gradient_is_the_inner_minimisation():
    on, l0, u0, lb, ub = _base()
    (lam, P, eta), _ = _states(on, l0, u0, lb, ub)
    lamp = [None] + [lam[k] + (P.xB[k] - P.xA[k]) / eta for k in range(1, on.n)]
    sol = oracle.inner_minimisation(on, l0, u0, lb, ub, lamp)
    for k in range(on.n):
        lp_k, lp_k1 = px.block_duals(on, P, lam, eta, k)
        zB, zA = px.conditional_gradient(on, k, lp_k, lp_k1, l0, u0, lb, ub)
        assert np.array_equal(zA, sol.xA[k + 1])
        if k >= 1:
            assert np.array_equal(zB, sol.xB[k])


@pytest.mark.parametrize("settings", ["incomplete", "bab"])
def test_iterates_stay_below_the_planet_lp_and_approach_it(settings):
    s = px.ProxSettings() if settings == "incomplete" else px.BAB_SETTINGS
    gaps = []
    for i in range(6):
        on, l0, u0, lb, ub = _tiny(i)
        p = lp.planet_lp(on, l0[0], u0[0], [None] + [x[0] for x in lb[1:]], [None] + [x[0] for x in ub[1:]])
        r = px.proximal_solver(on, l0, u0, lb, ub, 1000, s)
        tol = 1e-9 * max(1.0, abs(p.p_star))
        assert r.q_trace.max() <= p.p_star + tol and r.q_final[0] <= p.p_star + tol
        gaps.append((p.p_star - r.q_final[0]) / max(1.0, abs(p.p_star)))
    assert max(gaps) < 2e-3, gaps
    assert np.median(gaps) < 1e-4, gaps


def test_dual_update_and_momentum():
    on, l0, u0, lb, ub = _tiny(2)
    for mu in (0.0, 0.3):
        s = px.ProxSettings(eta0=20.0, eta_end=20.0, mu=mu, J=2)
        r1 = px.proximal_solver(on, l0, u0, lb, ub, 1, s)
        r2 = px.proximal_solver(on, l0, u0, lb, ub, 1, s, lam0=r1.lam, primal0=r1.primal, pi0=r1.pi, t0=1, T_sched=2)
        r0 = px.proximal_solver(on, l0, u0, lb, ub, 0, s)
        for k in range(1, on.n):
            step1 = (r1.primal.xB[k] - r1.primal.xA[k]) / 20.0
            np.testing.assert_allclose(r1.lam[k] - r0.lam[k], step1, rtol=0, atol=1e-14)
            step2 = (r2.primal.xB[k] - r2.primal.xA[k]) / 20.0
            np.testing.assert_allclose(r2.lam[k] - r1.lam[k], mu * step1 + step2, rtol=0, atol=1e-14)
    # a run split across calls equals the whole run
    s = px.ProxSettings()
    whole = px.proximal_solver(on, l0, u0, lb, ub, 10, s)
    a = px.proximal_solver(on, l0, u0, lb, ub, 4, s, T_sched=10)
    b = px.proximal_solver(on, l0, u0, lb, ub, 6, s, lam0=a.lam, primal0=a.primal, pi0=a.pi, t0=4, T_sched=10)
    assert np.array_equal(whole.q_final, b.q_final)


def _plant(monkeypatch, what):
    real_step = px.optimal_step
    if what == "step_sign":
        monkeypatch.setattr(px, "optimal_step", lambda *a: np.clip(1.0 - real_step(*a), 0.0, 1.0))
    elif what == "dropped_curvature":
        def step(net, k, P, lp_k, lp_k1, zB, zA, eta):
            # curvature of the x_hat_A block left out
            dA = zA - P.xA[k + 1]
            gA = np.ones_like(zA) if k + 1 == net.n else -lp_k1
            num = -np.sum(gA * dA, axis=1)
            den = np.zeros_like(num)
            if k >= 1:
                dB = zB - P.xB[k]
                num -= np.sum(lp_k * dB, axis=1)
                den += np.sum(dB * dB, axis=1) / eta
            safe = np.where(den > 0, den, 1.0)
            return np.where(den > 0, np.clip(num / safe, 0.0, 1.0), np.where(num > 0, 1.0, 0.0))
        monkeypatch.setattr(px, "optimal_step", step)
    elif what == "stale_dual":
        real_duals = px.block_duals

        def duals(net, P, lam, eta, k):
            # the x_hat_A part of the gradient left out: lambda'_{k+1} = lambda_{k+1}
            lp_k, lp_k1 = real_duals(net, P, lam, eta, k)
            if k + 1 < net.n:
                lp_k1 = lam[k + 1]
            return lp_k, lp_k1
        monkeypatch.setattr(px, "block_duals", duals)


@pytest.mark.parametrize("what", ["step_sign", "dropped_curvature", "stale_dual"])
def test_planted_mistakes_in_the_proximal_oracle_are_caught(monkeypatch, what):
    cases = [_tiny(i) for i in range(6)] + [_base()]
    states = [(c, st) for c in cases for st in _states(*c)]
    _plant(monkeypatch, what)
    failed = False
    for (on, l0, u0, lb, ub), (lam, P, eta) in states:
        try:
            check_steps(on, l0, u0, lb, ub, lam, P, eta)
        except AssertionError:
            failed = True
    assert failed, f"planted mistake '{what}' passed every pin"


def test_sensitivity_of_long_runs_to_a_tiny_perturbation():
    pb = conv_problem("deep", 12, depth=(0, 8), block=5)
    on = pb["net"]
    L0, U0, lbs, ubs, empty = oracle_lists(on, pb)
    keep = ~empty
    sel = lambda l: [None] + [x[keep] for x in l[1:]]
    lbs, ubs, L0, U0 = sel(lbs), sel(ubs), L0[keep], U0[keep]
    rc, _ = oracle.crown_init(on, lbs, ubs)
    rng = np.random.default_rng(0)
    rp = [None] + [x * (1 + 1e-7 * rng.standard_normal(x.shape)) for x in rc[1:]]
    a = px.proximal_solver(on, L0, U0, lbs, ubs, 50, lam0=rc)
    b = px.proximal_solver(on, L0, U0, lbs, ubs, 50, lam0=rp)
    first = np.abs(a.q_trace[0] - b.q_trace[0]) / np.maximum(np.abs(a.q_trace[0]), 1.0)
    final = np.abs(a.q_final - b.q_final) / np.maximum(np.abs(a.q_final), 1.0)
    assert first.max() < 1e-6          # the perturbation itself is tiny ...
    assert final.max() > 1e-3          # ... and the trajectory amplifies it
