"""Pins of the DSG+ / Dec-DSG+ oracle (Sec. 2.2.2, Eq. (dj_prob-main),
Theorem 1, Prop. 3) against things other than itself:
  * d_O is the minimum of its Lagrangian: no sampled feasible point goes
    below it (brute force on the tiny MLPs), and the returned point attains
    it up to the tie margins of its x_hat choice;
  * Theorem 1: q(mu) >= d_O(mu, lambda) at random dual points, with equality
    at lambda_{k-1} = W_k^T mu_k, lambda_{n-1} = -W_n^T 1 (two independently
    written duals agree);
  * Prop. 3: at the CROWN start d_O equals the propagation bound of Eq.
    (bounds-propagation);
  * weak duality: every DSG+ iterate and random dual point stays below the
    Planet LP optimum and the exact (MILP) minimum.
"""
import numpy as np
import pytest

import oracle
from oracle import dsg, lp
from helpers import conv_problem, oracle_lists, tiny_problem


def _tiny(i):
    specs, on, l0, u0, lb, ub = tiny_problem(i)
    return on, l0, u0, [None] + lb[1:on.n], [None] + ub[1:on.n]


def _random_duals(on, B, seed):
    rng = np.random.default_rng(seed)
    mu = [None] + [rng.normal(scale=0.5, size=(B, on.L(k).n_out)) for k in range(1, on.n)]
    lam = [None] + [rng.normal(scale=0.5, size=(B, on.L(k).n_out)) for k in range(1, on.n)]
    return mu, lam


def lagrangian(on, mu, lam, x, xh):
    """The objective of Eq. (dj_prob-main) at a point (x_0..x_{n-1}, x_hat_1..x_hat_{n-1})."""
    n = on.n
    val = on.L(n).forward(x[n - 1])[:, 0]
    for k in range(1, n):
        val += np.sum(mu[k] * (xh[k] - on.L(k).forward(x[k - 1])), axis=1)
        val += np.sum(lam[k] * (x[k] - np.maximum(xh[k], 0.0)), axis=1)
    return val


def test_dsg_value_is_the_minimum_of_its_lagrangian():
    rng = np.random.default_rng(5)
    for i in range(6):
        on, l0, u0, lb, ub = _tiny(i)
        mu, lam = _random_duals(on, 1, 100 + i)
        inn = dsg.dsg_inner(on, l0, u0, lb, ub, mu, lam)
        at = lagrangian(on, mu, lam, inn.x, inn.xh)
        # the returned point attains d_O up to the tie margins of its x_hat choice
        marg = sum(np.sum(2.0 ** -16 * (np.abs(mu[k]) + np.abs(lam[k])) * np.maximum(np.abs(lb[k]), np.abs(ub[k])),
                          axis=1) for k in range(1, on.n))
        assert np.all(at >= inn.d - 1e-12) and np.all(at <= inn.d + marg + 1e-12)
        for _ in range(200):
            x = [l0 + (u0 - l0) * rng.random(l0.shape)]
            xh = [None]
            for k in range(1, on.n):
                x.append(np.maximum(lb[k], 0) + (np.maximum(ub[k], 0) - np.maximum(lb[k], 0)) * rng.random(lb[k].shape))
                xh.append(lb[k] + (ub[k] - lb[k]) * rng.random(lb[k].shape))
            assert lagrangian(on, mu, lam, x, xh)[0] >= inn.d[0] - 1e-12


@pytest.mark.parametrize("case", ["tiny", "base"])
def test_theorem_1(case):
    if case == "tiny":
        cases = [_tiny(i) for i in range(6)]
    else:
        pb = conv_problem("base", 4, depth=(0, 6), block=51)
        on = pb["net"]
        L0, U0, lbs, ubs, empty = oracle_lists(on, pb)
        keep = ~empty
        sel = lambda l: [None] + [x[keep] for x in l[1:]]
        cases = [(on, L0[keep], U0[keep], sel(lbs), sel(ubs))]
    for j, (on, l0, u0, lb, ub) in enumerate(cases):
        B = l0.shape[0]
        mu, lam = _random_duals(on, B, 200 + j)
        q = oracle.dual_value(on, l0, u0, lb, ub, mu)
        d = dsg.dsg_value(on, l0, u0, lb, ub, mu, lam)
        assert np.all(q >= d - 1e-10 * (1 + np.abs(q)))
        # lambda' of Theorem 1 makes the two duals equal
        lamp = [None] * on.n
        for k in range(1, on.n):
            nxt = -np.ones((B, 1)) if k + 1 == on.n else mu[k + 1]
            lamp[k] = on.L(k + 1).transposed(nxt)
        dp = dsg.dsg_value(on, l0, u0, lb, ub, mu, lamp)
        np.testing.assert_allclose(dp, q, rtol=1e-10, atol=1e-10)


def test_crown_start_is_the_propagation_bound():
    for i in range(6):
        on, l0, u0, lb, ub = _tiny(i)
        mu, lam = dsg.dsg_init(on, lb, ub)
        d = dsg.dsg_value(on, l0, u0, lb, ub, mu, lam)
        prop = oracle.propagation_bound(on, l0, u0, lb, ub, mu, lam)
        np.testing.assert_allclose(d, prop, rtol=1e-10, atol=1e-10)


def test_dsg_iterates_stay_below_the_lp_and_exact_minimum():
    for i in range(6):
        on, l0, u0, lb, ub = _tiny(i)
        lb1 = [None] + [x[0] for x in lb[1:]]
        ub1 = [None] + [x[0] for x in ub[1:]]
        p = lp.planet_lp(on, l0[0], u0[0], lb1, ub1).p_star
        ex = lp.exact_min_milp(on, l0[0], u0[0], lb1, ub1)
        r = dsg.dsg_plus(on, l0, u0, lb, ub, 200)
        tol = 1e-9 * max(1.0, abs(p))
        assert r.d_trace.max() <= p + tol and r.d_final[0] <= p + tol and r.q_final[0] <= p + tol
        assert p <= ex + tol
        assert r.q_final[0] >= r.d_final[0] - 1e-10   # Theorem 1 at the final iterate
        mu, lam = _random_duals(on, 1, 300 + i)
        assert dsg.dsg_value(on, l0, u0, lb, ub, mu, lam)[0] <= p + tol
