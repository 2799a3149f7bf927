"""Pins of the oracle's tie reading (Eq. (min-pk) is silent on ties).

The oracle returns, per ReLU subproblem, a vertex of the Planet hull whose
value may exceed the subproblem's minimum by at most a stated margin: for an
ambiguous ReLU the vertex (u,u) is taken only if it beats the better of (l,0)
and (0,0) by more than 2^-16 (|rho| + |g|) max(|l|, u); for a passing ReLU
the lower end is taken only if rho - g exceeds 2^-16 (|rho| + |g|).  So the
returned point is an eps-minimiser of the Lagrangian of Eq. (nonprox_problem),
and the supergradient read off it must satisfy the eps-supergradient
inequality of a concave function

    q(rho') <= q(rho) + <s, rho' - rho> + eps    for every rho',

with eps = q_point - q(rho), the returned point's excess, which the reading
bounds by the sum of the margins.  The inequality is a property of the
Lagrangian (it is linear in rho and q is its minimum over the same feasible
set), checked here at random rho' near and far from rho, at the CROWN point
of Prop. 3 (where the ties are exact), after a few Adam steps and at random
rho, on the tiny MLPs and the Base convnet.  The direction of the reading
(which side a tie goes to) is pinned separately, and planted mistakes in the
oracle (the margin's sign flipped, a margin 2^10 times the reading, a sign
error in the supergradient, a dropped bias term in q) each make a pin fail.
"""
import numpy as np
import pytest

import oracle
from oracle import ld_oracle
from paper_2104_06718_gb300 import synth
from helpers import conv_problem, oracle_lists, tiny_problem

READING = 2.0 ** -16   # the margin of the reading, stated here independently of the oracle's constant


def _states(on, L0, U0, lbs, ubs, seed):
    """(name, rho) at the CROWN point, after 5 Adam steps from it, and at random rho."""
    rc, _ = oracle.crown_init(on, lbs, ubs)
    res = oracle.supergradient_adam(on, L0, U0, lbs, ubs, rc, 5)
    B = L0.shape[0]
    N = sum(lbs[k].shape[1] for k in range(1, on.n))
    rr = synth.random_duals([N], B, seed=seed, scale=0.05)[0].astype(np.float64)
    rnd = oracle.layer_lists(on, rr)
    return [("crown", rc), ("adam5", res.rho), ("random", rnd)]


def _excess_and_margin(on, lbs, ubs, rho, sol):
    """Per layer: the returned vertex's value minus the subproblem minimum,
    and the reading's margin, both [B, n_k]."""
    out = []
    for k in range(1, on.n):
        r, g, l, u = rho[k], sol.g[k], lbs[k], ubs[k]
        val = r * sol.xB[k] - g * sol.x[k]
        blk, pas = u <= 0, (l >= 0) & (u > 0)
        mn = np.where(blk, np.minimum(r * l, r * u),
                      np.where(pas, np.minimum((r - g) * l, (r - g) * u),
                               np.minimum(np.minimum(r * l, 0.0), (r - g) * u)))
        marg = np.where(blk, 0.0, np.where(pas, READING * (np.abs(r) + np.abs(g)) * (u - l),
                                            READING * (np.abs(r) + np.abs(g)) * np.maximum(np.abs(l), u)))
        out.append((val - mn, marg, val, mn))
    return out


def check_pins(on, L0, U0, lbs, ubs, rho, seed=0):
    sol = oracle.inner_minimisation(on, L0, U0, lbs, ubs, rho)
    sg = oracle.supergradient(sol)
    B = L0.shape[0]
    em = _excess_and_margin(on, lbs, ubs, rho, sol)
    mag = np.zeros(B)
    for k in range(1, on.n):
        mag += np.sum(np.abs(rho[k]) * np.maximum(np.abs(lbs[k]), np.abs(ubs[k])), axis=1)
    tol = 1e-11 * (1.0 + np.abs(sol.q) + mag)
    eps = sol.q_point - sol.q
    eps_reading = sum(np.sum(m, axis=1) for _, m, _, _ in em)
    # per unit: an eps-minimiser within the reading's margin
    for ex, m, _, _ in em:
        assert np.all(ex >= -1e-12 * (1 + np.abs(m) / READING)), "returned vertex below the exact minimum"
        assert np.all(ex <= m + 1e-12 * (1 + m / READING)), "returned vertex beyond the reading's margin"
    # the point's excess is what the per-unit excesses add up to, and within the summed margins
    assert np.all(eps >= -tol) and np.all(eps <= eps_reading + tol), (eps, eps_reading)
    # direction: a tie (or a near-tie within the margin) never goes to (u,u) / the lower end
    for k in range(1, on.n):
        r, g, l, u = rho[k], sol.g[k], lbs[k], ubs[k]
        code = sol.vertex[k]
        amb = (l < 0) & (u > 0)
        pas = (l >= 0) & (u > 0)
        vuu = (r - g) * u
        best = np.minimum(r * l, 0.0)
        assert np.all(vuu[amb & (code == 2)] < best[amb & (code == 2)]), "(u,u) taken without winning"
        assert np.all((r - g)[pas & (code == 0)] > 0), "passing lower end taken at a tie"
    # the eps-supergradient inequality at random rho' around rho
    rng = np.random.default_rng(1000 + seed)
    for delta in (1e-6, 1e-3, 1e-1, 1.0):
        rp = [None]
        for k in range(1, on.n):
            sc = np.abs(rho[k]) + np.mean(np.abs(rho[k])) + 1e-3
            rp.append(rho[k] + delta * sc * rng.standard_normal(rho[k].shape))
        qp = oracle.dual_value(on, L0, U0, lbs, ubs, rp)
        lin = sum(np.sum(sg[k] * (rp[k] - rho[k]), axis=1) for k in range(1, on.n))
        mag_p = mag + sum(np.sum(np.abs(rp[k]) * np.maximum(np.abs(lbs[k]), np.abs(ubs[k])), axis=1)
                          for k in range(1, on.n))
        slack = 1e-11 * (1.0 + np.abs(qp) + np.abs(sol.q) + np.abs(lin) + mag_p)
        assert np.all(qp <= sol.q + lin + eps + slack), (delta, np.max(qp - sol.q - lin - eps))
    return sol


def _tiny_cases():
    out = []
    for i in range(6):
        specs, on, l0, u0, lb, ub = tiny_problem(i)
        out.append((on, l0, u0, [None] + lb[1:on.n], [None] + ub[1:on.n]))
    return out


def _base_case():
    pb = conv_problem("base", 8, depth=(0, 8), block=12)
    on = pb["net"]
    L0, U0, lbs, ubs, empty = oracle_lists(on, pb)
    keep = ~empty
    sel = lambda l: [None] + [x[keep] for x in l[1:]]
    return on, L0[keep], U0[keep], sel(lbs), sel(ubs)


@pytest.mark.parametrize("case", ["tiny", "base"])
def test_supergradient_is_an_eps_supergradient_within_the_reading(case):
    cases = _tiny_cases() if case == "tiny" else [_base_case()]
    n_ties = 0
    for i, (on, L0, U0, lbs, ubs) in enumerate(cases):
        for name, rho in _states(on, L0, U0, lbs, ubs, seed=40 + i):
            sol = check_pins(on, L0, U0, lbs, ubs, rho, seed=i)
            if name == "crown":
                # Prop. 3 makes (l,0) and (u,u) tie exactly for ambiguous ReLUs with lambda > 0
                for k in range(1, on.n):
                    amb = (lbs[k] < 0) & (ubs[k] > 0)
                    vuu = (rho[k] - sol.g[k]) * ubs[k]
                    n_ties += int(np.sum(amb & (np.abs(vuu - rho[k] * lbs[k]) <= 1e-12 * (1 + np.abs(vuu)))
                                         & (rho[k] * lbs[k] < 0)))
    assert n_ties > 0, "the CROWN point should hold exact ties"


def _planted(monkeypatch, what):
    if what == "margin_sign":
        monkeypatch.setattr(ld_oracle, "TIE_REL", -ld_oracle.TIE_REL)
    elif what == "margin_too_wide":
        monkeypatch.setattr(ld_oracle, "TIE_REL", ld_oracle.TIE_REL * 2.0 ** 10)
    elif what == "supergradient_sign":
        monkeypatch.setattr(ld_oracle, "supergradient",
                            lambda sol: [None] + [sol.xA[k] - sol.xB[k] for k in range(1, len(sol.xB))])
        monkeypatch.setattr(oracle, "supergradient", ld_oracle.supergradient)
    elif what == "dropped_bias":
        real = ld_oracle.inner_minimisation

        def inner(net, l0, u0, lb, ub, rho, passes=None):
            sol = real(net, l0, u0, lb, ub, rho, passes)
            sol.q = sol.q - net.L(net.n).bias_vector()[0]
            return sol
        monkeypatch.setattr(ld_oracle, "inner_minimisation", inner)
        monkeypatch.setattr(oracle, "inner_minimisation", inner)


@pytest.mark.parametrize("what", ["margin_sign", "margin_too_wide", "supergradient_sign", "dropped_bias"])
def test_planted_mistakes_in_the_tie_reading_are_caught(monkeypatch, what):
    on, L0, U0, lbs, ubs = _base_case()
    states = _states(on, L0, U0, lbs, ubs, seed=7)
    _planted(monkeypatch, what)
    failed = False
    for _, rho in states:
        try:
            check_pins(on, L0, U0, lbs, ubs, rho, seed=3)
        except AssertionError:
            failed = True
    assert failed, f"planted mistake '{what}' passed every pin"
