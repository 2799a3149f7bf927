"""Pins of the branching, upper-bound and branch-and-bound oracle (Sec. 4,
Sec. 5.1.3, Sec. 5.2) against things other than itself:
  * the scores' backward pass is the WK propagation dual: the output bound
    built from it equals the independently written WK substitution;
  * hand-worked scores of a two-ReLU net (tests/golden/branching_scores_2x2.txt);
  * FSB's child bounds never exceed the exact minimum of the child (MILP
    with the split's bounds), and the upper bound from x0* is a network value
    in the box, at or above the exact minimum;
  * branch and bound decides the sign of the exact minimum on tiny MLPs whose
    output is shifted so that the minimum sits 0.02 above or below zero, with
    lower <= exact minimum <= upper, and FSB needs fewer subdomains than SR.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import branching as br
from oracle import intermediate as ib
from oracle import lp
from helpers import tiny_problem

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden(name):
    vals = {}
    for line in open(os.path.join(HERE, "golden", name)):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split("=")
            vals[k.strip()] = np.array([float(x) for x in v.split()])
    return vals


def _tiny(i):
    specs, on, l0, u0, lb, ub = tiny_problem(i)
    return on, l0, u0, [None] + lb[1:on.n], [None] + ub[1:on.n]


def test_backward_pass_is_the_wk_dual():
    for i in range(6):
        on, l0, u0, lb, ub = _tiny(i)
        lam = br.wk_backward(on, lb, ub)
        n = on.n
        val = on.L(n).bias_vector()[0] + np.zeros(l0.shape[0])
        for j in range(1, n):
            a = -lam[j]
            up, lo = np.maximum(ub[j], 0.0), np.minimum(lb[j], 0.0)
            den = np.where(up - lo > 0, up - lo, 1.0)
            slope = np.where(up - lo > 0, up / den, 0.0)
            amb = (lb[j] < 0) & (ub[j] > 0)
            b_bar = np.where(amb, -lb[j] * ub[j] / np.where(amb, ub[j] - lb[j], 1.0), 0.0)
            val += np.sum(np.minimum(a, 0.0) * b_bar, axis=1) + (slope * a) @ on.L(j).bias_vector()
        a0 = -on.L(1).transposed(np.where(np.maximum(ub[1], 0) - np.minimum(lb[1], 0) > 0,
                                          np.maximum(ub[1], 0) / np.where(np.maximum(ub[1], 0) - np.minimum(lb[1], 0) > 0,
                                                                          np.maximum(ub[1], 0) - np.minimum(lb[1], 0), 1.0),
                                          0.0) * lam[1])
        val += np.sum(np.minimum(a0 * l0, a0 * u0), axis=1)
        wk = ib.substitute(on, n, np.ones((l0.shape[0], 1, 1)), l0, u0, lb, ub, "wk")[:, 0]
        np.testing.assert_allclose(val, wk, rtol=1e-12, atol=1e-12)


def test_scores_of_the_hand_worked_net():
    g = _golden("branching_scores_2x2.txt")
    net = oracle.Net([oracle.Layer("fc", np.array([[1.0, 1.0], [1.0, -1.0]]), np.array([0.5, -0.25])),
                      oracle.Layer("fc", np.array([[1.0, -2.0]]), np.array([0.0]))])
    l0, u0 = -np.ones((1, 2)), np.ones((1, 2))
    lb, ub = oracle.ibp_bounds(net, l0, u0)
    np.testing.assert_allclose(lb[1][0], [-1.5, -2.25])
    np.testing.assert_allclose(ub[1][0], [2.5, 1.75])
    lam = br.wk_backward(net, lb, ub)
    np.testing.assert_allclose(lam[1][0], g["lam"])
    s_sr, s_fsb, t_sr = br.branching_scores(net, lb, ub)
    np.testing.assert_allclose(s_sr[1][0], g["s_sr"])
    np.testing.assert_allclose(s_fsb[1][0], g["s_fsb"])
    np.testing.assert_allclose(t_sr[1][0], g["t_sr"])
    assert br.sr_decision(net, lb, ub)[0] == int(g["sr_choice"][0])
    assert list(br.fsb_candidates(net, lb, ub)[0]) == [int(x) for x in g["fsb_candidates"]]


def test_fsb_child_bounds_and_upper_bound_are_sound():
    for i in range(6):
        on, l0, u0, lb, ub = _tiny(i)
        pick, child = br.fsb_decision(on, l0, u0, lb, ub)
        cand = br.fsb_candidates(on, lb, ub)
        for c in range(cand.shape[1]):
            j = cand[0, c]
            if j < 0:
                continue
            for h, ph in enumerate((1, -1)):
                l2, u2 = br.split_bounds(on, lb, ub, [j], [ph])
                if np.any(np.concatenate([l2[k] > u2[k] for k in range(1, on.n)], axis=1)):
                    continue
                try:
                    ex = lp.exact_min_milp(on, l0[0], u0[0], [None] + [x[0] for x in l2[1:]],
                                           [None] + [x[0] for x in u2[1:]])
                except RuntimeError as e:      # the split's phase is not reachable: an empty child
                    assert "infeasible" in str(e).lower()
                    continue
                assert child[0, c, h] <= ex + 1e-9 * max(1.0, abs(ex))
        assert pick[0] in cand[0]
        rho, _ = oracle.crown_init(on, lb, ub)
        ubv = br.upper_bound_at_x0(on, l0, u0, lb, ub, rho)
        sol = oracle.inner_minimisation(on, l0, u0, lb, ub, rho)
        assert np.all((sol.x[0] >= l0) & (sol.x[0] <= u0))
        ex = lp.exact_min_milp(on, l0[0], u0[0], [None] + [x[0] for x in lb[1:]], [None] + [x[0] for x in ub[1:]])
        assert ubv[0] >= ex - 1e-9 * max(1.0, abs(ex))
        np.testing.assert_allclose(ubv, on.evaluate(sol.x[0]))


def shifted_tiny(i, delta):
    """Tiny MLP i with its output bias moved so that the exact minimum is delta."""
    specs, on, l0, u0, lb, ub = tiny_problem(i)
    ex = lp.exact_min_milp(on, l0[0], u0[0], [None] + [x[0] for x in lb[1:on.n]], [None] + [x[0] for x in ub[1:on.n]])
    last = on.layers[-1]
    net = oracle.Net(on.layers[:-1] + [oracle.Layer("fc", last.W, last.b - ex + delta)])
    lb2, ub2 = oracle.ibp_bounds(net, l0, u0)
    flat = lambda x: np.concatenate([x[k] for k in range(1, net.n)], axis=1)
    return net, l0, u0, flat(lb2), flat(ub2)


@pytest.mark.parametrize("delta", [0.02, -0.02])
def test_branch_and_bound_decides_the_sign_of_the_minimum(delta):
    nodes = {"fsb": 0, "sr": 0}
    for i in range(6):
        net, l0, u0, lbk, ubk = shifted_tiny(i, delta)
        for rule in ("fsb", "sr", "msr"):
            r = br.bab(net, l0, u0, lbk, ubk, T=50, batch=4, max_nodes=400, branching=rule)
            assert r.status == ("verified" if delta > 0 else "counterexample"), (i, rule, r)
            assert r.upper >= delta - 1e-9
            if delta < 0:
                assert r.upper < 0.0
            if rule in nodes:
                nodes[rule] += r.nodes
    if delta > 0:
        assert nodes["fsb"] < nodes["sr"], nodes
