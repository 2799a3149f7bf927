"""Branching scores, upper bounds and a minimal branch and bound (Sec. 4,
Sec. 5.1.3, Sec. 5.2).

TEST INFRASTRUCTURE, NOT PRODUCT CODE: imported only by the test suite (the
same rule as the rest of this package).  Plain FP64.

What it computes.
* SR scores of BaBSR and the FSB/mSR scores, Eq. (babsr-scores) and Eq.
  (fsb-scores): one backward pass of the WK upper-relaxation slopes
      lam_{n-1} = -W_n^T 1,  lam_{k-1} = W_k^T ([u_k]_+ / ([u_k]_+ - [l_k]_-) * lam_k)
  then, for the ambiguous ReLUs of layer k (others score 0),
      s_SR  = | max(0, lam_k b_k) - u/(u-l) lam_k b_k + u l/(u-l) [lam_k]_+ |
      s_FSB = | min(0, lam_k b_k) - u/(u-l) lam_k b_k + u l/(u-l) [lam_k]_+ |
      t_SR  = -u l/(u-l) [lam_k]_+
  with b_k the bias of layer k at each neuron.
* SR's decision: the ReLU with the largest s_SR, or, when that score does
  not exceed the threshold, the largest t_SR; mSR: the same with s_FSB.
* FSB's decision, Eq. (fsb-prefilter): per layer the argmax of s_FSB and of
  t_SR form the candidates; each candidate's two children (split passing /
  blocking) are bounded by the better of the CROWN and WK bounds of the
  output (A_FSB) with the parent's intermediate bounds clamped by the split;
  FSB takes the candidate whose worse child bound is the largest.
* Upper bound (Sec. 5.1.3): the network's output at the inner minimiser's
  input point x0* of the last dual evaluated.
* A minimal batched branch and bound (Sec. 2.3, Sec. 5.2): the B subdomains
  with the lowest lower bounds are branched together, their 2B children
  bounded with the LD supergradient method (warm-started from the parent's
  duals), subdomains whose lower bound exceeds 0 are discarded, and the
  search stops when none is left (the property holds), when an upper bound
  falls below 0 (a counterexample), or after a node budget.
Readings (listed in the design notes): subdomains hold their intermediate
bounds fixed at the root's, clamped by the split (BaDNB, Sec. 5.1.1); every
argmax runs over the ambiguous ReLUs only and takes the first index on ties;
the SR threshold defaults to 0; splits already made are no longer ambiguous.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .intermediate import substitute
from .ld_oracle import Net, apply_masks, classify, inner_minimisation, ld_bound, layer_lists, split_offsets


def wk_backward(net: Net, lb, ub):
    """lam_k of Eq. (babsr-scores), k = 1..n-1 (lists indexed 1..n-1, [B, n_k])."""
    n = net.n
    B = lb[1].shape[0]
    lam = [None] * n
    cur = net.L(n).transposed(-np.ones((B, 1)))
    for k in range(n - 1, 0, -1):
        lam[k] = cur
        if k >= 2:
            up = np.maximum(ub[k], 0.0)
            lo = np.minimum(lb[k], 0.0)
            den = up - lo
            slope = np.where(den > 0, up / np.where(den > 0, den, 1.0), 0.0)
            cur = net.L(k).transposed(slope * cur)
    return lam


def branching_scores(net: Net, lb, ub):
    """(s_SR, s_FSB, t_SR), lists indexed 1..n-1 of [B, n_k], for clamped bounds lb, ub."""
    lam = wk_backward(net, lb, ub)
    s_sr, s_fsb, t_sr = [None], [None], [None]
    for k in range(1, net.n):
        l, u = lb[k], ub[k]
        amb = classify(l, u) == 2
        den = np.where(amb, u - l, 1.0)
        bk = net.L(k).bias_vector()[None, :]
        lb_k = lam[k] * bk
        common = -(u / den) * lam[k] * bk + (u * l / den) * np.maximum(lam[k], 0.0)
        s_sr.append(np.where(amb, np.abs(np.maximum(0.0, lb_k) + common), 0.0))
        s_fsb.append(np.where(amb, np.abs(np.minimum(0.0, lb_k) + common), 0.0))
        t_sr.append(np.where(amb, -(u * l / den) * np.maximum(lam[k], 0.0), 0.0))
    return s_sr, s_fsb, t_sr


def _flat(net, lst):
    return np.concatenate([lst[k] for k in range(1, net.n)], axis=1)


def sr_decision(net: Net, lb, ub, fsb_scores: bool = False, threshold: float = 0.0):
    """Flat ReLU index chosen by SR (mSR with fsb_scores) per subdomain [B];
    -1 where no ReLU is ambiguous."""
    s_sr, s_fsb, t_sr = branching_scores(net, lb, ub)
    amb = _flat(net, [None] + [classify(lb[k], ub[k]) == 2 for k in range(1, net.n)])
    s = np.where(amb, _flat(net, s_fsb if fsb_scores else s_sr), -np.inf)
    t = np.where(amb, _flat(net, t_sr), -np.inf)
    i_s = np.argmax(s, axis=1)
    i_t = np.argmax(t, axis=1)
    rows = np.arange(s.shape[0])
    pick = np.where(s[rows, i_s] > threshold, i_s, i_t)
    return np.where(amb.any(axis=1), pick, -1)


def fsb_candidates(net: Net, lb, ub):
    """Candidate flat indices [B, 2(n-1)] of Eq. (fsb-prefilter): per layer the
    argmax of s_FSB and of t_SR (-1 where the layer has no ambiguous ReLU)."""
    _, s_fsb, t_sr = branching_scores(net, lb, ub)
    offs = split_offsets(net)
    cols = []
    for k in range(1, net.n):
        amb_k = classify(lb[k], ub[k]) == 2
        amb = amb_k.any(axis=1)
        for sc in (s_fsb[k], t_sr[k]):
            cols.append(np.where(amb, offs[k - 1] + np.argmax(np.where(amb_k, sc, -np.inf), axis=1), -1))
    return np.stack(cols, axis=1)


def output_bound_best(net: Net, l0, u0, lb, ub):
    """A_FSB: the better of the CROWN and WK lower bounds of x_hat_n [B]."""
    c = np.ones((l0.shape[0], 1, 1))
    return np.maximum(substitute(net, net.n, c, l0, u0, lb, ub, "crown")[:, 0],
                      substitute(net, net.n, c, l0, u0, lb, ub, "wk")[:, 0])


def split_bounds(net: Net, lb, ub, flat_index, phase):
    """Bounds of the children: lists lb, ub with ReLU flat_index[b] clamped to
    phase[b] (+1 passing: l <- max(l, 0); -1 blocking: u <- min(u, 0))."""
    offs = split_offsets(net)
    lb2 = [None] + [x.copy() for x in lb[1:]]
    ub2 = [None] + [x.copy() for x in ub[1:]]
    for b, (j, ph) in enumerate(zip(flat_index, phase)):
        if j < 0:
            continue
        k = int(np.searchsorted(offs, j, side="right"))
        i = j - offs[k - 1]
        if ph > 0:
            lb2[k][b, i] = max(lb2[k][b, i], 0.0)
        else:
            ub2[k][b, i] = min(ub2[k][b, i], 0.0)
    return lb2, ub2


def fsb_decision(net: Net, l0, u0, lb, ub):
    """Flat ReLU index chosen by FSB per subdomain [B] (-1: none ambiguous),
    and the candidates' child bounds [B, C, 2]."""
    cand = fsb_candidates(net, lb, ub)
    B, C = cand.shape
    child = np.full((B, C, 2), -np.inf)
    for c in range(C):
        for h, ph in enumerate((+1, -1)):
            l2, u2 = split_bounds(net, lb, ub, cand[:, c], np.full(B, ph))
            val = output_bound_best(net, l0, u0, l2, u2)
            child[:, c, h] = np.where(cand[:, c] >= 0, val, -np.inf)
    worst = child.min(axis=2)
    pick = cand[np.arange(B), np.argmax(worst, axis=1)]
    return np.where((cand >= 0).any(axis=1), pick, -1), child


def upper_bound_at_x0(net: Net, l0, u0, lb, ub, rho):
    """Network output at the inner minimiser's input x0* of q(rho) (Sec. 5.1.3), [B]."""
    sol = inner_minimisation(net, l0, u0, lb, ub, rho)
    return net.evaluate(sol.x[0])


@dataclass
class BaBResult:
    status: str            # "verified", "counterexample" or "budget"
    lower: float           # global lower bound when stopped
    upper: float           # best upper bound found
    nodes: int             # subdomains bounded
    iterations: int
    trace: list = field(default_factory=list)


def bab(net: Net, l0, u0, lbk, ubk, T: int = 50, batch: int = 8, max_nodes: int = 2000, branching: str = "fsb"):
    """Minimal batched branch and bound of Sec. 2.3 / Sec. 5.2 for one
    property (l0, u0 [1, n_0]; lbk, ubk root intermediate bounds [1, N]):
    decides whether min x_hat_n over the box is positive."""
    N = lbk.shape[1]
    masks = np.zeros((1, N), np.int8)
    out, res, keep = ld_bound(net, l0, u0, lbk, ubk, None, masks, T)
    rho = np.zeros((1, N))
    if res is not None:
        rho[keep] = np.concatenate([res.rho[k] for k in range(1, net.n)], axis=1)
    lbs, ubs, _ = apply_masks(net, layer_lists(net, lbk.copy()), layer_lists(net, ubk.copy()), masks)
    best_ub = float(upper_bound_at_x0(net, l0, u0, lbs, ubs, layer_lists(net, rho))[0])
    dom = [(float(out[0]), masks[0], rho[0])]
    stuck = []        # subdomains with no ambiguous ReLU left and a bound <= 0: undecided
    nodes, it, trace = 1, 0, []
    while True:
        dom = [d for d in dom if d[0] <= 0.0]
        lowest = min([d[0] for d in dom + stuck], default=np.inf)
        if best_ub < 0.0:
            return BaBResult("counterexample", lowest, best_ub, nodes, it, trace)
        if not dom:
            return BaBResult("budget" if stuck else "verified", lowest if stuck else 0.0, best_ub, nodes, it, trace)
        if nodes >= max_nodes:
            return BaBResult("budget", lowest, best_ub, nodes, it, trace)
        dom.sort(key=lambda d: d[0])
        pick, dom = dom[:batch], dom[batch:]
        P = len(pick)
        m = np.stack([d[1] for d in pick])
        r = np.stack([d[2] for d in pick])
        L0 = np.repeat(l0, P, axis=0)
        U0 = np.repeat(u0, P, axis=0)
        lb, ub, _ = apply_masks(net, layer_lists(net, np.repeat(lbk, P, axis=0)),
                                layer_lists(net, np.repeat(ubk, P, axis=0)), m)
        if branching == "fsb":
            j, _ = fsb_decision(net, L0, U0, lb, ub)
        else:
            j = sr_decision(net, lb, ub, fsb_scores=branching == "msr")
        cm, cr = [], []
        for b in range(P):
            if j[b] < 0:
                stuck.append(pick[b])         # nothing ambiguous left to split
                continue
            for ph in (1, -1):
                mm = m[b].copy()
                mm[j[b]] = ph
                cm.append(mm)
                cr.append(r[b])
        if not cm:
            continue
        cm = np.stack(cm)
        cr = np.stack(cr)
        o, res, keep = ld_bound(net, l0, u0, lbk, ubk, None, cm, T, rho_in=cr)
        nodes += len(cm)
        it += 1
        if res is not None:
            rk = np.concatenate([res.rho[k] for k in range(1, net.n)], axis=1)
            cr[keep] = rk
            lb2, ub2, _ = apply_masks(net, layer_lists(net, np.repeat(lbk, len(cm), axis=0)[keep]),
                                      layer_lists(net, np.repeat(ubk, len(cm), axis=0)[keep]), cm[keep])
            ubv = upper_bound_at_x0(net, np.repeat(l0, len(keep), axis=0), np.repeat(u0, len(keep), axis=0),
                                    lb2, ub2, res.rho)
            best_ub = min(best_ub, float(ubv.min()))
        for c in range(len(cm)):
            if np.isfinite(o[c]):
                dom.append((float(o[c]), cm[c], cr[c]))
        trace.append(min([d[0] for d in dom], default=np.inf))


__all__ = ["wk_backward", "branching_scores", "sr_decision", "fsb_candidates", "output_bound_best", "split_bounds",
           "fsb_decision", "upper_bound_at_x0", "BaBResult", "bab"]
