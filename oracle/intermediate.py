"""Propagation-based intermediate bounds (CROWN, WK and their layer-wise best).

TEST INFRASTRUCTURE, NOT PRODUCT CODE: imported only by the test suite (the
same rule as the rest of this package).  Plain FP64, one objective row per
neuron, no blocking or fusion beyond what the definitions below state.

What it computes.  Intermediate bounds l_hat_k, u_hat_k on x_hat_k are the
bounds of versions of Eq. (noncvx_pb) whose objective is one neuron
x_hat_k[i] instead of x_hat_n, for k = 1..n-1 and every i (Sec. 2.2.3).  The
experiments take, for each layer, the layer-wise best of the bounds returned
by CROWN and by WK (Sec. 7.2; BaDNB, Sec. 5.1.1), layer by layer, each layer
bounded with the best bounds of the layers before it.

Both are propagation methods (Sec. 2.2.1): each ReLU is replaced by a linear
lower relaxation sigma_low(x_hat) = a_low * x_hat and the upper relaxation
sigma_up(x_hat) = a_bar * x_hat + b_bar of Eq. (slopes-biases) (a_bar = u/(u-l),
b_bar = -l*u/(u-l) for ambiguous ReLUs; passing 1 / 0; blocking 0 / 0), and
the objective row is substituted backwards through the layers.  They differ
only in the lower slope of an ambiguous ReLU:
  CROWN: a_low = 1 if u >= -l else 0 (footnote of Sec. 4.2)
  WK:    a_low = [u]_+ / ([u]_+ - [l]_-) = a_bar (the WK relaxation quoted in
         Sec. 4.1 for Smart Branching).

Backward substitution for a lower bound of c^T x_hat_k (an upper bound is
minus the lower bound of -c^T x_hat_k):
  a_{k-1} = W_k^T c, const = c^T b_k
  for j = k-1 .. 1 (coefficients a on x_j = relu(x_hat_j)):
    mu_j   = a_low * [a_j]_+ + a_bar * [a_j]_-     (coefficients on x_hat_j)
    const += [a_j]_-^T b_bar_j + mu_j^T b_j
    a_{j-1} = W_j^T mu_j
  bound = const + sum_i min(a_0[i] l0[i], a_0[i] u0[i])
For k = 1 this is the exact range of an affine map over the box.
"""
from __future__ import annotations

import numpy as np

from .ld_oracle import Net, classify, split_offsets

RULES = ("crown", "wk")


def relaxation(l, u, rule: str):
    """(a_low, a_bar, b_bar) of the ReLU relaxation for bounds (l, u)."""
    if rule not in RULES:
        raise ValueError(rule)
    cls = classify(l, u)
    amb = cls == 2
    den = np.where(amb, u - l, 1.0)
    a_bar = np.where(amb, u / den, np.where(cls == 1, 1.0, 0.0))
    b_bar = np.where(amb, -l * u / den, 0.0)
    if rule == "crown":
        a_low = np.where(amb, (u >= -l).astype(np.float64), np.where(cls == 1, 1.0, 0.0))
    else:
        a_low = a_bar.copy()
    return a_low, a_bar, b_bar


def substitute(net: Net, k: int, c, l0, u0, lb, ub, rule: str):
    """Lower bound of c^T x_hat_k over the box, propagated with `rule`.

    c: [P, R, n_k] objective rows per property; l0, u0: [P, n_0];
    lb, ub: lists indexed 1..k-1 of [P, n_j] bounds of the earlier layers.
    Returns [P, R].
    """
    P, R, _ = c.shape
    rows = c.reshape(P * R, -1)
    a = net.L(k).transposed(rows)                          # W_k^T c
    const = rows @ net.L(k).bias_vector()
    for j in range(k - 1, 0, -1):
        a_low, a_bar, b_bar = (np.repeat(x, R, axis=0) for x in relaxation(lb[j], ub[j], rule))
        pos, neg = np.maximum(a, 0.0), np.minimum(a, 0.0)
        mu = a_low * pos + a_bar * neg
        const = const + np.sum(neg * b_bar, axis=1) + mu @ net.L(j).bias_vector()
        a = net.L(j).transposed(mu)                        # W_j^T mu_j
    L0 = np.repeat(np.asarray(l0, np.float64), R, axis=0)
    U0 = np.repeat(np.asarray(u0, np.float64), R, axis=0)
    val = const + np.sum(np.minimum(a * L0, a * U0), axis=1)
    return val.reshape(P, R)


def layer_bounds(net: Net, k: int, l0, u0, lb, ub, rule: str):
    """Lower and upper bounds of every neuron of layer k with one rule."""
    P = np.asarray(l0).shape[0]
    nk = net.L(k).n_out
    eye = np.broadcast_to(np.eye(nk), (P, nk, nk))
    low = substitute(net, k, eye, l0, u0, lb, ub, rule)
    up = -substitute(net, k, -eye, l0, u0, lb, ub, rule)
    return low, up


def crown_wk_bounds(net: Net, l0, u0, rules=RULES, include_output: bool = False):
    """Layer-wise best intermediate bounds over `rules` (Sec. 7.2).

    l0, u0: [P, n_0].  Returns lists lb, ub indexed 1..n-1 (1..n with
    include_output), index 0 = the box; layer k is bounded with the best
    bounds of layers 1..k-1.
    """
    l0 = np.asarray(l0, np.float64)
    u0 = np.asarray(u0, np.float64)
    lb, ub = [l0], [u0]
    last = net.n if include_output else net.n - 1
    for k in range(1, last + 1):
        lows, ups = zip(*(layer_bounds(net, k, l0, u0, lb, ub, r) for r in rules))
        lb.append(np.max(np.stack(lows), axis=0))
        ub.append(np.min(np.stack(ups), axis=0))
    return lb, ub


def crown_wk_bounds_split(net: Net, l0, u0, masks, prop=None, rules=RULES):
    """Layer-wise best bounds recomputed per subdomain after its splits (the
    bounds refreshed after every activation split in the paper's comparison of
    intermediate-bound strategies, Sec. 8.4; split semantics of Sec. 2.3.2).

    For subdomain b, layer 1 is bounded over box prop[b]; layer k's best
    bounds are clamped by the subdomain's split mask (+1 => l <- max(l,0),
    -1 => u <- min(u,0)) before they enter the relaxations that bound the
    layers after it.  masks: [B, sum_k n_k] over layers 1..n-1.  Returns
    clamped lists lb, ub indexed 1..n-1 of [B, n_k] (index 0 = the boxes)
    and a boolean [B] that is True where some l > u (empty domain).
    """
    masks = np.asarray(masks)
    B = masks.shape[0]
    prop = np.zeros(B, dtype=np.int64) if prop is None else np.asarray(prop, dtype=np.int64)
    L0 = np.asarray(l0, np.float64)[prop]
    U0 = np.asarray(u0, np.float64)[prop]
    offs = split_offsets(net)
    lb, ub = [L0], [U0]
    empty = np.zeros(B, dtype=bool)
    for k in range(1, net.n):
        lows, ups = zip(*(layer_bounds(net, k, L0, U0, lb, ub, r) for r in rules))
        m = masks[:, offs[k - 1]:offs[k]]
        lk = np.max(np.stack(lows), axis=0)
        uk = np.min(np.stack(ups), axis=0)
        lk = np.where(m > 0, np.maximum(lk, 0.0), lk)
        uk = np.where(m < 0, np.minimum(uk, 0.0), uk)
        empty |= np.any(lk > uk, axis=1)
        lb.append(lk)
        ub.append(uk)
    return lb, ub, empty
