"""l2-ball input domains (Sec. 3.2.1).

TEST INFRASTRUCTURE, NOT PRODUCT CODE: imported only by the test suite (the
same rule as the rest of this package).  Plain FP64.

When the input domain is the ball ||x0 - c||_2 <= eps, the P0 subproblem of
the LD dual (Sec. 3.2.1) minimises the linear function -g_0^T x0 over the
ball: the minimiser is the boundary point in the direction of g_0,
x0* = c + eps g_0 / ||g_0||_2 (any point of the ball when g_0 = 0; c here),
and the minimum is -g_0^T c - eps ||g_0||_2.  Reading (listed in the design
notes): the section writes the direction as the dual vector of layer 1; the
cost of P0 is -(W_1^T rho_1)^T x0, so the direction is g_0 = W_1^T rho_1.
The first layer's exact interval bounds over the ball are
(W_1 c + b_1)_j -+ eps ||W_1[j, :]||_2 (Cauchy-Schwarz, attained at
c -+ eps W_1[j,:] / ||W_1[j,:]||); later layers by interval propagation.
"""
from __future__ import annotations

import numpy as np

from .ld_oracle import Net


def ball_argmin(g, c, eps):
    """argmin of -g^T x over ||x - c|| <= eps, rows of g [B, n0]; eps [B]."""
    g = np.asarray(g, np.float64)
    c = np.asarray(c, np.float64)
    eps = np.asarray(eps, np.float64).reshape(-1, 1)
    nrm = np.linalg.norm(g, axis=1, keepdims=True)
    step = np.divide(g, nrm, out=np.zeros_like(g), where=nrm > 0)
    return c + eps * step


def ball_min(g, c, eps):
    """min of -g^T x over ||x - c|| <= eps: -g^T c - eps ||g||  [B]."""
    g = np.asarray(g, np.float64)
    return -np.sum(g * np.asarray(c, np.float64), axis=1) - np.asarray(eps, np.float64).reshape(-1) * np.linalg.norm(
        g, axis=1)


def ball_first_layer_bounds(net: Net, c, eps):
    """Exact range of x_hat_1 = W_1 x0 + b_1 over the ball: (lower, upper) [P, n_1]."""
    lay = net.L(1)
    c = np.asarray(c, np.float64)
    mid = lay.forward(c)
    rows = np.sqrt(np.asarray(lay.mat.multiply(lay.mat).sum(axis=1)).reshape(-1)) if hasattr(lay.mat, "multiply") \
        else np.linalg.norm(lay.mat, axis=1)
    rad = np.asarray(eps, np.float64).reshape(-1, 1) * rows[None, :]
    return mid - rad, mid + rad


def ball_ibp_bounds(net: Net, c, eps):
    """Interval bounds of layers 1..n over the ball: the first layer exact
    (ball_first_layer_bounds), the rest by interval propagation as in
    ibp_bounds; lists indexed 1..n (index 0: None)."""
    l1, u1 = ball_first_layer_bounds(net, c, eps)
    lb, ub = [None, l1], [None, u1]
    lo, hi = np.maximum(l1, 0.0), np.maximum(u1, 0.0)
    for k in range(2, net.n + 1):
        lay = net.L(k)
        mid, rad = (lo + hi) / 2.0, (hi - lo) / 2.0
        cen = lay.forward(mid)
        r = np.asarray((abs(lay.mat) @ rad.T).T)
        lb.append(cen - r)
        ub.append(cen + r)
        lo, hi = np.maximum(lb[-1], 0.0), np.maximum(ub[-1], 0.0)
    return lb, ub


def ball_points(c, eps, n, seed):
    """n points of the ball around c (c [n0]): half on the sphere, half inside."""
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((n, c.shape[0]))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = np.ones(n)
    r[n // 2:] = rng.random(n - n // 2) ** (1.0 / c.shape[0])
    return c[None, :] + eps * r[:, None] * d


__all__ = ["ball_argmin", "ball_min", "ball_first_layer_bounds", "ball_ibp_bounds", "ball_points"]
