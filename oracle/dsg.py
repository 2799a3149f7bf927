"""The dual of Dvijotham et al. solved by supergradient ascent (DSG+) and its
decomposed evaluation Dec-DSG+ (Sec. 2.2.2, Eq. (dj_prob-main), Theorem 1,
Sec. 7.2).

TEST INFRASTRUCTURE, NOT PRODUCT CODE: imported only by the test suite (the
same rule as the rest of this package).  Plain FP64.

What it computes.  With multipliers mu_k on x_hat_k = W_k x_{k-1} + b_k and
lambda_k on x_k = relu(x_hat_k) (k = 1..n-1),

  d_O(mu, lambda) = min over x_0 in the box, x_k in [relu(l_k), relu(u_k)],
                    x_hat_k in [l_k, u_k] of
      sum_k mu_k^T (x_hat_k - W_k x_{k-1} - b_k)
    + sum_k lambda_k^T (x_k - relu(x_hat_k)) + W_n x_{n-1} + b_n,

which separates into independent minima (g_k := W_{k+1}^T mu_{k+1} with
mu_n := -1, the same transposed products as the LD dual):
  * x_0: min over the box of -g_0^T x_0 (the box argmin of Eq. (box_bounds_sol));
  * x_k: min over [relu(l_k), relu(u_k)] of (lambda_k - g_k)^T x_k, a box argmin;
  * x_hat_k: min over [l_k, u_k] of mu_k x_hat - lambda_k relu(x_hat), a
    piecewise-linear function minimised at l_k, 0 (when l_k < 0 < u_k) or u_k;
  * constants b_n - sum_k mu_k^T b_k.
Its supergradient is (x_hat_k* - W_k x_{k-1}* - b_k, x_k* - relu(x_hat_k*)).
DSG+ ascends it with Adam (step size linear between two values, Sec. 7.2),
started from CROWN (Prop. 3: mu = rho_CROWN and lambda_{k-1} = W_k^T mu_k,
lambda_{n-1} = -W_n^T 1, where d_O equals the CROWN bound).  Dec-DSG+
evaluates the LD dual q at mu (Theorem 1: q(mu) >= d_O(mu, lambda)).
Readings (listed in the design notes): box argmins take the upper end where
the coefficient is <= 0 (as in Eq. (box_bounds_sol)); d_O is summed from
the exact minima, while the returned x_hat (the supergradient's point) is
the first strict minimum in the order l, 0, u with u having to win by
2^-16 (|mu| + |lambda|) max(|l|, |u|), the LD dual's tie margin.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .ld_oracle import TIE_REL, AdamSettings, Net, adam_update, box_argmin, classify, crown_init


@dataclass
class DsgInner:
    d: np.ndarray          # [B] d_O(mu, lambda)
    g: list                # g_k = W_{k+1}^T mu_{k+1}, k = 0..n-1
    x: list                # x_k*, k = 0..n-1
    xh: list               # x_hat_k*, k = 1..n-1
    xA: list               # W_k x_{k-1}* + b_k, k = 1..n


def dsg_inner(net: Net, l0, u0, lb, ub, mu, lam) -> DsgInner:
    """The separable minimisation of d_O at (mu, lambda); lb, ub clamped
    intermediate bounds (lists 1..n-1 of [B, n_k])."""
    n = net.n
    B = l0.shape[0]
    g = [None] * n
    for k in range(n):
        nxt = -np.ones((B, 1)) if k + 1 == n else mu[k + 1]
        g[k] = net.L(k + 1).transposed(nxt)
    x = [box_argmin(-g[0], l0, u0)]
    d = np.sum(np.minimum(-g[0] * l0, -g[0] * u0), axis=1) + net.L(n).bias_vector()[0]
    xh = [None]
    for k in range(1, n):
        l, u = lb[k], ub[k]
        c = lam[k] - g[k]
        rl, ru = np.maximum(l, 0.0), np.maximum(u, 0.0)
        xk = box_argmin(c, rl, ru)
        # x_hat: candidates l, 0 (inside the interval), u.  The value is the
        # exact minimum; the returned point is the first strict minimum in
        # that order, u having to win by the tie margin of the LD reading: at
        # the CROWN start (Prop. 3) mu l and (mu - lambda) u tie exactly for
        # every ambiguous ReLU with lambda > 0, and rounding must not decide.
        f = lambda v: mu[k] * v - lam[k] * np.maximum(v, 0.0)
        inside = (l < 0) & (u > 0)
        fl, f0, fu = f(l), np.where(inside, 0.0, np.inf), f(u)
        best = np.minimum(np.minimum(fl, f0), fu)
        pick, arg = fl, l.copy()
        take = f0 < pick
        pick, arg = np.where(take, f0, pick), np.where(take, 0.0, arg)
        margin = TIE_REL * (np.abs(mu[k]) + np.abs(lam[k])) * np.maximum(np.abs(l), np.abs(u))
        take = fu < pick - margin
        arg = np.where(take, u, arg)
        d = d + np.sum(c * xk, axis=1) + np.sum(best, axis=1) - mu[k] @ net.L(k).bias_vector()
        x.append(xk)
        xh.append(arg)
    xA = [None] + [net.L(k).forward(x[k - 1]) for k in range(1, n + 1)]
    return DsgInner(d=d, g=g, x=x, xh=xh, xA=xA)


def dsg_value(net, l0, u0, lb, ub, mu, lam):
    """d_O(mu, lambda) of Eq. (dj_prob-main) [B]."""
    return dsg_inner(net, l0, u0, lb, ub, mu, lam).d


def dsg_init(net: Net, lb, ub):
    """(mu, lambda) from CROWN (Prop. 3): mu = the CROWN duals, lambda_k = g_k."""
    rho, lam = crown_init(net, lb, ub)
    return rho, lam


@dataclass
class DsgResult:
    mu: list
    lam: list
    d_trace: np.ndarray    # [T, B] d_O at the iterates
    d_final: np.ndarray    # [B] d_O(mu_T, lambda_T): the DSG+ bound
    q_final: np.ndarray    # [B] q(mu_T): the Dec-DSG+ bound (Theorem 1)


def dsg_plus(net: Net, l0, u0, lb, ub, T: int, s: AdamSettings = AdamSettings(), mu0=None, lam0=None):
    """T Adam steps of supergradient ascent on d_O from CROWN (or (mu0, lam0))."""
    from .ld_oracle import dual_value
    n = net.n
    if mu0 is None:
        mu0, lam0 = dsg_init(net, lb, ub)
    mu = [None] + [np.array(mu0[k], np.float64) for k in range(1, n)]
    lam = [None] + [np.array(lam0[k], np.float64) for k in range(1, n)]
    mm = [None] + [np.zeros_like(mu[k]) for k in range(1, n)]
    mv = [None] + [np.zeros_like(mu[k]) for k in range(1, n)]
    lm = [None] + [np.zeros_like(mu[k]) for k in range(1, n)]
    lv = [None] + [np.zeros_like(mu[k]) for k in range(1, n)]
    trace = []
    for t in range(T):
        inn = dsg_inner(net, l0, u0, lb, ub, mu, lam)
        trace.append(inn.d)
        for k in range(1, n):
            s_mu = inn.xh[k] - inn.xA[k]
            s_lam = inn.x[k] - np.maximum(inn.xh[k], 0.0)
            mu[k], mm[k], mv[k] = adam_update(mu[k], mm[k], mv[k], s_mu, t, T, s)
            lam[k], lm[k], lv[k] = adam_update(lam[k], lm[k], lv[k], s_lam, t, T, s)
    d_final = dsg_value(net, l0, u0, lb, ub, mu, lam)
    q_final = dual_value(net, l0, u0, lb, ub, mu)
    return DsgResult(mu=mu, lam=lam, d_trace=np.array(trace) if trace else np.zeros((0, l0.shape[0])),
                     d_final=d_final, q_final=q_final)


__all__ = ["DsgInner", "dsg_inner", "dsg_value", "dsg_init", "DsgResult", "dsg_plus"]
