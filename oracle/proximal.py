"""Proximal solver of the LD dual (Sec. 3.3, Algorithm 2).

TEST INFRASTRUCTURE, NOT PRODUCT CODE: imported only by the test suite (the
same rule as the rest of this package).  Plain FP64, one layer block at a
time, in the order Algorithm 2 states.

What it computes.  The method of multipliers on the dual q of Eq.
(nonprox_problem): the dual update of Eq. (lambda_updates)

    lambda_k <- lambda_k + (x_hat_B,k - x_hat_A,k) / eta_k,

or its momentum form of App. D, Eq. (momentum_updates),

    pi_k <- mu pi_k + (x_hat_B,k - x_hat_A,k) / eta_k,   lambda_k <- lambda_k + pi_k,

alternating with an approximate minimisation of the Augmented Lagrangian of
Eq. (z_updates) over the primal blocks (x_hat_B,k, x_hat_A,k+1), k = 0..n-1
(x_hat_B,0 := 0), each a layer-pair subproblem P_k:

    L(x_hat, lambda) = x_hat_A,n + sum_k lambda_k^T (x_hat_B,k - x_hat_A,k)
                       + sum_k 1/(2 eta_k) ||x_hat_B,k - x_hat_A,k||^2.

The minimisation is J sweeps of block-coordinate Frank-Wolfe (Sec. 3.3.2):
for k = 0..n-1, the conditional gradient of block k minimises the
linearisation of L over P_k, whose coefficients are
grad_{x_hat_B,k} L = lambda_k + (x_hat_B,k - x_hat_A,k)/eta_k and
grad_{x_hat_A,k+1} L = -(lambda_{k+1} + (x_hat_B,k+1 - x_hat_A,k+1)/eta_{k+1})
(= 1 for k + 1 = n) -- the inner minimisation of P_k used for the
supergradient, at those duals; the block then moves to the convex
combination gamma z + (1 - gamma) x with the optimal step of Eq.
(optimal-gamma-gauss), clipped to [0, 1] (eta_n = infinity).  Initialisation
(Algorithm 2): lambda^0 by Prop. 3 (CROWN), x_hat^0 the inner minimiser of
q(lambda^0).  The primal blocks carry over from one outer iteration to the
next.  Returned: q(lambda^T), and the trace q(lambda^t).

Hyper-parameters: J = 2 (Sec. 7.2); eta increased linearly from 10 to 500
over the iterations with momentum mu = 0.3 (the incomplete-verification
setting of Sec. 7.2), or eta fixed to 100 without momentum (the branch and
bound setting of Sec. 8.2).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .ld_oracle import Net, box_argmin, crown_init, dual_value, inner_minimisation, relu_subproblem_argmin


@dataclass
class ProxSettings:
    eta0: float = 1e1        # weight of the proximal terms at iteration 0
    eta_end: float = 5e2     # ... at the last iteration (linear schedule)
    mu: float = 0.3          # momentum of Eq. (momentum_updates); 0 = Eq. (lambda_updates)
    J: int = 2               # Frank-Wolfe sweeps per outer iteration


BAB_SETTINGS = ProxSettings(eta0=1e2, eta_end=1e2, mu=0.0, J=2)


def eta_at(t: int, T: int, s: ProxSettings) -> float:
    """eta of outer iteration t (the same for every layer), linear from eta0 to eta_end."""
    return s.eta0 + (s.eta_end - s.eta0) * t / max(T - 1, 1)


@dataclass
class Primal:
    """The primal blocks: xB[k] (k = 1..n-1) and xA[k] (k = 1..n), lists with
    unused index 0; each [B, n_k]."""
    xB: list
    xA: list

    def copy(self):
        return Primal([None] + [x.copy() for x in self.xB[1:]], [None] + [x.copy() for x in self.xA[1:]])


def augmented_lagrangian(net: Net, P: Primal, lam, eta: float):
    """L(x_hat, lambda) of Eq. (z_updates), per subdomain [B]."""
    val = P.xA[net.n][:, 0].copy()
    for k in range(1, net.n):
        d = P.xB[k] - P.xA[k]
        val += np.sum(lam[k] * d, axis=1) + np.sum(d * d, axis=1) / (2.0 * eta)
    return val


def block_duals(net: Net, P: Primal, lam, eta: float, k: int):
    """(grad of L wrt x_hat_B,k, the dual whose transposed pass gives the
    coefficient of x_k) for block k: lambda'_k and lambda'_{k+1}, with
    lambda'_j = lambda_j + (x_hat_B,j - x_hat_A,j)/eta and lambda'_n = -1."""
    n = net.n
    B = P.xA[n].shape[0]
    lp_k = None if k == 0 else lam[k] + (P.xB[k] - P.xA[k]) / eta
    lp_k1 = -np.ones((B, 1)) if k + 1 == n else lam[k + 1] + (P.xB[k + 1] - P.xA[k + 1]) / eta
    return lp_k, lp_k1


def conditional_gradient(net: Net, k: int, lp_k, lp_k1, l0, u0, lb, ub):
    """Minimiser (z_B,k, z_A,k+1) of lp_k^T x_hat_B,k - lp_k1^T x_hat_A,k+1
    over P_k: the inner minimisation of P_k (P_0 for k = 0) at rho = lp_k,
    g_k = W_{k+1}^T lp_k1 (Sec. 3.3.2, conditional gradient computation).
    z_B,0 is None (the dummy zero block)."""
    g = net.L(k + 1).transposed(lp_k1)
    if k == 0:
        x0 = box_argmin(-g, l0, u0)
        return None, net.L(1).forward(x0)
    zb, xk, _ = relu_subproblem_argmin(lp_k, g, lb[k], ub[k])
    return zb, net.L(k + 1).forward(xk)


def optimal_step(net: Net, k: int, P: Primal, lp_k, lp_k1, zB, zA, eta: float):
    """gamma_k^* of Eq. (optimal-gamma-gauss): the exact minimiser over [0,1]
    of L along the segment from block k's current value to (zB, zA).  The
    derivative of L along the segment at gamma = 0 is -num; its curvature is
    den.  With den = 0, L is linear along the segment: gamma = 1 if it
    decreases, else 0."""
    n = net.n
    dA = zA - P.xA[k + 1]
    gA = np.ones_like(zA) if k + 1 == n else -lp_k1
    num = -np.sum(gA * dA, axis=1)
    den = np.zeros_like(num)
    if k >= 1:
        dB = zB - P.xB[k]
        num -= np.sum(lp_k * dB, axis=1)
        den += np.sum(dB * dB, axis=1) / eta
    if k + 1 < n:
        den += np.sum(dA * dA, axis=1) / eta
    safe = np.where(den > 0, den, 1.0)
    gam = np.where(den > 0, np.clip(num / safe, 0.0, 1.0), np.where(num > 0, 1.0, 0.0))
    return gam


def frank_wolfe_sweep(net: Net, P: Primal, lam, eta: float, l0, u0, lb, ub):
    """One block-coordinate sweep k = 0..n-1 (the inner loop of Algorithm 2);
    P is updated in place.  Returns the step sizes [n, B]."""
    gams = []
    for k in range(net.n):
        lp_k, lp_k1 = block_duals(net, P, lam, eta, k)
        zB, zA = conditional_gradient(net, k, lp_k, lp_k1, l0, u0, lb, ub)
        gam = optimal_step(net, k, P, lp_k, lp_k1, zB, zA, eta)[:, None]
        if k >= 1:
            P.xB[k] = gam * zB + (1.0 - gam) * P.xB[k]
        P.xA[k + 1] = gam * zA + (1.0 - gam) * P.xA[k + 1]
        gams.append(gam[:, 0])
    return np.array(gams)


@dataclass
class ProxResult:
    lam: list
    pi: list
    primal: Primal
    q_trace: np.ndarray   # [T, B]: q(lambda^t), t = 0..T-1
    q_final: np.ndarray   # [B]: q(lambda^T)


def proximal_solver(net: Net, l0, u0, lb, ub, T: int, s: ProxSettings = ProxSettings(), lam0=None,
                    primal0: Primal = None, pi0=None, t0: int = 0, T_sched: int | None = None):
    """Algorithm 2 for T outer iterations (lb, ub: clamped intermediate
    bounds, lists 1..n-1 of [B, n_k]).  lam0 None = CROWN (Prop. 3);
    primal0 None = the inner minimiser of q(lam0); t0, pi0 and T_sched resume
    a run split across calls."""
    n = net.n
    lam = crown_init(net, lb, ub)[0] if lam0 is None else [None] + [np.array(x, np.float64) for x in lam0[1:]]
    if primal0 is None:
        sol = inner_minimisation(net, l0, u0, lb, ub, lam)
        P = Primal([None] + [sol.xB[k].copy() for k in range(1, n)], [None] + [sol.xA[k].copy() for k in range(1, n + 1)])
    else:
        P = primal0.copy()
    pi = [None] + [np.zeros_like(lam[k]) if pi0 is None else np.array(pi0[k], np.float64) for k in range(1, n)]
    Ts = T if T_sched is None else T_sched
    trace = []
    for t in range(T):
        trace.append(dual_value(net, l0, u0, lb, ub, lam))
        eta = eta_at(t0 + t, Ts, s)
        for _ in range(s.J):
            frank_wolfe_sweep(net, P, lam, eta, l0, u0, lb, ub)
        for k in range(1, n):
            step = (P.xB[k] - P.xA[k]) / eta
            pi[k] = s.mu * pi[k] + step
            lam[k] = lam[k] + pi[k]
    q_final = dual_value(net, l0, u0, lb, ub, lam)
    q_trace = np.array(trace) if trace else np.zeros((0, l0.shape[0]))
    return ProxResult(lam=lam, pi=pi, primal=P, q_trace=q_trace, q_final=q_final)


__all__ = ["ProxSettings", "BAB_SETTINGS", "eta_at", "Primal", "augmented_lagrangian", "block_duals",
           "conditional_gradient", "optimal_step", "frank_wolfe_sweep", "ProxResult", "proximal_solver"]
