"""Independent evaluators for the oracle: LPs and exact minima (SciPy HiGHS).

TEST INFRASTRUCTURE, NOT PRODUCT CODE (see the header of ld_oracle.py).

* planet_lp: the Planet relaxation of Eq. (planet-relax) with the ReLU hull of
  Eq. (planet-relu-hull), written with the copies x_hat_A / x_hat_B of Eq.
  (primal_lag_problem) so that the multipliers of the agreement rows
  x_hat_B,k - x_hat_A,k = 0 are the LD duals (Prop. 1: max q = LP optimum).
* exact_min_enumeration: the exact minimum of Eq. (noncvx_pb), one LP per
  activation pattern of the ambiguous ReLUs (tiny nets only).
* exact_min_milp: the same minimum as a big-M mixed-integer program.

Nets here are dense (FC) oracle nets; conv layers are used through their
explicit matrices.  Bounds passed in are the per-subdomain, mask-clamped
intermediate bounds of one subdomain (1-D arrays per layer).
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
from scipy.optimize import linprog, milp, LinearConstraint, Bounds

from .ld_oracle import Net, classify


def _dense(m):
    return m.toarray() if sp.issparse(m) else np.asarray(m)


@dataclass
class LPResult:
    p_star: float
    rho: list          # LD duals recovered from the agreement-row multipliers (1..n-1)
    status: int


def planet_lp(net: Net, l0, u0, lb, ub) -> LPResult:
    """Solve Eq. (planet-relax) for one subdomain in the split form.

    Variables, in order: x0 [n0], x_hat_A,k [n_k] for k=1..n, x_hat_B,k and
    x_k [n_k] for k=1..n-1.  Objective x_hat_A,n.
    """
    n = net.n
    w = net.widths
    idx = {}
    pos = 0

    def alloc(name, size):
        nonlocal pos
        idx[name] = (pos, pos + size)
        pos += size

    alloc("x0", w[0])
    for k in range(1, n + 1):
        alloc(f"A{k}", w[k])
    for k in range(1, n):
        alloc(f"B{k}", w[k])
        alloc(f"x{k}", w[k])
    nv = pos
    lo = np.full(nv, -np.inf)
    hi = np.full(nv, np.inf)
    a, b_ = idx["x0"]
    lo[a:b_] = l0
    hi[a:b_] = u0

    Aeq_rows, beq = [], []
    Aub_rows, bub = [], []

    def row():
        return np.zeros(nv)

    # linear layers: x_hat_A,k - W_k x_{k-1} = b_k
    for k in range(1, n + 1):
        Wk = _dense(net.L(k).mat)
        bk = net.L(k).bias_vector()
        prev = "x0" if k == 1 else f"x{k-1}"
        pa, _ = idx[prev]
        aa, _ = idx[f"A{k}"]
        for i in range(w[k]):
            r = row()
            r[aa + i] = 1.0
            r[pa:pa + w[k - 1]] -= Wk[i]
            Aeq_rows.append(r)
            beq.append(bk[i])
    # agreement rows: x_hat_B,k - x_hat_A,k = 0 (these carry the LD duals)
    agree_start = len(Aeq_rows)
    for k in range(1, n):
        ba, _ = idx[f"B{k}"]
        aa, _ = idx[f"A{k}"]
        for i in range(w[k]):
            r = row()
            r[ba + i] = 1.0
            r[aa + i] = -1.0
            Aeq_rows.append(r)
            beq.append(0.0)
    # ReLU hulls on (x_k, x_hat_B,k), Eq. (planet-relu-hull)
    for k in range(1, n):
        l, u = lb[k], ub[k]
        cls = classify(l, u)
        ba, _ = idx[f"B{k}"]
        xa, _ = idx[f"x{k}"]
        for i in range(w[k]):
            lo[ba + i], hi[ba + i] = l[i], u[i]
            if cls[i] == 0:          # blocking: x = 0
                lo[xa + i], hi[xa + i] = 0.0, 0.0
            elif cls[i] == 1:        # passing: x = x_hat
                lo[xa + i], hi[xa + i] = l[i], u[i]
                r = row()
                r[xa + i] = 1.0
                r[ba + i] = -1.0
                Aeq_rows.append(r)
                beq.append(0.0)
            else:                    # ambiguous: x >= 0, x >= x_hat, x <= u (x_hat - l)/(u - l)
                lo[xa + i], hi[xa + i] = 0.0, u[i]
                r = row()
                r[ba + i] = 1.0
                r[xa + i] = -1.0
                Aub_rows.append(r)
                bub.append(0.0)
                r = row()
                r[xa + i] = u[i] - l[i]
                r[ba + i] = -u[i]
                Aub_rows.append(r)
                bub.append(-u[i] * l[i])
    c = np.zeros(nv)
    c[idx[f"A{n}"][0]] = 1.0
    res = linprog(c, A_ub=np.array(Aub_rows) if Aub_rows else None,
                  b_ub=np.array(bub) if bub else None,
                  A_eq=np.array(Aeq_rows), b_eq=np.array(beq),
                  bounds=list(zip(lo, hi)), method="highs")
    if res.status != 0:
        return LPResult(p_star=np.nan, rho=None, status=res.status)
    y = res.eqlin.marginals[agree_start:agree_start + sum(w[1:n])]
    rho, off = [None], 0
    for k in range(1, n):
        # HiGHS marginals are d p*/d b_eq, i.e. the Lagrangian c^T z - y^T (A z - b);
        # the LD Lagrangian adds +rho^T (x_hat_B - x_hat_A), hence rho = -y.
        rho.append(-y[off:off + w[k]])
        off += w[k]
    return LPResult(p_star=float(res.fun), rho=rho, status=0)


def exact_min_enumeration(net: Net, l0, u0, lb, ub, max_ambiguous: int = 12) -> float:
    """Exact min of Eq. (noncvx_pb) over the box: one LP per activation pattern.

    Stable ReLUs keep their phase; each ambiguous ReLU is either on
    (x = x_hat >= 0) or off (x = 0, x_hat <= 0).  Uses the intermediate bounds
    only to classify (they are valid, so no minimiser is cut off).
    """
    n = net.n
    w = net.widths
    cls = [None] + [classify(lb[k], ub[k]) for k in range(1, n)]
    amb = [(k, i) for k in range(1, n) for i in range(w[k]) if cls[k][i] == 2]
    if len(amb) > max_ambiguous:
        raise ValueError(f"{len(amb)} ambiguous ReLUs: too many to enumerate")
    best = np.inf
    Ws = [None] + [_dense(net.L(k).mat) for k in range(1, n + 1)]
    bs = [None] + [net.L(k).bias_vector() for k in range(1, n + 1)]
    for pattern in itertools.product((0, 1), repeat=len(amb)):
        on = [None] + [cls[k] == 1 for k in range(1, n)]
        for (k, i), p in zip(amb, pattern):
            on[k] = on[k].copy()
            on[k][i] = bool(p)
        # x_hat_k is affine in x0 under a fixed pattern: x_hat_k = M_k x0 + c_k
        M = np.eye(w[0])
        cvec = np.zeros(w[0])
        A_ub, b_ub = [], []
        for k in range(1, n + 1):
            M = Ws[k] @ M
            cvec = Ws[k] @ cvec + bs[k]
            if k == n:
                break
            for i in range(w[k]):
                if on[k][i]:          # x_hat >= 0  ->  -M x0 <= c
                    A_ub.append(-M[i])
                    b_ub.append(cvec[i])
                else:                 # x_hat <= 0
                    A_ub.append(M[i])
                    b_ub.append(-cvec[i])
            D = on[k].astype(np.float64)
            M = D[:, None] * M
            cvec = D * cvec
        res = linprog(M[0], A_ub=np.array(A_ub) if A_ub else None,
                      b_ub=np.array(b_ub) if b_ub else None,
                      bounds=list(zip(l0, u0)), method="highs")
        if res.status == 0:
            best = min(best, res.fun + cvec[0])
    return float(best)


def exact_min_milp(net: Net, l0, u0, lb, ub) -> float:
    """Exact min of Eq. (noncvx_pb) as a big-M MILP (valid bounds as big-M).

    Ambiguous ReLU with binary z: x >= x_hat, x >= 0, x <= x_hat - l (1 - z),
    x <= u z.  Stable ReLUs are fixed to their phase.
    """
    n = net.n
    w = net.widths
    idx = {}
    pos = 0
    for name, size in [("x0", w[0])] + [(f"h{k}", w[k]) for k in range(1, n + 1)] + \
            [(f"x{k}", w[k]) for k in range(1, n)] + [(f"z{k}", w[k]) for k in range(1, n)]:
        idx[name] = pos
        pos += size
    nv = pos
    lo = np.full(nv, -np.inf)
    hi = np.full(nv, np.inf)
    integ = np.zeros(nv)
    lo[idx["x0"]:idx["x0"] + w[0]] = l0
    hi[idx["x0"]:idx["x0"] + w[0]] = u0
    rows, rl, ru = [], [], []

    def add(r, a, b):
        rows.append(r)
        rl.append(a)
        ru.append(b)

    for k in range(1, n + 1):
        Wk = _dense(net.L(k).mat)
        bk = net.L(k).bias_vector()
        prev = idx["x0"] if k == 1 else idx[f"x{k-1}"]
        for i in range(w[k]):
            r = np.zeros(nv)
            r[idx[f"h{k}"] + i] = 1.0
            r[prev:prev + w[k - 1]] -= Wk[i]
            add(r, bk[i], bk[i])
    for k in range(1, n):
        cls = classify(lb[k], ub[k])
        for i in range(w[k]):
            h = idx[f"h{k}"] + i
            x = idx[f"x{k}"] + i
            z = idx[f"z{k}"] + i
            l, u = lb[k][i], ub[k][i]
            lo[h], hi[h] = l, u
            lo[z], hi[z] = 0.0, 1.0
            integ[z] = 1
            if cls[i] == 0:
                lo[x], hi[x] = 0.0, 0.0
                hi[z] = 0.0
            elif cls[i] == 1:
                lo[z] = 1.0
                r = np.zeros(nv)
                r[x] = 1.0
                r[h] = -1.0
                add(r, 0.0, 0.0)
            else:
                lo[x], hi[x] = 0.0, u
                r = np.zeros(nv); r[x] = 1.0; r[h] = -1.0
                add(r, 0.0, np.inf)                 # x >= x_hat
                r = np.zeros(nv); r[x] = 1.0; r[h] = -1.0; r[z] = -l
                add(r, -np.inf, -l)                 # x <= x_hat - l + l z
                r = np.zeros(nv); r[x] = 1.0; r[z] = -u
                add(r, -np.inf, 0.0)                # x <= u z
    c = np.zeros(nv)
    c[idx[f"h{n}"]] = 1.0
    res = milp(c, constraints=LinearConstraint(np.array(rows), rl, ru),
               integrality=integ, bounds=Bounds(lo, hi))
    if res.status != 0:
        raise RuntimeError(f"milp status {res.status}: {res.message}")
    return float(res.fun)
