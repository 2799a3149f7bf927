"""Plain FP64 CPU oracle for the Lagrangian-Decomposition (LD) dual bound.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke check
and the benchmark's CPU-baseline leg may import, call or execute anything in
this package.  It shares no code with the CUDA path and imports nothing from
the product package.

What it computes (De Palma et al., "Improved Branch and Bound for Neural
Network Verification via Lagrangian Decomposition"):

* problem:   min x_hat_n over an L-infinity box, Sec. 2.1, Eq. (noncvx_pb)
* intermediate bounds: interval bound propagation (IBP), Sec. 2.2.3 and the
  IBP item of Sec. 7.2 (IBP = all duals set to zero)
* split masks: a ReLU fixed to its passing or blocking phase, Sec. 2.3.2
* LD dual q(rho), Sec. 3.1 Eq. (nonprox_problem); its inner minimisation:
  P0 box argmin Eq. (box_bounds_sol), Pk 3-vertex argmin Eq. (min-pk) and the
  box argmins for non-ambiguous ReLUs (Sec. 3.2.2)
* supergradient x_hat_B - x_hat_A and the Adam ascent of Algorithm 1,
  Eq. (subgradient_update), step size decayed linearly (Sec. 7.2)
* dual initialisation from CROWN, Prop. 3 and Eq. (salman-assignment), with
  the CROWN slopes of the footnote in Sec. 4.2 and Eq. (slopes-biases)
* the closed-form propagation bound Eq. (bounds-propagation)
* Danskin gradients of q at fixed rho (not in the paper: Danskin's theorem
  applied to the inner minimum of Eq. (nonprox_problem))

Conventions (readings of the paper, each one listed in the design notes):

* layers are numbered k = 1..n; layer k maps x_{k-1} to x_hat_k; ReLU after
  every layer but the last; the last layer has one output (margin folded in);
* rho is a list indexed 1..n-1 (index 0 unused); rho_n := -1 (App. A/B);
* g_k := W_{k+1}^T rho_{k+1}, k = 0..n-1;
* min_{y in [l,u]} a*y is taken at y = u if a <= 0 else y = l (matches
  Eq. (box_bounds_sol), which picks u0 where rho_1^T W_1 >= 0);
* ambiguous vertex ties: the first strict minimum in the order
  (l,0), (0,0), (u,u);
* classification: blocking if u <= 0 (checked first), passing if l >= 0,
  ambiguous otherwise (Sec. 2.3.2);
* split mask +1 => l <- max(l,0); -1 => u <- min(u,0); l > u after that =>
  empty domain, bound +inf.

All arrays carry a leading subdomain axis: a per-layer quantity of layer k is
an array of shape [B, n_k].
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp


# --------------------------------------------------------------------------
# Network: layers as explicit matrices (a conv layer becomes a sparse matrix)
# --------------------------------------------------------------------------

@dataclass
class Layer:
    """One linear layer x_hat = W x + b of Eq. (noncvx_pb).

    kind 'fc': W is [n_out, n_in].  kind 'conv': W is [cout, cin, kh, kw],
    cross-correlation with zero padding (the usual deep-learning 'conv'),
    input and output flattened in channel-major (C, H, W) order.
    """
    kind: str
    W: np.ndarray
    b: np.ndarray
    in_shape: tuple = ()
    stride: int = 1
    pad: int = 0
    mat: object = field(default=None, repr=False)

    def __post_init__(self):
        self.W = np.asarray(self.W, dtype=np.float64)
        self.b = np.asarray(self.b, dtype=np.float64)
        if self.kind == "fc":
            self.mat = self.W
        elif self.kind == "conv":
            self.mat = conv_matrix(self.W, self.in_shape, self.stride, self.pad)
        else:
            raise ValueError(self.kind)

    @property
    def n_in(self) -> int:
        return self.mat.shape[1]

    @property
    def n_out(self) -> int:
        return self.mat.shape[0]

    def bias_vector(self) -> np.ndarray:
        """Per-output bias (a conv bias is repeated over the output plane)."""
        if self.kind == "fc":
            return self.b
        cout = self.W.shape[0]
        return np.repeat(self.b, self.n_out // cout)

    def forward(self, x: np.ndarray) -> np.ndarray:
        """x [B, n_in] -> W x + b, [B, n_out]."""
        return np.asarray((self.mat @ x.T).T) + self.bias_vector()[None, :]

    def transposed(self, r: np.ndarray) -> np.ndarray:
        """r [B, n_out] -> W^T r, [B, n_in] (no bias)."""
        return np.asarray((self.mat.T @ r.T).T)

    def linear(self, x: np.ndarray) -> np.ndarray:
        """x [B, n_in] -> W x, [B, n_out] (no bias)."""
        return np.asarray((self.mat @ x.T).T)


def conv_out_shape(in_shape, W, stride, pad):
    cout, cin, kh, kw = W.shape
    c, h, w = in_shape
    assert c == cin
    ho = (h + 2 * pad - kh) // stride + 1
    wo = (w + 2 * pad - kw) // stride + 1
    return cout, ho, wo


def conv_matrix(W, in_shape, stride, pad):
    """Sparse matrix of a zero-padded 2-D cross-correlation, written out tap by tap.

    Entry (o,y,x),(c,yy,xx) = W[o,c,i,j] where yy = y*stride - pad + i and
    xx = x*stride - pad + j lie inside the input plane.
    """
    cout, cin, kh, kw = W.shape
    c, h, w = in_shape
    _, ho, wo = conv_out_shape(in_shape, W, stride, pad)
    rows, cols, vals = [], [], []
    ys, xs = np.meshgrid(np.arange(ho), np.arange(wo), indexing="ij")
    ys = ys.ravel()
    xs = xs.ravel()
    for o in range(cout):
        out_idx = (o * ho + ys) * wo + xs
        for ci in range(cin):
            for i in range(kh):
                for j in range(kw):
                    yy = ys * stride - pad + i
                    xx = xs * stride - pad + j
                    ok = (yy >= 0) & (yy < h) & (xx >= 0) & (xx < w)
                    rows.append(out_idx[ok])
                    cols.append(((ci * h + yy[ok]) * w + xx[ok]))
                    vals.append(np.full(int(ok.sum()), W[o, ci, i, j]))
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    return sp.csr_matrix((vals, (rows, cols)), shape=(cout * ho * wo, c * h * w))


class Net:
    """An n-layer ReLU network in canonical form (scalar output), Sec. 2.1.

    `layers[0]` is layer 1 of the paper; `layers[k-1]` maps x_{k-1} to x_hat_k.
    """

    def __init__(self, layers):
        self.layers = list(layers)
        assert self.layers[-1].n_out == 1, "canonical form needs a scalar output"
        for a, b in zip(self.layers[:-1], self.layers[1:]):
            assert a.n_out == b.n_in

    @property
    def n(self) -> int:
        return len(self.layers)

    def L(self, k: int) -> Layer:
        """Layer k of the paper (1-based)."""
        return self.layers[k - 1]

    @property
    def widths(self):
        """[n_0, n_1, ..., n_n]."""
        return [self.layers[0].n_in] + [l.n_out for l in self.layers]

    def evaluate(self, x0: np.ndarray) -> np.ndarray:
        """The network itself: x0 [B, n_0] -> x_hat_n [B]."""
        x = x0
        for k in range(1, self.n + 1):
            xh = self.L(k).forward(x)
            x = np.maximum(xh, 0.0) if k < self.n else xh
        return x[:, 0]


def fold_margin(W_last, b_last, c):
    """Canonical form of a margin property (Sec. 2.1; Sec. 8.1 sets the output
    to ground-truth logit minus target logit): x_hat_n = c^T (W x + b)."""
    c = np.asarray(c, dtype=np.float64)
    return (c @ np.asarray(W_last, np.float64))[None, :], np.array([c @ np.asarray(b_last, np.float64)])


# --------------------------------------------------------------------------
# Intermediate bounds (IBP) and split masks
# --------------------------------------------------------------------------

def ibp_bounds(net: Net, l0: np.ndarray, u0: np.ndarray):
    """Interval bounds for every layer k = 1..n (Sec. 2.2.3; IBP in Sec. 7.2).

    l0, u0: [P, n_0].  Returns lists lb, ub indexed 1..n (index 0 = the box).
    Layer 1 is bounded over the box; layer k >= 2 over [relu(l_{k-1}), relu(u_{k-1})].
    """
    lb = [np.asarray(l0, np.float64)]
    ub = [np.asarray(u0, np.float64)]
    lo, hi = lb[0], ub[0]
    for k in range(1, net.n + 1):
        lay = net.L(k)
        mid = (lo + hi) / 2.0
        rad = (hi - lo) / 2.0
        Wabs = abs(lay.mat)
        c = lay.forward(mid)
        r = np.asarray((Wabs @ rad.T).T)
        lb.append(c - r)
        ub.append(c + r)
        lo = np.maximum(lb[-1], 0.0)
        hi = np.maximum(ub[-1], 0.0)
    return lb, ub


def split_offsets(net: Net):
    """Offsets of layers 1..n-1 inside a flat [sum_k n_k] vector."""
    offs = [0]
    for k in range(1, net.n):
        offs.append(offs[-1] + net.L(k).n_out)
    return offs  # offs[k-1] .. offs[k] is layer k


def apply_masks(net: Net, lb, ub, masks):
    """Clamp per-subdomain intermediate bounds by the split masks (Sec. 2.3.2).

    lb, ub: lists indexed 1..n-1 of [B, n_k] (already broadcast per subdomain).
    masks: int8 [B, sum n_k] in {-1, 0, +1}.  Returns clamped lists and a
    boolean [B] that is True where some l > u (empty subdomain).
    """
    offs = split_offsets(net)
    lb2, ub2 = [None], [None]
    empty = np.zeros(masks.shape[0], dtype=bool)
    for k in range(1, net.n):
        m = masks[:, offs[k - 1]:offs[k]]
        lo = np.where(m > 0, np.maximum(lb[k], 0.0), lb[k])
        hi = np.where(m < 0, np.minimum(ub[k], 0.0), ub[k])
        empty |= np.any(lo > hi, axis=1)
        lb2.append(lo)
        ub2.append(hi)
    return lb2, ub2, empty


def ibp_bounds_split(net: Net, l0: np.ndarray, u0: np.ndarray, masks: np.ndarray, prop=None):
    """Interval bounds recomputed per subdomain after its splits (the
    per-subdomain intermediate bounds of BaBSR, Sec. 5.1.1 / Sec. 2.3.2).

    For subdomain b, layer 1 is bounded over box prop[b]; the split clamp of
    Sec. 2.3.2 is applied to layer k's bounds (+1 => l <- max(l,0),
    -1 => u <- min(u,0)) before they bound layer k+1 through
    [relu(l_k), relu(u_k)].  Returns clamped lists lb, ub indexed 1..n-1 of
    [B, n_k] and a boolean [B] that is True where some l > u (empty domain).
    """
    masks = np.asarray(masks)
    B = masks.shape[0]
    prop = np.zeros(B, dtype=np.int64) if prop is None else np.asarray(prop, dtype=np.int64)
    lo = np.asarray(l0, np.float64)[prop]
    hi = np.asarray(u0, np.float64)[prop]
    offs = split_offsets(net)
    lb, ub = [None], [None]
    empty = np.zeros(B, dtype=bool)
    for k in range(1, net.n):
        lay = net.L(k)
        mid = (lo + hi) / 2.0
        rad = (hi - lo) / 2.0
        c = lay.forward(mid)
        r = np.asarray((abs(lay.mat) @ rad.T).T)
        m = masks[:, offs[k - 1]:offs[k]]
        lk = np.where(m > 0, np.maximum(c - r, 0.0), c - r)
        uk = np.where(m < 0, np.minimum(c + r, 0.0), c + r)
        empty |= np.any(lk > uk, axis=1)
        lb.append(lk)
        ub.append(uk)
        lo = np.maximum(lk, 0.0)
        hi = np.maximum(uk, 0.0)
    return lb, ub, empty


def classify(l, u):
    """ReLU phases of Sec. 2.3.2: 0 blocking (u <= 0), 1 passing (l >= 0), 2 ambiguous."""
    cls = np.full(l.shape, 2, dtype=np.int8)
    cls[l >= 0] = 1
    cls[u <= 0] = 0
    return cls


# --------------------------------------------------------------------------
# LD dual q(rho): inner minimisation of Eq. (nonprox_problem)
# --------------------------------------------------------------------------

@dataclass
class InnerSolution:
    q: np.ndarray          # [B] dual value q(rho)
    g: list                # g_k = W_{k+1}^T rho_{k+1}, k = 0..n-1
    x: list                # x_k^*, k = 0..n-1 (x_0 = box argmin)
    xB: list               # x_hat_B,k^*, k = 1..n-1 (index 0 unused)
    xA: list               # x_hat_A,k^*, k = 1..n   (index 0 unused)
    vertex: list           # chosen vertex/endpoint code per neuron, k = 1..n-1
    q_point: np.ndarray = None  # [B] Lagrangian at the returned point (>= q by at most the tie margins)


TIE_REL = 2.0 ** -16   # vertex tie tolerance of the (u,u) comparison (a reading; see inner_minimisation)


def box_argmin(a, l, u):
    """argmin_{y in [l,u]} a*y, taking u when a <= 0 (Eq. (box_bounds_sol) rule)."""
    return np.where(a <= 0, u, l)


class ExactPasses:
    """The two linear passes of the inner minimisation in FP64 arithmetic."""

    def __init__(self, net: Net):
        self.net = net

    def transposed(self, k: int, r):
        """g_{k-1} = W_k^T r (no bias)."""
        return self.net.L(k).transposed(r)

    def forward(self, k: int, x):
        """x_hat_A,k = W_k x + b_k."""
        return self.net.L(k).forward(x)


def relu_subproblem_argmin(r, c, l, u):
    """argmin of r * x_hat_B - c * x over the Planet hull of one ReLU layer
    (Sec. 3.2.2, Eq. (min-pk)), elementwise.  Returns (x_hat_B, x, vertex
    code): 0 -> (l,0) / lower end, 1 -> (0,0), 2 -> (u,u) / upper end."""
    cls = classify(l, u)
    xb = np.zeros_like(r)
    xk = np.zeros_like(r)
    code = np.zeros(r.shape, dtype=np.int8)
    # blocking: x = 0, minimise r * x_hat_B over [l, u]
    blk = cls == 0
    xb[blk] = box_argmin(r, l, u)[blk]
    code[blk] = np.where(r <= 0, 2, 0)[blk]
    # passing: x = x_hat_B, minimise (r - c) * x_hat_B over [l, u]; the
    # lower end needs r - c > TIE_REL (|r| + |c|): at the CROWN point
    # r = c exactly for every passing ReLU, and rounding must not decide
    pas = cls == 1
    low = (r - c) > TIE_REL * (np.abs(r) + np.abs(c))
    yp = np.where(low, l, u)
    xb[pas] = yp[pas]
    xk[pas] = yp[pas]
    code[pas] = np.where(low, 0, 2)[pas]
    # ambiguous: the three vertices of Fig. (relucvx), Eq. (min-pk)
    amb = cls == 2
    v_l0 = r * l                  # vertex (l, 0)
    v_00 = np.zeros_like(r)       # vertex (0, 0)
    v_uu = (r - c) * u            # vertex (u, u)
    best = v_l0.copy()
    choice = np.zeros(r.shape, dtype=np.int8)
    take = v_00 < best
    best = np.where(take, v_00, best)
    choice[take] = 1
    # (u,u) must win by more than TIE_REL of the magnitudes that enter
    # the comparison, (|r| + |g|) * max(|l|, u): the CROWN point of
    # Prop. 3 puts (l,0) and (u,u) at an exact tie for every ambiguous
    # ReLU with lambda > 0, and (r - g) * u is then a cancellation whose
    # rounding error scales with |r| + |g|; rounding must not decide it.
    margin = TIE_REL * (np.abs(r) + np.abs(c)) * np.maximum(np.abs(l), np.abs(u))
    take = v_uu < best - margin
    choice[take] = 2
    xb_amb = np.select([choice == 0, choice == 1], [l, np.zeros_like(l)], u)
    xk_amb = np.where(choice == 2, u, 0.0)
    xb[amb] = xb_amb[amb]
    xk[amb] = xk_amb[amb]
    code[amb] = choice[amb]
    return xb, xk, code


def inner_minimisation(net: Net, l0, u0, lb, ub, rho, passes=None, ball_eps=None) -> InnerSolution:
    """Solve the decomposed inner problem of Eq. (nonprox_problem) at rho.

    l0, u0 [B, n_0]; lb, ub lists 1..n-1 of [B, n_k] (clamped); rho list 1..n-1.
    Vertex codes: 0 -> (l,0) / lower endpoint, 1 -> (0,0), 2 -> (u,u) / upper.
    `passes` supplies the linear passes (default: exact FP64, ExactPasses);
    q is always computed from the g of those passes.  ball_eps [B]: the
    input domain is the l2 ball of that radius around l0 (Sec. 3.2.1) instead
    of the box [l0, u0].
    """
    n = net.n
    B = l0.shape[0]
    ps = ExactPasses(net) if passes is None else passes
    g = [None] * n
    for k in range(n):
        rho_next = -np.ones((B, 1)) if k + 1 == n else rho[k + 1]
        g[k] = ps.transposed(k + 1, rho_next)

    # P0 (Sec. 3.2.1): minimise -g_0^T x0 over the input domain: the box
    # (Eq. (box_bounds_sol)) or the l2 ball
    if ball_eps is None:
        x = [box_argmin(-g[0], l0, u0)]
    else:
        from .l2 import ball_argmin
        x = [ball_argmin(g[0], l0, ball_eps)]
    xB = [None]
    vertex = [None]
    # Pk (Sec. 3.2.2): minimise rho_k x_hat_B,k - g_k x_k over the ReLU hull.
    for k in range(1, n):
        xb, xk, code = relu_subproblem_argmin(rho[k], g[k], lb[k], ub[k])
        x.append(xk)
        xB.append(xb)
        vertex.append(code)

    xA = [None] + [ps.forward(k, x[k - 1]) for k in range(1, n + 1)]
    # Lagrangian of Eq. (nonprox_problem) at the returned primal point
    q_point = xA[n][:, 0].copy()
    for k in range(1, n):
        q_point += np.sum(rho[k] * (xB[k] - xA[k]), axis=1)
    # q itself from the exact per-subproblem minima (App. A, Eq.
    # (dual_decomp_vs_dj)): the tie margins above may return a vertex whose
    # value exceeds the minimum by at most the margin, so q is not read off
    # the returned point.
    if ball_eps is None:
        q = np.sum(np.minimum(-g[0] * l0, -g[0] * u0), axis=1) + net.L(n).bias_vector()[0]
    else:
        from .l2 import ball_min
        q = ball_min(g[0], l0, ball_eps) + net.L(n).bias_vector()[0]
    for k in range(1, n):
        r, c, l, u = rho[k], g[k], lb[k], ub[k]
        cls = classify(l, u)
        m_blk = np.minimum(r * l, r * u)
        m_pas = np.minimum((r - c) * l, (r - c) * u)
        m_amb = np.minimum(np.minimum(r * l, 0.0), (r - c) * u)
        q += np.sum(np.select([cls == 0, cls == 1], [m_blk, m_pas], m_amb), axis=1)
        q -= rho[k] @ net.L(k).bias_vector()
    return InnerSolution(q=q, g=g, x=x, xB=xB, xA=xA, vertex=vertex, q_point=q_point)


def dual_value(net, l0, u0, lb, ub, rho, ball_eps=None):
    """q(rho) of Eq. (nonprox_problem); any rho gives a valid lower bound."""
    return inner_minimisation(net, l0, u0, lb, ub, rho, ball_eps=ball_eps).q


def supergradient(sol: InnerSolution):
    """nabla q = x_hat_B^* - x_hat_A^* (Algorithm 1, Sec. 3.2), layers 1..n-1."""
    return [None] + [sol.xB[k] - sol.xA[k] for k in range(1, len(sol.xB))]


# --------------------------------------------------------------------------
# BF16 operands (the precision of the tensor-core passes)
# --------------------------------------------------------------------------

def round_bf16(a):
    """Nearest bfloat16 value (ties to even) of each element, via its float32
    value: keep the top 16 bits of the float32 encoding after adding half an
    ulp of the kept part (0x7FFF plus the lowest kept bit)."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


class BF16Passes:
    """Linear passes with BF16 operands and exact accumulation: the weights of
    layers 1..n-1 and the vectors they multiply (rho_k in the transposed pass,
    x_{k-1} in the forward pass) rounded to bfloat16.  Layer n is exact (its
    transposed pass is g_{n-1} = -W_n, no product is formed).  The box enters
    the forward pass of layer 1 as x_0 = c_0 + delta_0 with c_0 = l_0 +
    (u_0 - l_0)/2 exact and only delta_0 = x_0 - c_0 rounded, so that the box
    width survives the rounding."""

    def __init__(self, net: Net, l0, u0):
        self.net = net
        self.rounded = {}
        for k in range(1, net.n):
            lay = net.L(k)
            Wr = round_bf16(lay.W)
            self.rounded[k] = Layer(lay.kind, Wr, np.zeros_like(lay.b), lay.in_shape, lay.stride, lay.pad)
        self.c0 = l0 + (u0 - l0) / 2
        self.c1 = net.L(1).forward(self.c0)

    def transposed(self, k: int, r):
        if k == self.net.n:
            return self.net.L(k).transposed(r)
        return self.rounded[k].transposed(round_bf16(r))

    def forward(self, k: int, x):
        if k == self.net.n:
            return self.net.L(k).forward(x)
        if k == 1:
            return self.c1 + self.rounded[1].linear(round_bf16(x - self.c0))
        return self.rounded[k].linear(round_bf16(x)) + self.net.L(k).bias_vector()[None, :]


class FP32Passes:
    """Linear passes with float32 operands, products and sums: an emulation
    of an FP32 evaluation of the method, used by the tests to measure how far
    the Adam trajectory moves when only the rounding of the passes changes
    (the device kernels sum in other orders; this is a model of their
    precision, not of their arithmetic).  Every layer is held as a float32
    sparse matrix, so the sums run in a fixed order on every machine."""

    def __init__(self, net: Net):
        self.net = net
        self.mats = {k: sp.csr_matrix(net.L(k).mat, dtype=np.float32) for k in range(1, net.n + 1)}
        self.tmats = {k: sp.csr_matrix(self.mats[k].T) for k in range(1, net.n + 1)}
        self.bias = {k: net.L(k).bias_vector().astype(np.float32) for k in range(1, net.n + 1)}

    def transposed(self, k: int, r):
        out = self.tmats[k] @ np.asarray(r, np.float32).T
        return np.asarray(out, dtype=np.float32).T.astype(np.float64)

    def forward(self, k: int, x):
        out = np.asarray(self.mats[k] @ np.asarray(x, np.float32).T, dtype=np.float32).T
        return (out + self.bias[k][None, :]).astype(np.float64)


# --------------------------------------------------------------------------
# Dual initialisation (Prop. 3) and the propagation bound
# --------------------------------------------------------------------------

def crown_slopes(l, u):
    """Upper slope a_bar and lower slope a_low of the CROWN relaxation.

    Eq. (slopes-biases): ambiguous a_bar = u/(u-l); blocking 0/0; passing 1/1.
    CROWN's lower slope (footnote of Sec. 4.2) for ambiguous ReLUs: 1 if
    u >= -l else 0.  Returns (a_bar, a_low, b_bar) with b_bar = -l*u/(u-l) on
    ambiguous ReLUs and 0 elsewhere.
    """
    cls = classify(l, u)
    amb = cls == 2
    den = np.where(amb, u - l, 1.0)
    a_bar = np.where(cls == 1, 1.0, 0.0)
    a_bar = np.where(amb, u / den, a_bar)
    a_low = np.where(cls == 1, 1.0, 0.0)
    a_low = np.where(amb, (u >= -l).astype(np.float64), a_low)
    b_bar = np.where(amb, -l * u / den, 0.0)
    return a_bar, a_low, b_bar


def crown_init(net: Net, lb, ub, passes=None):
    """rho^0 = mu_bar of Eq. (salman-assignment), Prop. 3 (one backward pass).

    lambda_{n-1} = -W_n^T 1; mu_k = a_bar*[lambda_k]_+ + a_low*[lambda_k]_-;
    lambda_{k-1} = W_k^T mu_k.  Returns (rho list 1..n-1, lambda list 1..n-1).
    `passes` supplies the transposed products (default exact); the iterations
    must use the same ones, or the exact (l,0)/(u,u) ties that Prop. 3 puts
    at rho^0 are broken by the difference between the two.
    """
    n = net.n
    B = lb[1].shape[0]
    ps = ExactPasses(net) if passes is None else passes
    rho = [None] * n
    lam = [None] * n
    lam_k = ps.transposed(n, -np.ones((B, 1)))
    for k in range(n - 1, 0, -1):
        lam[k] = lam_k
        a_bar, a_low, _ = crown_slopes(lb[k], ub[k])
        rho[k] = a_bar * np.maximum(lam_k, 0.0) + a_low * np.minimum(lam_k, 0.0)
        if k >= 2:
            lam_k = ps.transposed(k, rho[k])
    return rho, lam


def propagation_bound(net: Net, l0, u0, lb, ub, mu, lam):
    """Closed form Eq. (bounds-propagation) of the propagation dual at (mu, lambda).

    min_{x0 in box}(-mu_1^T W_1 x0) + b_n - sum_k([lambda_k]_+^T b_bar_k + mu_k^T b_k)
    (the lower relaxation has zero bias, Eq. (slopes-biases)).
    """
    n = net.n
    c0 = net.L(1).transposed(mu[1])              # W_1^T mu_1
    val = np.sum(np.minimum(-c0 * l0, -c0 * u0), axis=1)
    val = val + net.L(n).bias_vector()[0]
    for k in range(1, n):
        _, _, b_bar = crown_slopes(lb[k], ub[k])
        val = val - np.sum(np.maximum(lam[k], 0.0) * b_bar, axis=1)
        val = val - mu[k] @ net.L(k).bias_vector()
    return val


# --------------------------------------------------------------------------
# Algorithm 1: supergradient ascent with Adam
# --------------------------------------------------------------------------

@dataclass
class AdamSettings:
    """Hyper-parameters of the Adam ascent (Sec. 7.2: step size decreased
    linearly from alpha0 to alpha_end; Adam moments as Kingma & Ba)."""
    alpha0: float = 1e-2
    alpha_end: float = 1e-4
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8


def step_size(t: int, T: int, s: AdamSettings) -> float:
    """alpha_t decreased linearly over t = 0..T-1 (Sec. 7.2)."""
    return s.alpha0 + (s.alpha_end - s.alpha0) * t / max(T - 1, 1)


def adam_update(rho, m, v, sg, tt: int, Ts: int, s: AdamSettings):
    """One Adam ascent step of one layer at schedule index tt of Ts (Algorithm 1
    with Adam in place of Eq. (subgradient_update); bias corrections with step
    count tt + 1, step size of the linear schedule of Sec. 7.2):
        m <- b1 m + (1-b1) s;  v <- b2 v + (1-b2) s^2
        rho <- rho + alpha_tt * (m / (1-b1^(tt+1))) / (sqrt(v / (1-b2^(tt+1))) + eps)
    Returns the new (rho, m, v)."""
    alpha = step_size(tt, Ts, s)
    bc1 = 1.0 - s.beta1 ** (tt + 1)
    bc2 = 1.0 - s.beta2 ** (tt + 1)
    m = s.beta1 * m + (1.0 - s.beta1) * sg
    v = s.beta2 * v + (1.0 - s.beta2) * sg ** 2
    rho = rho + alpha * (m / bc1) / (np.sqrt(v / bc2) + s.eps)
    return rho, m, v


@dataclass
class AdamResult:
    rho: list
    m: list
    v: list
    q_trace: np.ndarray    # [T, B]: q(rho^t), t = 0..T-1
    q_final: np.ndarray    # [B]: q(rho^T)


def supergradient_adam(net, l0, u0, lb, ub, rho0, T, s: AdamSettings = AdamSettings(),
                       m0=None, v0=None, t0: int = 0, T_sched: int | None = None, passes=None, ball_eps=None):
    """Algorithm 1 with the Adam update in place of Eq. (subgradient_update).

    For t = 0..T-1: inner minimisation at rho^t, supergradient
    x_hat_B - x_hat_A, then
        m <- b1 m + (1-b1) s;  v <- b2 v + (1-b2) s^2
        rho <- rho + alpha_t * (m / (1-b1^(t+1))) / (sqrt(v / (1-b2^(t+1))) + eps)
    and finally q(rho^T).  `t0`, `m0`, `v0`, `T_sched` resume a run that was
    split across calls (the schedule index is t0 + t out of T_sched).
    `passes` replaces the linear passes of the iterations (not of the final
    q(rho^T), which is always exact).  ball_eps: l2-ball input domain
    (inner_minimisation).
    """
    n = net.n
    rho = [None] + [np.array(rho0[k], dtype=np.float64, copy=True) for k in range(1, n)]
    m = [None] + [np.zeros_like(rho[k]) if m0 is None else np.array(m0[k], np.float64) for k in range(1, n)]
    v = [None] + [np.zeros_like(rho[k]) if v0 is None else np.array(v0[k], np.float64) for k in range(1, n)]
    Ts = T if T_sched is None else T_sched
    trace = []
    for t in range(T):
        tt = t0 + t
        sol = inner_minimisation(net, l0, u0, lb, ub, rho, passes, ball_eps=ball_eps)
        trace.append(sol.q)
        sg = supergradient(sol)
        for k in range(1, n):
            rho[k], m[k], v[k] = adam_update(rho[k], m[k], v[k], sg[k], tt, Ts, s)
    q_final = inner_minimisation(net, l0, u0, lb, ub, rho, ball_eps=ball_eps).q
    q_trace = np.array(trace) if trace else np.zeros((0, l0.shape[0]))
    return AdamResult(rho=rho, m=m, v=v, q_trace=q_trace, q_final=q_final)


# --------------------------------------------------------------------------
# Batched driver: properties, subdomains, masks
# --------------------------------------------------------------------------

def expand_per_subdomain(x, prop_of_subdomain):
    """Row i of the result is row prop_of_subdomain[i] of x."""
    return np.asarray(x)[np.asarray(prop_of_subdomain)]


def layer_lists(net, flat):
    """Flat [P, sum n_k] (layers 1..n-1) -> list indexed 1..n-1."""
    offs = split_offsets(net)
    return [None] + [flat[:, offs[k - 1]:offs[k]] for k in range(1, net.n)]


def flatten_layers(net, lst):
    return np.concatenate([lst[k] for k in range(1, net.n)], axis=1)


def ld_bound(net: Net, l0, u0, lbk, ubk, prop_of_subdomain, masks, T,
             s: AdamSettings = AdamSettings(), init: str = "crown", rho_in=None, operands: str = "fp64",
             ball_eps=None):
    """Lower bound of min x_hat_n for each subdomain after T Adam updates.

    l0, u0 [P, n_0]; lbk, ubk [P, sum n_k] intermediate bounds of layers
    1..n-1; masks int8 [B, sum n_k].  Empty subdomains get +inf and no
    iterations.  operands "bf16" runs the iterations with BF16Passes (the
    final bound stays exact).  ball_eps [P]: the input domain of property p
    is the l2 ball of radius ball_eps[p] around l0[p] (Sec. 3.2.1; u0 is then
    not used).  Returns (bounds [B], AdamResult over the feasible rows,
    feasible-row index array).
    """
    B = masks.shape[0]
    pos = np.zeros(B, dtype=np.int64) if prop_of_subdomain is None else np.asarray(prop_of_subdomain)
    L0 = expand_per_subdomain(l0, pos)
    U0 = expand_per_subdomain(u0, pos)
    lb = layer_lists(net, expand_per_subdomain(lbk, pos))
    ub = layer_lists(net, expand_per_subdomain(ubk, pos))
    lb, ub, empty = apply_masks(net, lb, ub, masks)
    keep = np.nonzero(~empty)[0]
    out = np.full(B, np.inf)
    if keep.size == 0:
        return out, None, keep
    sel = lambda lst: [None] + [lst[k][keep] for k in range(1, net.n)]
    lbs, ubs = sel(lb), sel(ub)
    if rho_in is not None:
        rho0 = sel(layer_lists(net, np.asarray(rho_in, np.float64)))
    elif init == "crown":
        rho0, _ = crown_init(net, lbs, ubs,
                             BF16Passes(net, L0[keep], U0[keep]) if operands == "bf16" else None)
    elif init == "zero":
        rho0 = [None] + [np.zeros_like(lbs[k]) for k in range(1, net.n)]
    else:
        raise ValueError(init)
    passes = None
    if operands == "bf16":
        passes = BF16Passes(net, L0[keep], U0[keep])
    elif operands != "fp64":
        raise ValueError(operands)
    eps = None if ball_eps is None else expand_per_subdomain(np.asarray(ball_eps, np.float64), pos)[keep]
    res = supergradient_adam(net, L0[keep], U0[keep], lbs, ubs, rho0, T, s, passes=passes, ball_eps=eps)
    out[keep] = res.q_final
    return out, res, keep


# --------------------------------------------------------------------------
# Danskin gradients of q(rho) at fixed rho
# --------------------------------------------------------------------------

@dataclass
class DualGradients:
    gW: list   # index 1..n, same shape as Layer.W
    gb: list   # index 1..n, same shape as Layer.b
    gl0: np.ndarray
    gu0: np.ndarray
    glb: list  # index 1..n-1 (w.r.t. the clamped-and-used bounds' inputs)
    gub: list


def conv_weight_grad(lay: Layer, out_grad, x_in):
    """d/dW of sum_b out_grad[b]^T (W conv x_in[b]) for a conv layer, tap by tap."""
    cout, cin, kh, kw = lay.W.shape
    c, h, w = lay.in_shape
    _, ho, wo = conv_out_shape(lay.in_shape, lay.W, lay.stride, lay.pad)
    G = np.zeros_like(lay.W)
    og = out_grad.reshape(-1, cout, ho, wo)
    xi = x_in.reshape(-1, cin, h, w)
    xp = np.zeros((xi.shape[0], cin, h + 2 * lay.pad + lay.stride * kh, w + 2 * lay.pad + lay.stride * kw))
    xp[:, :, lay.pad:lay.pad + h, lay.pad:lay.pad + w] = xi
    for i in range(kh):
        for j in range(kw):
            patch = xp[:, :, i:i + lay.stride * ho:lay.stride, j:j + lay.stride * wo:lay.stride]
            G[:, :, i, j] = np.einsum("boyx,bcyx->oc", og, patch)
    return G


def danskin_gradients(net: Net, l0, u0, lb, ub, masks_clamp_info, rho, grad_out):
    """Gradient of sum_b grad_out[b] * q_b(rho_b) w.r.t. W, b, box and the
    (unclamped) intermediate bounds, holding rho fixed (Danskin's theorem).

    Writing x_hat_A,k = W_k x_{k-1} + b_k in the Lagrangian of Eq.
    (nonprox_problem) with rho_n = -1:
        dq/db_k = -rho_k,  dq/dW_k = -rho_k x_{k-1}^{*T}
        dq/dl0  = -g_0 where x0* = l0, dq/du0 = -g_0 where x0* = u0
    and for layer k, the bound that the chosen vertex sits on receives the
    coefficient of x_hat_B,k in its subproblem (rho for the (l,0) vertex and
    blocking ReLUs, rho - g for the (u,u) vertex and passing ReLUs).  A bound
    clamped by a split mask (l <- max(l,0) with l < 0, u <- min(u,0) with u > 0)
    passes no gradient to its input.

    masks_clamp_info: list 1..n-1 of (lower_clamped, upper_clamped) booleans.
    """
    n = net.n
    sol = inner_minimisation(net, l0, u0, lb, ub, rho)
    w = np.asarray(grad_out, np.float64)[:, None]
    coef = [None] + [-w * rho[k] for k in range(1, n)] + [w * np.ones((l0.shape[0], 1))]
    gW, gb = [None], [None]
    for k in range(1, n + 1):
        lay = net.L(k)
        if lay.kind == "fc":
            gW.append(coef[k].T @ sol.x[k - 1])
            gb.append(coef[k].sum(axis=0))
        else:
            gW.append(conv_weight_grad(lay, coef[k], sol.x[k - 1]))
            cout = lay.W.shape[0]
            gb.append(coef[k].reshape(coef[k].shape[0], cout, -1).sum(axis=(0, 2)))
    # x0* = u0 where -g_0 <= 0 (Eq. (box_bounds_sol)), l0 elsewhere
    at_u = sol.g[0] >= 0
    gl0 = -w * sol.g[0] * ~at_u
    gu0 = -w * sol.g[0] * at_u
    glb, gub = [None], [None]
    for k in range(1, n):
        r, c = rho[k], sol.g[k]
        cls = classify(lb[k], ub[k])
        code = sol.vertex[k]
        a = np.where(cls == 1, r - c, r)            # coefficient of x_hat_B in its box
        a = np.where(cls == 2, np.where(code == 2, r - c, r), a)
        on_l = code == 0
        on_u = code == 2
        gl = w * a * on_l
        gu = w * a * on_u
        lo_cl, hi_cl = masks_clamp_info[k]
        glb.append(np.where(lo_cl, 0.0, gl))
        gub.append(np.where(hi_cl, 0.0, gu))
    return DualGradients(gW=gW, gb=gb, gl0=gl0, gu0=gu0, glb=glb, gub=gub)


def clamp_info(net, lb, ub, masks):
    """Which bounds a split mask actually moved (lists 1..n-1 of bool pairs)."""
    offs = split_offsets(net)
    info = [None]
    for k in range(1, net.n):
        m = masks[:, offs[k - 1]:offs[k]]
        info.append(((m > 0) & (lb[k] < 0), (m < 0) & (ub[k] > 0)))
    return info


# --------------------------------------------------------------------------
# FP64 outward slack for a sound final bound
# --------------------------------------------------------------------------

def gamma(K: int) -> float:
    """Higham's a-priori constant gamma_K = K u / (1 - K u), u = 2^-53."""
    u = 2.0 ** -53
    return K * u / (1.0 - K * u)


def net_summary(net: Net):
    """Widths and ReLU count, for reports."""
    w = net.widths
    return {"widths": w, "relus": int(sum(w[1:-1]))}


def relative_gap(a, b):
    """|a - b| / max(|b|, 1) elementwise."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b) / np.maximum(np.abs(b), 1.0)


__all__ = [n for n in dir() if not n.startswith("_") and n not in ("annotations", "math")]
