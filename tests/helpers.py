"""Test helpers: build oracle nets from the synthetic layer specs."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2104_06718_gb300 import synth


def oracle_net(specs, margin=None):
    """LayerSpec list (+ optional margin vector on the last layer) -> oracle Net."""
    layers = []
    for i, s in enumerate(specs):
        W = np.asarray(s.W, np.float64)
        b = np.asarray(s.b, np.float64)
        if i == len(specs) - 1 and margin is not None:
            W, b = oracle.fold_margin(W, b, np.asarray(margin, np.float64))
        if s.kind == "fc":
            layers.append(oracle.Layer("fc", W, b))
        else:
            layers.append(oracle.Layer("conv", W, b, in_shape=tuple(s.in_shape), stride=s.stride, pad=s.pad))
    return oracle.Net(layers)


def folded_specs(specs, margin):
    """Float32 specs with the margin folded into the last layer in float64 and
    rounded once to float32, so that the device and the oracle see one net."""
    out = list(specs[:-1])
    last = specs[-1]
    if margin is not None:
        W, b = oracle.fold_margin(np.asarray(last.W, np.float64), np.asarray(last.b, np.float64),
                                  np.asarray(margin, np.float64))
        last = synth.LayerSpec("fc", W.astype(np.float32), b.astype(np.float32), last.in_shape)
    out.append(last)
    return out


def tiny_problem(i=0):
    specs = synth.tiny_mlp(i)
    net = oracle_net(specs)
    l0, u0 = synth.tiny_box(i)
    lb, ub = oracle.ibp_bounds(net, l0.astype(np.float64), u0.astype(np.float64))
    return specs, net, l0.astype(np.float64), u0.astype(np.float64), lb, ub


def outward_f32(lo, hi):
    """Round float64 bounds to float32 outward (lo down, hi up)."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    l32 = lo.astype(np.float32)
    h32 = hi.astype(np.float32)
    l32 = np.where(l32.astype(np.float64) > lo, np.nextafter(l32, np.float32(-np.inf)), l32)
    h32 = np.where(h32.astype(np.float64) < hi, np.nextafter(h32, np.float32(np.inf)), h32)
    return l32.astype(np.float32), h32.astype(np.float32)


def conv_problem(name, B, depth=(0, 8), props=(0,), block=0, eps_range=(1 / 255, 8 / 255)):
    """Oracle-side synthetic problem on a CIFAR-shaped convnet: folded float32
    specs (margin of property props[0]), oracle net, float32 boxes and
    outward-rounded IBP bounds per property, masks over root-ambiguous ReLUs,
    and subdomain -> property map (contiguous blocks)."""
    specs = synth.make_convnet(name)
    boxes = [synth.image_property(p, eps_range) for p in props]
    fspecs = folded_specs(specs, boxes[0][2])
    net = oracle_net(fspecs)
    l0 = np.stack([b[0] for b in boxes])
    u0 = np.stack([b[1] for b in boxes])
    lb, ub = oracle.ibp_bounds(net, l0.astype(np.float64), u0.astype(np.float64))
    flat_l = np.concatenate([lb[k] for k in range(1, net.n)], axis=1)
    flat_u = np.concatenate([ub[k] for k in range(1, net.n)], axis=1)
    lbk, ubk = outward_f32(flat_l, flat_u)
    P = len(props)
    prop = (np.arange(B) * P // max(B, 1)).astype(np.int32)
    amb = np.nonzero((lbk[0] < 0) & (ubk[0] > 0))[0]
    masks = synth.split_masks(lbk.shape[1], B, amb, depth, block=block)
    return dict(specs=fspecs, net=net, l0=l0, u0=u0, lbk=lbk, ubk=ubk, prop=prop, masks=masks, B=B)


def oracle_lists(net, pb, rows=None):
    """Per-subdomain clamped bound lists and boxes (float64) for the oracle."""
    prop = pb["prop"] if rows is None else pb["prop"][rows]
    masks = pb["masks"] if rows is None else pb["masks"][rows]
    L0 = pb["l0"][prop].astype(np.float64)
    U0 = pb["u0"][prop].astype(np.float64)
    lb = oracle.layer_lists(net, pb["lbk"][prop].astype(np.float64))
    ub = oracle.layer_lists(net, pb["ubk"][prop].astype(np.float64))
    lb, ub, empty = oracle.apply_masks(net, lb, ub, masks)
    return L0, U0, lb, ub, empty


def near_tie_mask(on, L0, U0, lbs, ubs, rho, sol, rel_tol=5e-5):
    """Decisions an FP32 evaluation may legitimately take differently from
    the FP64 oracle: those whose deciding quantity is within rel_tol of its
    threshold, relative to the magnitude of the terms that produce it.
    Returns (box near-ties [B, n0], list of per-layer near-ties 1..n-1)."""
    def absg_of(k):
        nxt = -np.ones((rho[1].shape[0], 1)) if k + 1 == on.n else rho[k + 1]
        return np.asarray((abs(on.L(k + 1).mat).T @ np.abs(nxt).T).T)
    box = np.abs(sol.g[0]) < rel_tol * (absg_of(0) + 1e-30)
    ties = [None]
    for k in range(1, on.n):
        r, g, l, u = rho[k], sol.g[k], lbs[k], ubs[k]
        absg = absg_of(k)
        mag = (np.abs(r) + absg + 1e-30) * (np.maximum(np.abs(l), np.abs(u)) + 1e-30)
        cls = oracle.classify(l, u)
        best0 = np.minimum(r * l, 0.0)
        vuu = (r - g) * u
        gap = best0 - oracle.TIE_REL * (np.abs(r) + np.abs(g)) * np.maximum(np.abs(l), np.abs(u)) - vuu
        amb_tie = np.abs(gap) < rel_tol * mag
        pas_tie = np.abs(r - g) < rel_tol * (np.abs(r) + absg + 1e-30)
        ties.append(np.where(cls == 2, amb_tie, np.where(cls == 1, pas_tie, False)))
    return box, ties
