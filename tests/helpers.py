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
