"""Seeded synthetic inputs: networks, input boxes, margin vectors, split masks.

This module holds random draws only and none of the bounding arithmetic; the
CUDA path, the tests and the benchmark all take their inputs from here so
that every comparison runs on identical data.

The shapes are those of the paper's CIFAR-10 networks (Table 1: Base, Wide,
Deep) and of a tiny MLP; the trained weights and the OVAL properties are not
available, so weights are Kaiming-normal draws and the image is uniform noise.

Every array is float32 (what the device path consumes); the oracle reads the
same float32 values as float64.  Seeds: weights 1000 + net id, boxes
2000 + property id, masks 3000 + subdomain block (NumPy PCG64).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

NET_IDS = {"tiny": 1, "base": 2, "wide": 3, "deep": 4}


@dataclass
class LayerSpec:
    kind: str                 # "fc" or "conv"
    W: np.ndarray             # fc [out, in]; conv [cout, cin, kh, kw]
    b: np.ndarray             # [out] or [cout]
    in_shape: tuple           # fc (n_in,); conv (cin, h, w)
    stride: int = 1
    pad: int = 0

    @property
    def out_shape(self):
        if self.kind == "fc":
            return (self.W.shape[0],)
        cout, cin, kh, kw = self.W.shape
        _, h, w = self.in_shape
        return (cout, (h + 2 * self.pad - kh) // self.stride + 1,
                (w + 2 * self.pad - kw) // self.stride + 1)

    @property
    def n_in(self):
        return int(np.prod(self.in_shape))

    @property
    def n_out(self):
        return int(np.prod(self.out_shape))


# (cout, k, stride, pad) per conv, then FC widths; input 3x32x32, 10 logits.
ARCHS = {
    "base": ([(8, 4, 2, 1), (16, 4, 2, 1)], [100, 10]),
    "wide": ([(16, 4, 2, 1), (32, 4, 2, 1)], [100, 10]),
    "deep": ([(8, 4, 2, 1), (8, 3, 1, 1), (8, 3, 1, 1), (8, 4, 2, 1)], [100, 10]),
}


def make_convnet(name: str, seed: int | None = None):
    """CIFAR-shaped convnet with Kaiming weights N(0, 2/fan_in) and biases
    U(-1/sqrt(fan_in), 1/sqrt(fan_in)).  Returns a list of LayerSpec whose
    last layer has 10 outputs (fold a margin vector to get canonical form)."""
    convs, fcs = ARCHS[name]
    rng = np.random.Generator(np.random.PCG64(1000 + NET_IDS[name] if seed is None else seed))
    layers = []
    shape = (3, 32, 32)
    for cout, k, s, p in convs:
        cin = shape[0]
        fan_in = cin * k * k
        W = rng.normal(0.0, np.sqrt(2.0 / fan_in), size=(cout, cin, k, k))
        b = rng.uniform(-1 / np.sqrt(fan_in), 1 / np.sqrt(fan_in), size=cout)
        L = LayerSpec("conv", W.astype(np.float32), b.astype(np.float32), shape, s, p)
        layers.append(L)
        shape = L.out_shape
    n_in = int(np.prod(shape))
    for n_out in fcs:
        W = rng.normal(0.0, np.sqrt(2.0 / n_in), size=(n_out, n_in))
        b = rng.uniform(-1 / np.sqrt(n_in), 1 / np.sqrt(n_in), size=n_out)
        layers.append(LayerSpec("fc", W.astype(np.float32), b.astype(np.float32), (n_in,)))
        n_in = n_out
    return layers


def make_mlp(widths, seed: int, bias_std: float = 0.1):
    """FC ReLU net with W ~ N(0, 1/fan_in), b ~ N(0, bias_std^2)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    layers = []
    for a, b in zip(widths[:-1], widths[1:]):
        W = rng.normal(0.0, np.sqrt(1.0 / a), size=(b, a))
        bb = rng.normal(0.0, bias_std, size=b)
        layers.append(LayerSpec("fc", W.astype(np.float32), bb.astype(np.float32), (a,)))
    return layers


def tiny_mlp(i: int = 0):
    """FC 10 -> 20 -> ReLU -> 20 -> ReLU -> 1 (the tiny canonical-form MLP)."""
    return make_mlp([10, 20, 20, 1], seed=1000 + NET_IDS["tiny"] * 100 + i)


def tiny_box(i: int = 0, eps: float = 0.1):
    """Box centre U[-1,1]^10, radius eps."""
    rng = np.random.Generator(np.random.PCG64(2000 + 100 + i))
    c = rng.uniform(-1.0, 1.0, size=10)
    return (c - eps).astype(np.float32)[None, :], (c + eps).astype(np.float32)[None, :]


def image_property(prop: int, eps_range=(1 / 255, 8 / 255), n_classes: int = 10):
    """A synthetic CIFAR-shaped robustness property.

    x ~ U[0,1]^(3x32x32), eps ~ U[eps_range], box [x - eps, x + eps] (no
    clipping to the image range); ground-truth class uniform (a random net
    has no meaningful label), target uniform among the other classes.
    Returns (l0 [3072], u0 [3072], margin c [10]) with c = e_gt - e_target.
    """
    rng = np.random.Generator(np.random.PCG64(2000 + prop))
    x = rng.uniform(0.0, 1.0, size=3 * 32 * 32)
    eps = rng.uniform(*eps_range)
    gt = int(rng.integers(n_classes))
    target = int(rng.integers(n_classes - 1))
    target = target + (target >= gt)
    c = np.zeros(n_classes)
    c[gt] = 1.0
    c[target] = -1.0
    return (x - eps).astype(np.float32), (x + eps).astype(np.float32), c.astype(np.float32)


def split_masks(n_relu: int, B: int, candidates, depth_range=(0, 8), block: int = 0):
    """Random ReLU splits for B subdomains.

    Subdomain 0 is the root (no split).  Every other subdomain draws a depth
    k ~ U{depth_range}, picks k distinct indices from `candidates` (the
    caller's list of ambiguous ReLUs, flat over layers 1..n-1) and a phase +1
    (passing) or -1 (blocking) for each.  Returns int8 [B, n_relu].
    """
    rng = np.random.Generator(np.random.PCG64(3000 + block))
    cand = np.asarray(candidates, dtype=np.int64)
    masks = np.zeros((B, n_relu), dtype=np.int8)
    lo, hi = depth_range
    for i in range(1, B):
        k = int(rng.integers(lo, hi + 1))
        k = min(k, cand.size)
        if k == 0:
            continue
        idx = rng.choice(cand, size=k, replace=False)
        masks[i, idx] = np.where(rng.random(k) < 0.5, 1, -1).astype(np.int8)
    return masks


def random_box_points(l0, u0, count: int, seed: int):
    """Uniform samples inside a box (for weak-duality checks)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    l0 = np.asarray(l0, np.float64)
    u0 = np.asarray(u0, np.float64)
    return l0 + (u0 - l0) * rng.random((count,) + l0.shape)


def random_duals(sizes, B: int, seed: int, scale: float = 1.0):
    """Random dual points rho (float32), one [B, n] array per size."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [(scale * rng.normal(size=(B, n))).astype(np.float32) for n in sizes]
