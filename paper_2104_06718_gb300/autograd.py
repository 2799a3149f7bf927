"""torch.autograd wrapper of the LD bound (forward: ld_bound; backward: the
Danskin adjoint ld_bound_backward at the returned rho, recomputing the inner
argmins instead of storing iterates).

The gradient is that of q(rho_T; theta) with rho_T held fixed (Danskin's
theorem applied to the inner minimum of Eq. (nonprox_problem)); it flows to
the input box, the intermediate bounds and the layer parameters.  The net
handle holds its own copy of the weights: pass the same parameter tensors it
was built from (they route gradients only), and rebuild the handle after
changing their values.  The first call with a set of parameter tensors checks
their values against the handle's weights; later calls check that the
tensors have not been written since (their version counters), so a changed
parameter without a rebuilt handle raises instead of returning stale bounds
and gradients.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as ldb


class StaleParametersError(RuntimeError):
    """The parameter tensors differ from the weights the net handle was built from."""


def check_params(net, params):
    """Raise StaleParametersError unless params (W_1, b_1, ..., W_n, b_n, or a
    prefix of them) hold the weights net was built from (the last layer
    before margin folding)."""
    if not params:
        return
    key = tuple((p.data_ptr(), p._version) for p in params)
    if getattr(net, "_param_key", None) == key:
        return
    expect = []
    for s in net.specs:
        expect += [np.asarray(s.W, np.float32), np.asarray(s.b, np.float32)]
    if len(params) > len(expect):
        raise StaleParametersError(f"{len(params)} parameter tensors for a net of {len(expect)}")
    for i, (p, e) in enumerate(zip(params, expect)):
        t = p.detach()
        if tuple(t.shape) != e.shape or not torch.equal(t.to(device="cpu", dtype=torch.float32),
                                                        torch.from_numpy(np.ascontiguousarray(e))):
            raise StaleParametersError(f"parameter {i} differs from the weights the net handle holds: rebuild the "
                                       "net (binding.Net) after changing its parameters")
    net._param_key = key


class LDBound(torch.autograd.Function):
    """out[b] = LD lower bound of subdomain b (float64 [B]).

    Inputs: net (binding.Net), n_iters, opts (binding.Options or None), prop
    ([B] int or None), masks ([B, N] int8 or None), lb0, ub0 ([P, n0] float32),
    lbk, ubk ([P, N] float32), then the layer parameters W_1, b_1, ..., W_n,
    b_n as built into the net (the last layer before margin folding).
    """

    @staticmethod
    def forward(ctx, net, n_iters, opts, prop, masks, lb0, ub0, lbk, ubk, *params):
        check_params(net, params)
        out, rho = ldb.ld_bound(net, lb0, ub0, lbk, ubk, prop, masks, n_iters=n_iters, opts=opts, return_rho=True)
        ctx.net = net
        ctx.prop = prop
        ctx.masks = masks
        ctx.n_params = len(params)
        ctx.save_for_backward(lb0, ub0, lbk, ubk, rho)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        lb0, ub0, lbk, ubk, rho = ctx.saved_tensors
        net = ctx.net
        g = ldb.ld_bound_backward(net, lb0, ub0, lbk, ubk, rho, grad_out=grad_out.contiguous(), prop=ctx.prop,
                                  masks=ctx.masks)
        grads = []
        woff = boff = 0
        n = len(net.specs)
        for k, s in enumerate(net.specs):
            W = np.asarray(s.W)
            if k < n - 1:
                gW = g["gW"][woff:woff + W.size].view(W.shape)
                gb = g["gb"][boff:boff + W.shape[0]]
                woff += W.size
                boff += W.shape[0]
            else:
                # the handle folds the margin c into the last layer: W_n = c^T W, b_n = c^T b
                n_in = W.shape[1]
                gWn = g["gW"][woff:woff + n_in]
                gbn = g["gb"][boff:boff + 1]
                c = torch.ones(1, device=gWn.device) if net.margin is None else \
                    torch.as_tensor(net.margin, device=gWn.device, dtype=torch.float32)
                gW = torch.outer(c, gWn)
                gb = c * gbn
            grads += [gW, gb]
        return (None, None, None, None, None, g["glb0"], g["gub0"], g["glbk"], g["gubk"], *grads[:ctx.n_params])


def bound(net, lb0, ub0, lbk, ubk, params=(), prop=None, masks=None, n_iters: int = 100, opts=None):
    """Differentiable LD lower bounds (float64 [B])."""
    return LDBound.apply(net, n_iters, opts, prop, masks, lb0, ub0, lbk, ubk, *params)
