"""Batched branch and bound over the library's kernels (Sec. 2.3, Sec. 5.2).

Host-side queue management only: the lower bounds (ld_bound, warm-started
from the parent's duals), the upper bounds at the inner minimiser's x0*
(ld_upper_bound, Sec. 5.1.3) and the branching decisions (ld_branch: SR,
mSR or FSB, Sec. 4) all run on the GPU; the subdomains' split masks and duals
stay in device memory.  Each step branches the `batch` subdomains with the
lowest lower bounds and bounds their 2 x batch children at once.  A
subdomain is discarded once its lower bound is positive; the search ends
when none is left (the property min x_hat_n > 0 holds), when an upper bound
is negative (a counterexample), or at the node budget.  Intermediate bounds
stay those of the root, clamped by each subdomain's splits (BaDNB, Sec.
5.1.1).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

from . import binding as ldb


@dataclass
class BaBResult:
    status: str            # "verified", "counterexample" or "budget"
    lower: float           # lowest lower bound among the open subdomains when stopped (0 when verified)
    upper: float           # best upper bound found
    nodes: int             # subdomains bounded
    iterations: int        # branching steps
    trace: list = field(default_factory=list)   # lowest open lower bound after every step


def verify(net: ldb.Net, l0, u0, lbk, ubk, T: int = 50, batch: int = 64, max_nodes: int = 20000,
           branching: str = "fsb", opts: ldb.Options | None = None) -> BaBResult:
    """Decide min x_hat_n > 0 over the box [l0, u0] (one property; lbk, ubk:
    the root's intermediate bounds [1, N]) by batched branch and bound."""
    dev = torch.device("cuda", torch.cuda.current_device())
    l0 = torch.as_tensor(np.asarray(l0, np.float32), device=dev).reshape(1, -1)
    u0 = torch.as_tensor(np.asarray(u0, np.float32), device=dev).reshape(1, -1)
    lbk = torch.as_tensor(lbk, device=dev, dtype=torch.float32).reshape(1, -1)
    ubk = torch.as_tensor(ubk, device=dev, dtype=torch.float32).reshape(1, -1)
    N = net.N
    masks = torch.zeros((1, N), dtype=torch.int8, device=dev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count

    def shape(B, warm):
        # fixed fused launch shapes (the autotuner would probe every new batch
        # size): one subdomain per 512-thread CTA while the batch fits the
        # SMs in one wave, two per CTA beyond that; children start from their
        # parent's duals
        o = opts or ldb.Options(engine="fused", tile=1 if B <= sms else 2, cta_threads=512)
        return ldb.Options(**{**o.__dict__, "init": "given"}) if warm else o

    lo, rho = ldb.ld_bound(net, l0, u0, lbk, ubk, None, masks, n_iters=T, opts=shape(1, False), return_rho=True)
    best_ub = float(ldb.ld_upper_bound(net, l0, u0, lbk, ubk, rho, masks=masks).min().item())
    bounds = lo.cpu().numpy()
    stuck = []
    nodes, it, trace = 1, 0, []
    while True:
        open_ = bounds <= 0.0
        idx = np.nonzero(open_)[0]
        if idx.size < bounds.size:
            keep = torch.as_tensor(idx, device=dev, dtype=torch.long)
            masks, rho, bounds = masks[keep], rho[keep], bounds[idx]
        lowest = min([float(bounds.min())] if bounds.size else [np.inf])
        lowest = min([lowest] + stuck)
        if best_ub < 0.0:
            return BaBResult("counterexample", lowest, best_ub, nodes, it, trace)
        if bounds.size == 0:
            return BaBResult("budget" if stuck else "verified", lowest if stuck else 0.0, best_ub, nodes, it, trace)
        if nodes >= max_nodes:
            return BaBResult("budget", lowest, best_ub, nodes, it, trace)
        order = np.argsort(bounds, kind="stable")
        pick, rest = order[:batch], order[batch:]
        tp = torch.as_tensor(pick, device=dev, dtype=torch.long)
        m, r = masks[tp], rho[tp]
        dec = ldb.ld_branch(net, l0, u0, lbk, ubk, masks=m, rule=branching).cpu().numpy()
        split = np.nonzero(dec >= 0)[0]
        stuck += [float(bounds[pick[i]]) for i in np.nonzero(dec < 0)[0]]
        tr = torch.as_tensor(rest, device=dev, dtype=torch.long)
        masks, rho, bounds = masks[tr], rho[tr], bounds[rest]
        if split.size == 0:
            continue
        ts = torch.as_tensor(split, device=dev, dtype=torch.long)
        col = torch.as_tensor(dec[split], device=dev, dtype=torch.long)
        cm = torch.cat([m[ts], m[ts]])
        rows = torch.arange(2 * split.size, device=dev)
        cm[rows, torch.cat([col, col])] = torch.cat([torch.ones_like(col), -torch.ones_like(col)]).to(torch.int8)
        cr = torch.cat([r[ts], r[ts]])
        co, crho = ldb.ld_bound(net, l0, u0, lbk, ubk, None, cm, n_iters=T, opts=shape(int(cm.shape[0]), True),
                                rho_in=cr, return_rho=True)
        ub = ldb.ld_upper_bound(net, l0, u0, lbk, ubk, crho, masks=cm).cpu().numpy()
        co = co.cpu().numpy()
        fin = np.isfinite(co)
        if fin.any():
            best_ub = min(best_ub, float(ub[fin].min()))
        nodes += int(cm.shape[0])
        it += 1
        tf = torch.as_tensor(np.nonzero(fin)[0], device=dev, dtype=torch.long)
        masks = torch.cat([masks, cm[tf]])
        rho = torch.cat([rho, crho[tf]])
        bounds = np.concatenate([bounds, co[fin]])
        trace.append(float(min([bounds.min()] if bounds.size else [np.inf])))
