"""torch.autograd wrapper and CUDA-graph capture of the bound."""
import numpy as np
import pytest
import torch

from paper_2104_06718_gb300 import autograd as lda
from paper_2104_06718_gb300 import binding as ldb
from paper_2104_06718_gb300 import synth
from helpers import conv_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_06718_gb300 import build
    build.build()
    ldb.load_library()


def _params(specs):
    ps = []
    for s in specs:
        ps.append(torch.tensor(np.asarray(s.W), device="cuda", requires_grad=True))
        ps.append(torch.tensor(np.asarray(s.b), device="cuda", requires_grad=True))
    return ps


def test_autograd_matches_direct_adjoint_and_margin_chain_rule():
    specs = synth.make_convnet("base")
    l0, u0, c = synth.image_property(2)
    net = ldb.Net(specs, margin=c)
    lbk, ubk = ldb.ld_intermediate_bounds(net, l0[None], u0[None])
    B = 6
    amb = np.nonzero((lbk[0] < 0).cpu().numpy() & (ubk[0] > 0).cpu().numpy())[0]
    masks = synth.split_masks(net.N, B, amb, (0, 4), block=21)
    lb0 = torch.tensor(l0[None], device="cuda", requires_grad=True)
    ub0 = torch.tensor(u0[None], device="cuda", requires_grad=True)
    lk = lbk.clone().requires_grad_(True)
    uk = ubk.clone().requires_grad_(True)
    params = _params(specs)
    w = torch.linspace(0.5, 1.5, B, device="cuda", dtype=torch.float64)
    out = lda.bound(net, lb0, ub0, lk, uk, params, masks=masks, n_iters=20)
    (out * w).sum().backward()
    # the same adjoint called directly at the same rho
    _, rho = ldb.ld_bound(net, lb0.detach(), ub0.detach(), lbk, ubk, None, masks, n_iters=20, return_rho=True)
    g = ldb.ld_bound_backward(net, lb0.detach(), ub0.detach(), lbk, ubk, rho, grad_out=w, masks=masks)
    assert torch.allclose(lb0.grad, g["glb0"]) and torch.allclose(ub0.grad, g["gub0"])
    assert torch.allclose(lk.grad, g["glbk"]) and torch.allclose(uk.grad, g["gubk"])
    off = 0
    for k in range(len(specs) - 1):
        n = params[2 * k].numel()
        assert torch.allclose(params[2 * k].grad.flatten(), g["gW"][off:off + n])
        off += n
    gWn = g["gW"][off:off + params[-2].shape[1]]
    cc = torch.tensor(c, device="cuda")
    assert torch.allclose(params[-2].grad, torch.outer(cc, gWn))
    assert torch.allclose(params[-1].grad, cc * g["gb"][-1])


def test_danskin_gradient_matches_finite_differences_of_the_bound():
    """d/db of the FP64 bound at a fixed rho (ld_bound with init=given and no
    iterations) equals the adjoint, bias by bias of the first FC layer."""
    pb = conv_problem("base", 4, depth=(0, 4), block=22)
    net = ldb.Net(pb["specs"])
    args = (pb["l0"], pb["u0"], pb["lbk"], pb["ubk"], pb["prop"], pb["masks"])
    _, rho = ldb.ld_bound(net, *args, n_iters=15, return_rho=True)
    g = ldb.ld_bound_backward(net, pb["l0"], pb["u0"], pb["lbk"], pb["ubk"], rho, prop=pb["prop"], masks=pb["masks"])
    k = 2  # FC 1024 -> 100
    boff = sum(pb["specs"][i].W.shape[0] for i in range(k))
    h = 1e-3
    for o in (0, 17, 63):
        vals = []
        for sgn in (1, -1):
            specs = [synth.LayerSpec(s.kind, s.W.copy(), s.b.copy(), s.in_shape, s.stride, s.pad) for s in pb["specs"]]
            specs[k].b[o] += sgn * h
            q = ldb.ld_bound(ldb.Net(specs), *args, n_iters=0, rho_in=rho).cpu().numpy()
            vals.append(q[np.isfinite(q)].sum())
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - g["gb"][boff + o].item()) < 1e-3 * max(1.0, abs(fd))


def test_bound_captures_in_a_cuda_graph():
    pb = conv_problem("base", 32, depth=(0, 8), block=23)
    net = ldb.Net(pb["specs"])
    B = pb["B"]
    net.reserve(B)
    dev = torch.device("cuda")
    l0 = torch.tensor(pb["l0"], device=dev)
    u0 = torch.tensor(pb["u0"], device=dev)
    lk = torch.tensor(pb["lbk"], device=dev)
    uk = torch.tensor(pb["ubk"], device=dev)
    masks = torch.tensor(pb["masks"], device=dev)
    ref = ldb.ld_bound(net, l0, u0, lk, uk, None, masks, n_iters=30)  # first call: autotune outside capture
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        ldb.ld_bound(net, l0, u0, lk, uk, None, masks, n_iters=30)  # warm the side stream
    torch.cuda.current_stream().wait_stream(s)
    with torch.cuda.graph(graph):
        out = ldb.ld_bound(net, l0, u0, lk, uk, None, masks, n_iters=30)
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
