"""torch.autograd wrapper and CUDA-graph capture of the bound."""
import dataclasses

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


def test_deep_128_backward_matches_finite_differences():
    """Deep convnet, 128 subdomains: the Danskin gradients of the summed FP64
    bound at a fixed rho (the autograd backward, recomputing the argmins)
    against central differences of the bound, for conv and FC weights,
    biases and the input box."""
    pb = conv_problem("deep", 128, depth=(0, 8), block=24)
    specs = pb["specs"]
    net = ldb.Net(specs)
    args = (pb["l0"], pb["u0"], pb["lbk"], pb["ubk"], pb["prop"], pb["masks"])
    _, rho = ldb.ld_bound(net, *args, n_iters=40, return_rho=True)
    # autograd over the weights and the box, at the rho of this run
    params = _params(specs)
    lb0 = torch.tensor(pb["l0"], device="cuda", requires_grad=True)
    ub0 = torch.tensor(pb["u0"], device="cuda", requires_grad=True)
    q0 = ldb.ld_bound(net, *args, n_iters=0, rho_in=rho).cpu().numpy()
    fin = np.isfinite(q0)
    g = ldb.ld_bound_backward(net, pb["l0"], pb["u0"], pb["lbk"], pb["ubk"], rho, prop=pb["prop"], masks=pb["masks"])
    woff = np.cumsum([0] + [s.W.size for s in specs])
    boff = np.cumsum([0] + [s.b.size for s in specs])

    def q_sum(specs2=None, l0=None, u0=None):
        n2 = net if specs2 is None else ldb.Net(specs2)
        a = (pb["l0"] if l0 is None else l0, pb["u0"] if u0 is None else u0) + args[2:]
        q = ldb.ld_bound(n2, *a, n_iters=0, rho_in=rho).cpu().numpy()
        assert np.array_equal(np.isfinite(q), fin)
        return q[fin].sum()

    def copy_specs():
        return [synth.LayerSpec(s.kind, s.W.copy(), s.b.copy(), s.in_shape, s.stride, s.pad) for s in specs]

    h = 1e-3
    checks = 0
    # weights: conv 3->8 (k4s2), conv 8->8 (k3s1), FC 512->100; biases of the conv layers
    for k, idx in [(0, (2, 1, 3, 0)), (2, (5, 7, 1, 2)), (4, (17, 300)), (1, None), (3, None)]:
        what = "W" if idx is not None else "b"
        vals = []
        for sgn in (1, -1):
            sp = copy_specs()
            if what == "W":
                sp[k].W[idx] += sgn * h
            else:
                sp[k].b[3] += sgn * h
            vals.append(q_sum(sp))
        fd = (vals[0] - vals[1]) / (2 * h)
        if what == "W":
            ad = g["gW"][woff[k] + np.ravel_multi_index(idx, specs[k].W.shape)].item()
        else:
            ad = g["gb"][boff[k] + 3].item()
        assert abs(fd - ad) < 1e-3 * max(1.0, abs(fd)), (k, what, fd, ad)
        checks += 1
    # the input box: pixels whose box argmin sits at the lower or the upper end
    for j in (5, 1000, 2500):
        for which in ("l0", "u0"):
            vals = []
            for sgn in (1, -1):
                l0, u0 = pb["l0"].copy(), pb["u0"].copy()
                (l0 if which == "l0" else u0)[:, j] += sgn * h
                vals.append(q_sum(l0=l0, u0=u0))
            fd = (vals[0] - vals[1]) / (2 * h)
            ad = g["glb0" if which == "l0" else "gub0"][:, j].sum().item()
            assert abs(fd - ad) < 1e-3 * max(1.0, abs(fd)), (which, j, fd, ad)
            checks += 1
    assert checks == 11
    del q0
    # the autograd Function gives the same gradients for the box and the weights
    out = lda.bound(net, lb0, ub0, torch.tensor(pb["lbk"], device="cuda"), torch.tensor(pb["ubk"], device="cuda"),
                    params, masks=pb["masks"], prop=pb["prop"], n_iters=40)
    out[torch.isfinite(out)].sum().backward()
    assert torch.allclose(lb0.grad, g["glb0"], rtol=1e-5, atol=1e-6)
    assert torch.allclose(ub0.grad, g["gub0"], rtol=1e-5, atol=1e-6)
    assert torch.allclose(params[2].grad.flatten(), g["gW"][woff[1]:woff[2]], rtol=1e-5, atol=1e-6)


def test_changed_parameters_without_a_rebuilt_net_raise():
    """The handle keeps its own weight copy: parameters changed in place after
    the net was built must not give silently stale bounds and gradients."""
    specs = synth.make_convnet("base")
    l0, u0, c = synth.image_property(2)
    net = ldb.Net(specs, margin=c)
    l0 = torch.tensor(l0[None], device="cuda")
    u0 = torch.tensor(u0[None], device="cuda")
    lbk, ubk = ldb.ld_intermediate_bounds(net, l0, u0)
    params = _params(specs)
    out = lda.bound(net, l0, u0, lbk, ubk, params, n_iters=3)
    assert torch.isfinite(out).all()
    with torch.no_grad():
        params[2].mul_(1.01)          # conv2 weights updated in place (e.g. an optimiser step)
    with pytest.raises(lda.StaleParametersError):
        lda.bound(net, l0, u0, lbk, ubk, params, n_iters=3)
    wrong = _params(specs)
    with torch.no_grad():
        wrong[0].add_(1.0)
    with pytest.raises(lda.StaleParametersError):
        lda.bound(ldb.Net(specs, margin=c), l0, u0, lbk, ubk, wrong, n_iters=3)
    # a rebuilt net with the new values is accepted
    specs2 = [dataclasses.replace(s, W=p.detach().cpu().numpy(), b=q.detach().cpu().numpy())
              for s, p, q in zip(specs, params[0::2], params[1::2])]
    net2 = ldb.Net(specs2, margin=c)
    out2 = lda.bound(net2, l0, u0, lbk, ubk, params, n_iters=3)
    assert torch.isfinite(out2).all()
