"""Edge cases through the C ABI: empty batches, ragged batches that leave
the last fused CTA or tensor-core tile partly filled, and the batch limit."""
import numpy as np
import pytest
import torch

import oracle
from paper_2104_06718_gb300 import binding as ldb
from helpers import conv_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_06718_gb300 import build
    build.build()
    ldb.load_library()


def rel(a, b):
    return np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)) / np.maximum(np.abs(np.asarray(b, np.float64)), 1.0)


OPTS = {"layerwise": ldb.Options(engine="layerwise"), "fused2": ldb.Options(engine="fused", tile=2),
        "fused4": ldb.Options(engine="fused", tile=4), "fused2w": ldb.Options(engine="fused", tile=2, cta_threads=512),
        "auto": ldb.Options(), "bf16": ldb.Options(precision="bf16")}


@pytest.mark.parametrize("opt", sorted(OPTS))
def test_empty_batch(opt):
    pb = conv_problem("base", 4, block=30)
    net = ldb.Net(pb["specs"])
    masks = np.zeros((0, pb["lbk"].shape[1]), np.int8)
    out, rho = ldb.ld_bound(net, pb["l0"], pb["u0"], pb["lbk"], pb["ubk"], np.zeros(0, np.int32), masks, n_iters=5,
                            opts=OPTS[opt], B=0, return_rho=True)
    assert out.shape == (0,) and rho.shape == (0, net.N)
    lk, uk = ldb.ld_intermediate_bounds_split(net, pb["l0"], pb["u0"], masks)
    assert lk.shape == (0, net.N)
    assert net.sync_status() == ldb.LD_OK


@pytest.mark.parametrize("opt", ["fused2", "fused4", "fused2w", "layerwise", "bf16"])
@pytest.mark.parametrize("name", ["base", "deep"])
def test_ragged_batch_matches_oracle(name, opt):
    """B = 7: the last CTA of every fused shape and the last tensor-core tiles
    hold fewer subdomains than they could."""
    pb = conv_problem(name, 7, depth=(0, 8), block=31)
    net = ldb.Net(pb["specs"])
    T = 3
    out = ldb.ld_bound(net, pb["l0"], pb["u0"], pb["lbk"], pb["ubk"], pb["prop"], pb["masks"], n_iters=T,
                       opts=OPTS[opt]).cpu().numpy()
    ref, _, _ = oracle.ld_bound(pb["net"], pb["l0"].astype(np.float64), pb["u0"].astype(np.float64),
                                pb["lbk"].astype(np.float64), pb["ubk"].astype(np.float64), pb["prop"],
                                pb["masks"], T, operands="bf16" if opt == "bf16" else "fp64")
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(out), fin)
    assert np.max(rel(out[fin], ref[fin])) < 1e-5


def test_batch_beyond_limit_is_rejected_before_any_work():
    pb = conv_problem("base", 4, block=32)
    net = ldb.Net(pb["specs"])
    B = 70000
    with pytest.raises(ldb.LDError) as e:
        ldb.ld_bound(net, pb["l0"], pb["u0"], pb["lbk"], pb["ubk"], None, None, n_iters=1, B=B)
    assert e.value.code == ldb.LD_ERR_UNSUPPORTED
    assert net.sync_status() == ldb.LD_OK


def test_injected_allocation_failures_leave_the_handle_usable():
    """Failure detection on the allocation paths without a GPU fault: the
    host-side hook fails one of the library's device allocations; the call
    that made it returns LD_ERR_NOMEM (or LD_ERR_CUDA), and the handle still
    bounds correctly afterwards (the workspace is allocated again)."""
    pb = conv_problem("base", 8, depth=(0, 4), block=9)
    args = (pb["l0"], pb["u0"], pb["lbk"], pb["ubk"], pb["prop"], pb["masks"])
    ref = ldb.ld_bound(ldb.Net(pb["specs"]), *args, n_iters=3, opts=ldb.Options(engine="layerwise"))
    try:
        for after, code in ((0, ldb.LD_ERR_NOMEM), (3, ldb.LD_ERR_CUDA)):
            ldb.inject_alloc_failure(after, code)
            with pytest.raises(ldb.LDError) as e:
                ldb.Net(pb["specs"])
            assert e.value.code == code
        net = ldb.Net(pb["specs"])
        for code in (ldb.LD_ERR_NOMEM, ldb.LD_ERR_CUDA):
            ldb.inject_alloc_failure(0, code)
            with pytest.raises(ldb.LDError) as e:
                net.reserve(64)
            assert e.value.code == code
            out = ldb.ld_bound(net, *args, n_iters=3, opts=ldb.Options(engine="layerwise"))
            assert torch.equal(out, ref)
        # the BF16 engine's own allocations (its shadow workspace and re-laid weights)
        net.reserve(8)
        ldb.inject_alloc_failure(0, ldb.LD_ERR_NOMEM)
        with pytest.raises(ldb.LDError) as e:
            ldb.ld_bound(net, *args, n_iters=3, opts=ldb.Options(precision="bf16"))
        assert e.value.code == ldb.LD_ERR_NOMEM
        out = ldb.ld_bound(net, *args, n_iters=3, opts=ldb.Options(precision="bf16"))
        assert np.all(np.isfinite(out.cpu().numpy()) == np.isfinite(ref.cpu().numpy()))
        assert net.sync_status() == ldb.LD_OK
    finally:
        ldb.inject_alloc_failure(-1)
