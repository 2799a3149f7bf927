"""The allocation-free final-bound entry point (ld_final_bound_noalloc).

Some callers cannot call cudaMalloc when they need a bound (code running
where allocation is not permitted, or that must keep its device memory fixed
after start-up); this entry point keeps its scratch in a fixed array inside
the library.  It must return what the allocating path returns: the sound FP64
bound of ld_bound with n_iters = 0 at the same rho.  This file is collected
last so that a run stopping at the first failure has run everything else.
"""
import numpy as np
import pytest
import torch

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


def test_noalloc_matches_allocating_path_on_two_calls():
    pb = conv_problem("base", 24, depth=(0, 8), block=11)
    net = ldb.Net(pb["specs"])
    N = pb["lbk"].shape[1]
    args = (pb["l0"], pb["u0"], pb["lbk"], pb["ubk"])
    for seed in (31, 32):  # two calls in a row, with different duals
        rho = synth.random_duals([N], pb["B"], seed=seed, scale=0.05)[0]
        ref = ldb.ld_bound(net, *args, pb["prop"], pb["masks"], n_iters=0, rho_in=rho).cpu().numpy()
        got = ldb.ld_final_bound_noalloc(net, *args, rho, prop=pb["prop"], masks=pb["masks"]).cpu().numpy()
        fin = np.isfinite(ref)
        assert np.array_equal(np.isfinite(got), fin)
        rel = np.abs(got[fin] - ref[fin]) / np.maximum(np.abs(ref[fin]), 1.0)
        assert rel.max() <= 1e-12


def test_noalloc_rejects_batches_beyond_its_scratch():
    pb = conv_problem("base", 1, depth=(0, 0), block=12)
    net = ldb.Net(pb["specs"])
    B = 60000
    rho = torch.zeros((B, pb["lbk"].shape[1]), dtype=torch.float32, device="cuda")
    with pytest.raises(ldb.LDError) as e:
        ldb.ld_final_bound_noalloc(net, pb["l0"], pb["u0"], pb["lbk"], pb["ubk"], rho)
    assert e.value.code == ldb.LD_ERR_UNSUPPORTED
