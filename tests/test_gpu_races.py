"""Race detection without a sanitizer: repeated runs of every engine on the
same inputs must give bitwise the same duals.  The FP32 and BF16 iterations
sum in a fixed order (no atomics), so any difference in rho_T between two
runs is a race (a read before its writer's barrier, a lost write).  The FP64
final bound adds fixed partial-sum slots in a fixed order, so it is
deterministic too; it is held to 1e-12 relative here, the duals bitwise.
Ragged batches (B not a multiple of the subdomains per CTA) cover the padding
subdomains of the last CTA; Base runs the fused engine's FC and conv thread
groups side by side, Deep a split transposed FC pass inside the FC group."""
import numpy as np
import pytest
import torch

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


ENGINES = {"layerwise": ldb.Options(engine="layerwise"), "fused1": ldb.Options(engine="fused", tile=1),
           "fused2": ldb.Options(engine="fused", tile=2), "fused4": ldb.Options(engine="fused", tile=4),
           "fused2w": ldb.Options(engine="fused", tile=2, cta_threads=512),
           "fused1w": ldb.Options(engine="fused", tile=1, cta_threads=512),
           "bf16": ldb.Options(precision="bf16")}


@pytest.mark.parametrize("engine", sorted(ENGINES))
@pytest.mark.parametrize("name,B", [("base", 37), ("deep", 13)])
def test_repeated_runs_give_bitwise_the_same_duals(name, B, engine):
    pb = conv_problem(name, B, depth=(0, 8), block=31)
    runs = []
    for _ in range(3):
        net = ldb.Net(pb["specs"])
        out, rho = ldb.ld_bound(net, pb["l0"], pb["u0"], pb["lbk"], pb["ubk"], pb["prop"], pb["masks"], n_iters=7,
                                opts=ENGINES[engine], return_rho=True)
        runs.append((out.cpu().numpy(), rho.cpu().numpy()))
    out0, rho0 = runs[0]
    for out, rho in runs[1:]:
        assert np.array_equal(rho, rho0), np.argwhere(rho != rho0)[:8].tolist()
        fin = np.isfinite(out0)
        assert np.array_equal(np.isfinite(out), fin)
        assert np.all(np.abs(out[fin] - out0[fin]) <= 1e-12 * np.maximum(np.abs(out0[fin]), 1.0))
