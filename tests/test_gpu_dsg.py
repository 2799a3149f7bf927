"""GPU: DSG+ and Dec-DSG+ (Sec. 2.2.2, Eq. (dj_prob-main), Theorem 1) against
oracle/dsg.py.

  * at the CROWN start (no iteration) both bounds equal the CROWN bound
    (Prop. 3; Theorem 1's equality case) within 1e-5;
  * after 1 and 3 iterations both match the oracle within 1e-5;
  * Theorem 1 on the device: after 50 iterations the Dec-DSG+ bound q(mu) is
    at least DSG+'s own d_O(mu, lambda) for every subdomain;
  * tiny MLPs after 200 iterations: never above the Planet LP optimum.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import dsg, lp
from paper_2104_06718_gb300 import binding as ldb
from helpers import conv_problem, oracle_lists, outward_f32, tiny_problem

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


def run_both(pb, T):
    on = pb["net"]
    net = ldb.Net(pb["specs"])
    dec, d = ldb.ld_bound_dsg(net, pb["l0"], pb["u0"], pb["lbk"], pb["ubk"], pb["prop"], pb["masks"], n_iters=T)
    L0, U0, lbs, ubs, empty = oracle_lists(on, pb)
    keep = ~empty
    sel = lambda l: [None] + [x[keep] for x in l[1:]]
    r = dsg.dsg_plus(on, L0[keep], U0[keep], sel(lbs), sel(ubs), T)
    dec, d = dec.cpu().numpy(), d.cpu().numpy()
    assert np.all(np.isinf(dec[~keep])) and np.all(np.isinf(d[~keep]))
    return dec[keep], d[keep], r


@pytest.mark.parametrize("name", ["base", "deep"])
@pytest.mark.parametrize("T", [0, 1, 3])
def test_dsg_short_runs_match_oracle(name, T):
    pb = conv_problem(name, 16, depth=(0, 8), block=8)
    dec, d, r = run_both(pb, T)
    assert np.max(rel(d, r.d_final)) < 1e-5
    assert np.max(rel(dec, r.q_final)) < 1e-5
    if T == 0:
        assert np.max(rel(d, dec)) < 1e-5    # Prop. 3 / Theorem 1's equality case


def test_theorem_1_on_the_device():
    pb = conv_problem("base", 32, depth=(0, 8), block=12)
    net = ldb.Net(pb["specs"])
    dec, d = ldb.ld_bound_dsg(net, pb["l0"], pb["u0"], pb["lbk"], pb["ubk"], pb["prop"], pb["masks"], n_iters=50)
    dec, d = dec.cpu().numpy(), d.cpu().numpy()
    fin = np.isfinite(dec)
    assert np.all(dec[fin] >= d[fin] - 1e-6 * np.maximum(np.abs(d[fin]), 1.0))
    assert np.mean(dec[fin] - d[fin]) > 0        # the decomposed evaluation helps on average


def test_dsg_tiny_nets_stay_below_the_lp():
    for i in range(6):
        specs, on, l0, u0, lb, ub = tiny_problem(i)
        flat_l = np.concatenate([lb[k] for k in range(1, on.n)], axis=1)
        flat_u = np.concatenate([ub[k] for k in range(1, on.n)], axis=1)
        lbk, ubk = outward_f32(flat_l, flat_u)
        net = ldb.Net(specs)
        dec, d = ldb.ld_bound_dsg(net, l0.astype(np.float32), u0.astype(np.float32), lbk, ubk,
                                  masks=np.zeros((1, lbk.shape[1]), np.int8), n_iters=200)
        lbs = oracle.layer_lists(on, lbk.astype(np.float64))
        ubs = oracle.layer_lists(on, ubk.astype(np.float64))
        p = lp.planet_lp(on, l0[0], u0[0], [None] + [x[0] for x in lbs[1:]], [None] + [x[0] for x in ubs[1:]]).p_star
        tol = 1e-9 * max(1.0, abs(p))
        assert dec.item() <= p + tol and d.item() <= p + 1e-5 * max(1.0, abs(p))
