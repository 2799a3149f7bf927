"""Host-only checks of the fused tensor-core engine's layout (no GPU).

The plan places the BF16 shadow planes of every conv layer's input x_k and
output dual rho_{k+1} in shared memory and lists the tcgen05.mma operations
of one iteration with their shared-memory operand descriptors.  Building it
checks, for every MMA and every valid output row, that the 2 x 8 channels the
descriptor addresses are exactly those the epilogues write for the tap and
channel group of that K chunk (the forward pass reading x_k at (stride y + i -
pad, stride x + j - pad), the transposed pass reading rho_{k+1} at
((Y + pad - i) / stride, ...)), and that every operand stays inside the
CTA's shared memory.  These tests run that check on the benchmark's nets.
"""
import pytest

from paper_2104_06718_gb300 import binding as ldb
from paper_2104_06718_gb300 import synth

SMEM = 232448  # bytes of shared memory a GB300 CTA may opt in to


def plan(name, S, smem=SMEM):
    try:
        return ldb.fused_tc_plan(synth.make_convnet(name), S, smem)
    except OSError as e:  # library not built
        pytest.skip(str(e))


@pytest.mark.parametrize("name,S", [("base", 1), ("base", 2), ("wide", 1), ("deep", 1)])
def test_plan_is_consistent_and_fits(name, S):
    p = plan(name, S)
    assert p is not None
    assert p["smem_bytes"] <= SMEM
    assert p["tmem_cols"] in (32, 64, 128, 256, 512)
    n_conv = sum(1 for s in synth.make_convnet(name) if s.kind == "conv")
    assert p["passes"] == 2 * n_conv
    assert p["shadow_bytes"] % 128 == 0 and p["weight_tile_bytes"] % 128 == 0


def test_base_plan_counts():
    # Base: conv 3->8 4x4/2 on 32x32, conv 8->16 4x4/2; two subdomains per CTA
    # give full 128-row tiles everywhere: transposed conv1 16 tiles x 2 K steps,
    # transposed conv2 4 x 4, forward conv1 4 x 8, forward conv2 1 x 8
    p = plan("base", 2)
    assert p["mmas_per_iteration"] == 16 * 2 + 4 * 4 + 4 * 8 + 1 * 8
    assert p["half_tile_mmas"] == 0
    # one subdomain per CTA: the 8-row grids (forward conv2, the phases of
    # transposed conv2) fill half a tile
    p1 = plan("base", 1)
    assert p1["half_tile_mmas"] == 4 * 4 + 8


def test_no_plan_when_it_does_not_fit_or_for_fc_nets():
    assert plan("wide", 2) is None                     # the state of 2 Wide subdomains exceeds shared memory
    assert plan("base", 2, smem=100000) is None
    assert ldb.fused_tc_plan(synth.tiny_mlp(0), 1) is None  # no conv layer
