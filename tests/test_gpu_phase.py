"""The Erdos-Renyi phase-transition study (paper Section 5.4) on the GPU: a point of the study
(target G(150, p), pattern G(10, q), ten colourings, k = 10) gives the oracle's counts, and the
decomposition width it records is the pattern's treewidth."""
from __future__ import annotations

import numpy as np
import pytest

import bench
from tests import brute
import oracle
import synth

cc = pytest.importorskip("paper_1908_11248_gb300")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__

    __graft_entry__.build()
    with cc.Context(arena_bytes=8 << 30) as c:
        yield c


# (p index, q index) on the 0.03 grid: sparse and dense targets, paths, forests, an edgeless
# pattern, and an empty target (no copy)
POINTS = [(10, 5), (33, 2), (0, 10), (20, 6), (25, 4)]


@pytest.mark.parametrize("ip,iq", POINTS)
def test_phase_point_matches_oracle(ctx, ip, iq):
    p, q, g, pat, seed = synth.er_phase_instance(ip, iq)
    spec = synth.ER_PHASE
    cc.cc_load_graph(ctx.h, *g)
    status, width, found, counts, ent = bench.er_phase_point(
        cc, ctx.h, pat, spec["n_pattern"], seed, spec["iterations"])
    assert status == 0 and ent > 0
    assert width == brute.exact_treewidth(pat[0], pat[1])
    # the oracle on the first two of the ten colourings, over its own decomposition
    z = oracle.colors(spec["n_target"], 2, spec["n_pattern"], seed)
    ref = oracle.run_dp(g, (pat[0], pat[1], brute.elimination_td(pat[0], pat[1])), z,
                        spec["n_pattern"])
    assert np.array_equal(counts[:2], ref.count)
    if ref.exists.any():
        assert found
    if p == 0.0 and len(pat[1]):
        assert not found and not counts.any()


def test_phase_leg_small_grid(ctx):
    """The study's driver on a coarse grid (step 0.33: p, q in {0, 0.33, 0.66, 0.99}): every
    point completes or reports a resource status, and a dense target with a sparse pattern is
    found."""
    out = bench.er_phase_leg(cc, __import__("torch"), step=0.33, arena_gb=8)
    P = len(out["probs"])
    assert P == 4 and out["points"] == 16
    st = np.array(out["status_grid"])
    assert set(np.unique(st)) <= {0, cc.CC_ENOMEM, cc.CC_EKEYWIDTH}
    assert st[3, 0] == 0 and out["found_grid"][3][0] == 1
    assert out["found_grid"][0][1] == 0 or st[0][1] != 0
