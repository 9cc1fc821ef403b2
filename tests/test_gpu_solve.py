"""The repetition driver: batches of colourings continue one Philox trial sequence, so a solve
equals one run over all its trials; its merged enumeration is the oracle's union over the same
trials; decisions stop at the first batch with a colourful copy, or after the paper's number of
repetitions when there is none."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth

cc = pytest.importorskip("paper_1908_11248_gb300")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__

    __graft_entry__.build()
    c = cc.Context(arena_bytes=8 << 30)
    yield c
    c.close()


def test_solve_enumeration_is_the_union_over_trials(ctx):
    w = synth.WORKLOADS["er200_c5"]
    g = synth.make_graph(w["graph"])
    pat = synth.make_pattern(w["pattern"])
    cc.cc_load_graph(ctx.h, *g)
    pid = cc.cc_load_pattern(ctx.h, *pat)
    T = 40
    found, tr, rows, est = cc.cc_solve(ctx.h, pid, w["seed"], 5, 0.5, 16, T, 100000, 5)
    assert cc.cc_solve_trials(5, 0.5) == 103 and tr == T
    z = oracle.colors(200, T, 5, w["seed"])
    ref = oracle.run_dp(g, pat, z, 5)
    want, total, _ = ref.enumerate(100000)
    assert total < 100000
    assert found and np.array_equal(rows, want)
    p = 5 * 4 * 3 * 2 * 1 / 5 ** 5
    assert est == pytest.approx(float(ref.count.astype(np.float64).mean()) / p, rel=1e-12)
    # the same trials in one run give the same list
    cid = cc.cc_color(ctx.h, w["seed"], T, 5)
    run = cc.cc_run_dp(ctx.h, pid, cid, cc.cc_default_opts(retain=1))
    one, tot1 = cc.cc_enumerate(ctx.h, run, 100000, 5)
    assert np.array_equal(one, rows) and tot1 == len(rows)
    cc.cc_release(ctx.h, run)
    cc.cc_release_colors(ctx.h, cid)
    # a smaller limit keeps the smallest rows of the union
    _, _, few, _ = cc.cc_solve(ctx.h, pid, w["seed"], 5, 0.5, 7, T, 50, 5)
    assert np.array_equal(few, want[:50])


def test_solve_decision(ctx):
    # present: the first batch already finds a colourful 5-cycle
    w = synth.WORKLOADS["er200_c5"]
    cc.cc_load_graph(ctx.h, *synth.make_graph(w["graph"]))
    pid = cc.cc_load_pattern(ctx.h, *synth.cycle_pattern(5))
    found, tr, rows, _ = cc.cc_solve(ctx.h, pid, 3, 5, 0.1, 8, 1000, 0, 5)
    assert found and tr == 8 and len(rows) == 0
    # absent: no 4-clique in a tree, so every one of the ceil(e^4 ln 10) = 126 trials runs
    tree = synth.barabasi_albert(500, 1, 4)
    cc.cc_load_graph(ctx.h, *tree)
    pid = cc.cc_load_pattern(ctx.h, *synth.clique_pattern(4))
    found, tr, rows, est = cc.cc_solve(ctx.h, pid, 9, 4, 0.1, 32, 1000, 0, 4)
    assert cc.cc_solve_trials(4, 0.1) == 126
    assert not found and tr == 126 and est == 0.0
    found, tr, _, _ = cc.cc_solve(ctx.h, pid, 9, 4, 0.1, 32, 50, 0, 4)
    assert not found and tr == 50
    with pytest.raises(cc.CCError):
        cc.cc_solve(ctx.h, pid, 9, 3, 0.1, 32, 50, 0, 4)  # k < n_F
    with pytest.raises(cc.CCError):
        cc.cc_solve(ctx.h, pid, 9, 4, 1.5, 32, 50, 0, 4)  # epsilon outside (0, 1)
