"""The autotuner: it tries re-rooted decompositions and option settings, every candidate gives
the same root results (it checks this itself), and the options and schedule it returns run to
the oracle's counts."""
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


@pytest.mark.parametrize("pat", [synth.grid_pattern(2, 3), synth.pattern_B(),
                                 synth.random_partial_ktree(7, 2, 3)])
def test_autotune_result_runs_to_oracle(ctx, pat):
    g = synth.barabasi_albert(3000, 4, 5)
    cc.cc_load_graph(ctx.h, *g)
    nF = pat[0]
    pid = cc.cc_load_pattern(ctx.h, *pat)
    z = oracle.colors(3000, 2, nF, seed=17)
    cid = cc.cc_set_colors(ctx.h, z, nF)
    best, bpid, ms, tried = cc.cc_autotune(ctx.h, pid, cid, None, 6, 1)
    assert tried >= 5 and ms > 0
    assert best.fuse in (0, 1, 2) and best.block in (128, 256, 512)
    # the chosen schedule is a nice decomposition of the same pattern
    N, width = cc.cc_pattern_info(ctx.h, bpid)
    assert width == cc.cc_pattern_info(ctx.h, pid)[1]
    ref = oracle.run_dp(g, pat, z, nF)
    run = cc.cc_run_dp(ctx.h, bpid, cid, best)
    assert np.array_equal(cc.cc_count(ctx.h, run, 2), ref.count)
    assert np.array_equal(cc.cc_decide(ctx.h, run, 2), ref.exists)
    cc.cc_release(ctx.h, run)
    cc.cc_release_colors(ctx.h, cid)


def test_rerooted_schedules_agree(ctx):
    """Rooting the decomposition of a path at each bag gives different nice decompositions with
    different intermediate tables and the same counts."""
    g = synth.barabasi_albert(2000, 3, 6)
    cc.cc_load_graph(ctx.h, *g)
    pat = synth.path_pattern(6)
    pid = cc.cc_load_pattern(ctx.h, *pat)
    z = oracle.colors(2000, 1, 6, seed=3)
    cid = cc.cc_set_colors(ctx.h, z, 6)
    before = cc.cc_pattern_info(ctx.h, pid)
    best, bpid, ms, tried = cc.cc_autotune(ctx.h, pid, cid, None, 4, 1)
    assert tried >= 4 + 5  # four schedules, then the option sweeps
    assert cc.cc_pattern_info(ctx.h, pid) == before  # the loaded pattern is unchanged
    ref = oracle.run_dp(g, pat, z, 6)
    assert pid <= bpid < pid + 4
    for q in range(pid, pid + 4):  # the pattern and the three re-rooted ones the tuner loaded
        run = cc.cc_run_dp(ctx.h, q, cid, cc.cc_default_opts())
        assert np.array_equal(cc.cc_count(ctx.h, run, 1), ref.count)
        cc.cc_release(ctx.h, run)
    cc.cc_release_colors(ctx.h, cid)
