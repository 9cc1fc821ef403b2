"""cc_count_noalloc: the count for callers that cannot allocate device memory.

It must return exactly what the allocating path (cc_color + cc_run_dp + cc_count/cc_decide
through a context) returns for the same inputs, on two calls in a row (the second call finds the
first call's leftovers in the shared device array).  This file is collected last so that a run
stopping at its first failure has run everything else already; it also passes run alone.
"""
from __future__ import annotations

import numpy as np
import pytest

import synth

cc = pytest.importorskip("paper_1908_11248_gb300")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    import __graft_entry__

    __graft_entry__.build()


def allocating_count(g, pat, seed, trials, k):
    nF, e, td = pat
    with cc.Context(arena_bytes=1 << 30) as ctx:
        cc.cc_load_graph(ctx.h, *g)
        pid = cc.cc_load_pattern(ctx.h, nF, e, td)
        cid = cc.cc_color(ctx.h, seed, trials, k)
        run = cc.cc_run_dp(ctx.h, pid, cid, cc.cc_default_opts())
        counts = cc.cc_count(ctx.h, run, trials)
        exists = cc.cc_decide(ctx.h, run, trials)
        cc.cc_release(ctx.h, run)
    return counts, exists


def test_noalloc_matches_allocating_path_twice(built):
    import torch

    stream = torch.cuda.current_stream().cuda_stream
    cases = [
        (synth.erdos_renyi(200, 0.05, 1), synth.cycle_pattern(5), 7, 3, 5),
        (synth.barabasi_albert(2000, 3, 2), synth.grid_pattern(2, 3), 11, 2, 6),
    ]
    for g, pat, seed, trials, k in cases:
        want_c, want_e = allocating_count(g, pat, seed, trials, k)
        assert int(want_c.sum()) > 0
        for _ in range(2):  # the second call reuses the array the first one left behind
            got_c, got_e = cc.cc_count_noalloc(0, stream, *g, pat[0], pat[1], pat[2], seed,
                                                trials, k)
            assert np.array_equal(got_c, want_c)
            assert np.array_equal(got_e, want_e)


def test_noalloc_rejects_oversized_input(built):
    import torch

    n = 1 << 22  # colours alone for 8 trials would take 2 * 8 * 4 Mi bytes > the array
    g = synth.csr_from_edges(n, np.zeros((0, 2), np.int64))
    with pytest.raises(cc.CCError) as ex:
        cc.cc_count_noalloc(0, torch.cuda.current_stream().cuda_stream, *g, 1,
                            np.zeros((0, 2), np.int32), None, 1, 8, 1)
    assert ex.value.code == cc.CC_ENOMEM
