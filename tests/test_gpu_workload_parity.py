"""Workload-scale parity with more trials: the oracle runs the sampled colourings on spawned host
processes (one trial each) while the GPU runs the same colourings in one batched run, and every
trial's count and every node's table size (summed over the sample) must agree exactly.

* Barabasi-Albert n=20000, m=4, the 2x4 grid, k=8: 16 of the 64 trials of the benchmark's
  colouring (every fourth).
* Erdos-Renyi n=100000, average degree 10, the 3x3 grid, k=9: 16 of the 32 trials, with pattern
  vertex 0 restricted to the host vertices = 0 (mod 16) by allowed-mapping masks (Section 3.2),
  so that a trial's oracle run takes seconds; the GPU runs the same masked pattern, chained
  introduces included.
"""
from __future__ import annotations

import multiprocessing as mp

import numpy as np
import pytest

import oracle
import paper_1908_11248_gb300 as cc
import synth

pytestmark = pytest.mark.gpu

_JOB = {}


def _init(g, pat, k, allow):
    _JOB.update(g=g, pat=pat, k=k, allow=allow)


def _one(row):
    import oracle as o

    r = o.run_dp(_JOB["g"], _JOB["pat"], row[None, :], _JOB["k"], allow=_JOB["allow"])
    return int(r.count[0]), r.node_sizes[0].astype(np.int64)


def oracle_trials(g, pat, k, rows, allow=None):
    """Per trial (count, node sizes) from the oracle on spawned processes (a pool forked after
    the GPU was touched can hang)."""
    workers = max(1, min(len(rows), mp.cpu_count()))
    with mp.get_context("spawn").Pool(workers, initializer=_init,
                                      initargs=(g, pat, k, allow)) as pool:
        return pool.map_async(_one, list(rows), chunksize=1).get(timeout=1200)


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__

    __graft_entry__.build()
    oracle.build()
    c = cc.Context(arena_bytes=96 << 30)
    yield c
    c.close()


def _gpu(ctx, g, pid, z, k, N):
    cid = cc.cc_set_colors(ctx.h, z, k)
    out = None
    for _ in range(2):  # the second run is planned (the benchmark's launch configuration)
        run = cc.cc_run_dp(ctx.h, pid, cid, cc.cc_default_opts())
        out = (cc.cc_count(ctx.h, run, z.shape[0]), cc.cc_table_stats(ctx.h, run, N)[0],
               cc.cc_run_mode(ctx.h, run))
        cc.cc_release(ctx.h, run)
    cc.cc_release_colors(ctx.h, cid)
    return out


def test_ba20k_grid2x4_sixteen_trials(ctx):
    w = synth.WORKLOADS["ba20k_grid2x4"]
    g = synth.make_graph(w["graph"])
    pat = synth.make_pattern(w["pattern"])
    z = oracle.colors(20000, 64, 8, w["seed"])
    sample = list(range(0, 64, 4))
    ref = oracle_trials(g, pat, 8, [z[t] for t in sample])
    cc.cc_load_graph(ctx.h, *g)
    pid = cc.cc_load_pattern(ctx.h, *pat)
    N, _ = cc.cc_pattern_info(ctx.h, pid)
    counts, sizes, mode = _gpu(ctx, g, pid, z[sample], 8, N)
    assert mode == "planned"
    assert [int(c) for c in counts] == [c for c, _ in ref]
    assert np.array_equal(sizes.astype(np.int64), np.sum([s for _, s in ref], axis=0))


def test_er100k_grid3x3_sixteen_sliced_trials(ctx):
    w = synth.WORKLOADS["er100k_grid3x3"]
    n, k = 100000, 9
    g = synth.make_graph(w["graph"])
    nF, pe, td = synth.make_pattern(w["pattern"])
    z = oracle.colors(n, 32, k, w["seed"])
    allow = np.full(n, 0xFFFFFFFF, np.uint32)
    allow[np.arange(n) % 16 != 0] &= np.uint32(0xFFFFFFFE)  # pattern vertex 0: v = 0 mod 16
    sample = list(range(16))
    ref = oracle_trials(g, (nF, pe, td), k, [z[t] for t in sample], allow)
    cc.cc_load_graph(ctx.h, *g)
    pid = cc.cc_load_pattern_masked(ctx.h, nF, pe, td, allow)
    N, _ = cc.cc_pattern_info(ctx.h, pid)
    counts, sizes, mode = _gpu(ctx, g, pid, z[sample], k, N)
    assert mode == "planned"
    assert [int(c) for c in counts] == [c for c, _ in ref]
    assert np.array_equal(sizes.astype(np.int64), np.sum([s for _, s in ref], axis=0))
    assert int(sizes.sum()) > 10 ** 7  # the sample is not trivially small
