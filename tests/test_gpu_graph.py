"""Planned, graph-replayed and batched runs against the CPU oracle (bit-exact, integer results).

A run of a (pattern, graph content, trials, colours, options) key that has been seen before uses
the capacities planned by the earlier runs; with use_graph it is replayed from a captured CUDA
graph, and a batch of such requests is replayed as parallel branches of one graph.  Whatever
path a run takes, its per-trial counts, exists flags and table sizes are the oracle's.
"""
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


def _load(ctx, pat):
    nF, e, td = pat
    return cc.cc_load_pattern(ctx.h, nF, e, td)


def _check(ctx, run, pid, ref, trials):
    N, _ = cc.cc_pattern_info(ctx.h, pid)
    assert np.array_equal(cc.cc_count(ctx.h, run, trials), ref.count)
    assert np.array_equal(cc.cc_decide(ctx.h, run, trials), ref.exists)
    assert np.array_equal(cc.cc_table_stats(ctx.h, run, N)[0], ref.node_sizes.sum(axis=0))


def test_planned_mode_reached_and_exact(ctx):
    """The first run of a key is exact, later ones planned; both give the oracle's results, and a
    reload of the same graph content keeps the plan."""
    g = synth.barabasi_albert(3000, 4, 7)
    for pat in (synth.grid_pattern(2, 3), synth.pattern_B(), synth.random_partial_ktree(8, 2, 9)):
        nF = pat[0]
        cc.cc_load_graph(ctx.h, *g)
        pid = _load(ctx, pat)
        modes = []
        for rep in range(3):
            if rep == 2:
                cc.cc_load_graph(ctx.h, *g)  # same content: the plan stays
            z = oracle.colors(3000, 4, nF, seed=40 + rep)
            ref = oracle.run_dp(g, pat, z, nF)
            cid = cc.cc_set_colors(ctx.h, z, nF)
            run = cc.cc_run_dp(ctx.h, pid, cid, cc.cc_default_opts())
            _check(ctx, run, pid, ref, 4)
            modes.append(cc.cc_run_mode(ctx.h, run))
            cc.cc_release(ctx.h, run)
            cc.cc_release_colors(ctx.h, cid)
        assert modes == ["exact", "planned", "planned"]


@pytest.mark.parametrize("fuse", [2, 1, 0])
def test_graph_replay_matches_oracle(ctx, fuse):
    """use_graph: exact first, then captured and replayed with fresh colourings each time; every
    replay launches the same kernels and gives the oracle's results."""
    g = synth.barabasi_albert(2500, 4, 21)
    cc.cc_load_graph(ctx.h, *g)
    for pat in (synth.cycle_pattern(5), synth.grid_pattern(2, 3), synth.pattern_B()):
        nF = pat[0]
        pid = _load(ctx, pat)
        modes, launched = [], []
        for rep in range(4):
            z = oracle.colors(2500, 3, nF, seed=100 + rep)
            ref = oracle.run_dp(g, pat, z, nF)
            cid = cc.cc_set_colors(ctx.h, z, nF)
            before = cc.cc_context_stats(ctx.h)[0]
            run = cc.cc_run_dp(ctx.h, pid, cid, cc.cc_default_opts(use_graph=1, fuse=fuse))
            launched.append(cc.cc_context_stats(ctx.h)[0] - before)
            _check(ctx, run, pid, ref, 3)
            modes.append(cc.cc_run_mode(ctx.h, run))
            cc.cc_release(ctx.h, run)
            cc.cc_release_colors(ctx.h, cid)
        assert modes == ["exact", "graph", "graph", "graph"]
        assert launched[1] == launched[2] == launched[3] > 0


def test_graph_overflow_falls_back(ctx):
    """A graph captured with capacities planned on a one-colour colouring (no colourful edge)
    is too small for a random colouring: the replay notices, the graph is dropped and the run is
    repeated directly with the oracle's results; the next run captures a new graph."""
    g = synth.barabasi_albert(3000, 4, 8)
    pat = synth.grid_pattern(2, 3)
    cc.cc_load_graph(ctx.h, *g)
    pid = _load(ctx, pat)
    mono = np.zeros((4, 3000), np.uint8)
    opts = cc.cc_default_opts(use_graph=1)
    for want in ("exact", "graph"):
        cid = cc.cc_set_colors(ctx.h, mono, 6)
        run = cc.cc_run_dp(ctx.h, pid, cid, opts)
        assert int(cc.cc_count(ctx.h, run, 4).sum()) == 0
        assert cc.cc_run_mode(ctx.h, run) == want
        cc.cc_release(ctx.h, run)
        cc.cc_release_colors(ctx.h, cid)
    z = oracle.colors(3000, 4, 6, seed=9)
    ref = oracle.run_dp(g, pat, z, 6)
    for want in ("exact", "graph"):
        cid = cc.cc_set_colors(ctx.h, z, 6)
        run = cc.cc_run_dp(ctx.h, pid, cid, opts)
        _check(ctx, run, pid, ref, 4)
        assert cc.cc_run_mode(ctx.h, run) == want
        cc.cc_release(ctx.h, run)
        cc.cc_release_colors(ctx.h, cid)


def test_batch_graph_matches_oracle(ctx):
    """A batch of requests (different patterns, one pattern twice with different colourings,
    different trial counts, 64- and 128-bit keys) runs exactly, then as one graph of parallel
    branches; each request's results are the oracle's."""
    n = 2000
    g = synth.erdos_renyi(n, 6.0 / n, 5)
    cc.cc_load_graph(ctx.h, *g)
    reqs = [(synth.cycle_pattern(5), 5, 3), (synth.grid_pattern(2, 3), 6, 2),
            (synth.cycle_pattern(5), 5, 3), (synth.pattern_B(), None, 2),
            (synth.star_pattern(4), 7, 1), (synth.cycle_pattern(5), 31, 2)]
    pids = [_load(ctx, r[0]) for r in reqs]
    opts = cc.cc_default_opts(use_graph=1)
    for rep in range(3):
        cids, refs = [], []
        for i, (pat, k, T) in enumerate(reqs):
            k = k or pat[0]
            z = oracle.colors(n, T, k, seed=1000 * rep + i)
            refs.append(oracle.run_dp(g, pat, z, k))
            cids.append(cc.cc_set_colors(ctx.h, z, k))
        runs = cc.cc_run_batch(ctx.h, pids, cids, opts)
        for i, run in enumerate(runs):
            _check(ctx, run, pids[i], refs[i], reqs[i][2])
            assert cc.cc_run_mode(ctx.h, run) == ("exact" if rep == 0 else "graph")
            cc.cc_release(ctx.h, run)
        for cid in cids:
            cc.cc_release_colors(ctx.h, cid)


def test_batch_without_graph_and_errors(ctx):
    """Without use_graph a batch is a sequence of runs with the same results; a bad request in a
    batch fails the whole call and keeps no run."""
    n = 1500
    g = synth.barabasi_albert(n, 3, 2)
    cc.cc_load_graph(ctx.h, *g)
    pats = [synth.path_pattern(4), synth.cycle_pattern(4)]
    pids = [_load(ctx, p) for p in pats]
    z = oracle.colors(n, 2, 4, seed=5)
    cid = cc.cc_set_colors(ctx.h, z, 4)
    runs = cc.cc_run_batch(ctx.h, pids, [cid, cid], cc.cc_default_opts())
    for run, pid, pat in zip(runs, pids, pats):
        _check(ctx, run, pid, oracle.run_dp(g, pat, z, 4), 2)
        cc.cc_release(ctx.h, run)
    used = cc.cc_context_stats(ctx.h)[1]
    with pytest.raises(cc.CCError):
        cc.cc_run_batch(ctx.h, [pids[0], 999999], [cid, cid], cc.cc_default_opts())
    assert cc.cc_context_stats(ctx.h)[1] == used
    assert cc.cc_run_batch(ctx.h, [], [], None) == []
    cc.cc_release_colors(ctx.h, cid)


def test_graph_dropped_on_new_graph(ctx):
    """Loading a different graph drops captured graphs and plans: the next run is exact and
    correct on the new graph."""
    pat = synth.cycle_pattern(5)
    opts = cc.cc_default_opts(use_graph=1)
    pid = None
    for seed, want in ((31, ["exact", "graph"]), (32, ["exact", "graph"])):
        g = synth.barabasi_albert(2000, 3, seed)
        cc.cc_load_graph(ctx.h, *g)
        pid = pid or _load(ctx, pat)
        z = oracle.colors(2000, 2, 5, seed=seed)
        ref = oracle.run_dp(g, pat, z, 5)
        modes = []
        for _ in range(2):
            cid = cc.cc_set_colors(ctx.h, z, 5)
            run = cc.cc_run_dp(ctx.h, pid, cid, opts)
            _check(ctx, run, pid, ref, 2)
            modes.append(cc.cc_run_mode(ctx.h, run))
            cc.cc_release(ctx.h, run)
            cc.cc_release_colors(ctx.h, cid)
        assert modes == want


def test_trials_stream_when_memory_is_short(ctx):
    """In an arena too small for all 16 trials at once, a run without kept tables splits the
    trials into chunks that fit; counts, exists flags and table sizes are those of the run in a
    large arena (and of the oracle on a sample)."""
    g = synth.barabasi_albert(3000, 4, 13)
    pat = synth.grid_pattern(2, 3)
    z = oracle.colors(3000, 16, 6, seed=21)
    cc.cc_load_graph(ctx.h, *g)
    pid = _load(ctx, pat)
    cid = cc.cc_set_colors(ctx.h, z, 6)
    run = cc.cc_run_dp(ctx.h, pid, cid, cc.cc_default_opts())
    N, _ = cc.cc_pattern_info(ctx.h, pid)
    want = (cc.cc_count(ctx.h, run, 16), cc.cc_decide(ctx.h, run, 16),
            cc.cc_table_stats(ctx.h, run, N)[0])
    assert cc.cc_run_mode(ctx.h, run) == "exact"
    cc.cc_release(ctx.h, run)
    cc.cc_release_colors(ctx.h, cid)
    small = cc.Context(arena_bytes=96 << 20)
    try:
        cc.cc_load_graph(small.h, *g)
        spid = cc.cc_load_pattern(small.h, *pat)
        scid = cc.cc_set_colors(small.h, z, 6)
        with pytest.raises(cc.CCError) as e:  # tables kept: no streaming, nothing kept
            cc.cc_run_dp(small.h, spid, scid, cc.cc_default_opts(retain=1))
        assert e.value.code == -2
        used = cc.cc_context_stats(small.h)[1]
        for _ in range(2):
            srun = cc.cc_run_dp(small.h, spid, scid, cc.cc_default_opts())
            assert cc.cc_run_mode(small.h, srun) == "streamed"
            assert np.array_equal(cc.cc_count(small.h, srun, 16), want[0])
            assert np.array_equal(cc.cc_decide(small.h, srun, 16), want[1])
            assert np.array_equal(cc.cc_table_stats(small.h, srun, N)[0], want[2])
            cc.cc_release(small.h, srun)
        assert cc.cc_context_stats(small.h)[1] == used
    finally:
        small.close()
    ref = oracle.run_dp(g, pat, z[:2], 6)
    assert np.array_equal(want[0][:2], ref.count)


def test_single_trial_runs_in_slices_when_memory_is_short(ctx):
    """In an arena too small for even one trial, a run without kept tables splits each trial by
    the image of one pattern vertex (allowed-mapping masks, Section 3.2): the counts and exists
    flags are those of the run in a large arena and of the oracle, table sizes add up to at least
    the true ones, and a second run reuses the slice count it found."""
    g = synth.barabasi_albert(3000, 4, 13)
    pat = synth.cycle_pattern(6)
    z = oracle.colors(3000, 2, 6, seed=21)
    cc.cc_load_graph(ctx.h, *g)
    pid = _load(ctx, pat)
    cid = cc.cc_set_colors(ctx.h, z, 6)
    run = cc.cc_run_dp(ctx.h, pid, cid, cc.cc_default_opts())
    N, _ = cc.cc_pattern_info(ctx.h, pid)
    want = (cc.cc_count(ctx.h, run, 2), cc.cc_decide(ctx.h, run, 2),
            cc.cc_table_stats(ctx.h, run, N)[0])
    cc.cc_release(ctx.h, run)
    cc.cc_release_colors(ctx.h, cid)
    small = cc.Context(arena_bytes=256 << 20)
    try:
        cc.cc_load_graph(small.h, *g)
        spid = cc.cc_load_pattern(small.h, *pat)
        scid = cc.cc_set_colors(small.h, z, 6)
        used = cc.cc_context_stats(small.h)[1]
        for _ in range(2):
            srun = cc.cc_run_dp(small.h, spid, scid, cc.cc_default_opts())
            assert cc.cc_run_mode(small.h, srun) == "sliced"
            assert np.array_equal(cc.cc_count(small.h, srun, 2), want[0])
            assert np.array_equal(cc.cc_decide(small.h, srun, 2), want[1])
            assert (cc.cc_table_stats(small.h, srun, N)[0] >= want[2]).all()
            cc.cc_release(small.h, srun)
        assert cc.cc_context_stats(small.h)[1] == used
    finally:
        small.close()
    ref = oracle.run_dp(g, pat, z[:1], 6)
    assert int(want[0][0]) == int(ref.count[0]) > 0


def test_batch_of_partial_3trees(ctx):
    """The batched-patterns configuration at small scale: an erased power-law configuration
    graph (n=2000, exponent 2.5, mean degree 8) and 16 random partial 3-trees of 10-12 vertices,
    k = n_F, 4 trials each: single runs plan every request, then the batch is captured and
    replayed as CUDA graphs of parallel branches (a batch too large for the arena is split into
    graphs that fit).  Every request equals its own single run, and the three smallest equal the
    oracle on trial 0."""
    n, T = 2000, 4
    g = synth.power_law_config(n, 8.0, 2.5, 1)
    rng = np.random.default_rng(1)
    pats = []
    for i in range(16):
        nF = int(rng.integers(10, 13))
        pats.append(synth.random_partial_ktree(nF, 3, 7000 + i))
    big = cc.Context(arena_bytes=64 << 30)
    try:
        h = big.h
        cc.cc_load_graph(h, *g)
        pids = [cc.cc_load_pattern(h, *p) for p in pats]
        zs = [oracle.colors(n, T, p[0], seed=300 + i) for i, p in enumerate(pats)]
        opts = cc.cc_default_opts(use_graph=1)
        singles, sizes = [], []
        for pid, z, p in zip(pids, zs, pats):
            cid = cc.cc_set_colors(h, z, p[0])
            run = cc.cc_run_dp(h, pid, cid, cc.cc_default_opts())
            N, _ = cc.cc_pattern_info(h, pid)
            singles.append(cc.cc_count(h, run, T))
            sizes.append(cc.cc_table_stats(h, run, N)[0])
            cc.cc_release(h, run)
            cc.cc_release_colors(h, cid)
        # the batch: every request whose tables stay under 3*10^8 entries (the others need tens
        # of GB each at this size); the single runs planned them, so they run as a graph at once
        sel = [i for i in range(16) if int(sizes[i].sum()) <= 300_000_000]
        assert len(sel) >= 8
        for rep in range(2):
            cids = [cc.cc_set_colors(h, zs[i], pats[i][0]) for i in sel]
            runs = cc.cc_run_batch(h, [pids[i] for i in sel], cids, opts)
            for i, run in zip(sel, runs):
                N, _ = cc.cc_pattern_info(h, pids[i])
                assert cc.cc_run_mode(h, run) == "graph"
                assert np.array_equal(cc.cc_count(h, run, T), singles[i]), i
                assert np.array_equal(cc.cc_table_stats(h, run, N)[0], sizes[i]), i
                cc.cc_release(h, run)
            for cid in cids:
                cc.cc_release_colors(h, cid)
        # all 16 at once: the requests with a plan run from graphs, the large ones (whose single
        # runs went exactly or in chunks of trials) directly, with the same results
        cids = [cc.cc_set_colors(h, z, p[0]) for z, p in zip(zs, pats)]
        runs = cc.cc_run_batch(h, pids, cids, opts)
        for i, run in enumerate(runs):
            if i in sel:
                assert cc.cc_run_mode(h, run) == "graph"
            assert np.array_equal(cc.cc_count(h, run, T), singles[i]), i
            cc.cc_release(h, run)
        for cid in cids:
            cc.cc_release_colors(h, cid)
    finally:
        big.close()
    for i in sorted(range(16), key=lambda i: int(sizes[i].sum()))[:3]:
        ref = oracle.run_dp(g, pats[i], zs[i][:1], pats[i][0])
        assert int(ref.count[0]) == int(singles[i][0]), i
