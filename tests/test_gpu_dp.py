"""GPU parity of the dynamic programme against the CPU oracle (bit-exact, integer results).

Every GPU call goes through the C ABI (paper_1908_11248_gb300 is its ctypes binding).  Small
cases compare per trial: exists, the uint64 count, every node's table size and (with tables
kept and fusion off) every node's table contents.  The full-size workloads compare sampled
trials with the oracle and check properties that hold at any size.
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
    c = cc.Context(arena_bytes=24 << 30)
    yield c
    c.close()


def gpu_dp(ctx, g, pat, colours=None, k=None, seed=None, trials=1, pid=None, **opt):
    nF, e, td = pat
    k = k or nF
    cc.cc_load_graph(ctx.h, *g)
    if pid is None:
        pid = cc.cc_load_pattern(ctx.h, nF, e, td)
    n = len(g[0]) - 1
    if colours is not None:
        cid = cc.cc_set_colors(ctx.h, colours, k)
        trials = colours.shape[0]
    else:
        cid = cc.cc_color(ctx.h, seed, trials, k)
    o = cc.cc_default_opts(**opt)
    run = cc.cc_run_dp(ctx.h, pid, cid, o)
    N, _ = cc.cc_pattern_info(ctx.h, pid)
    res = dict(
        count=cc.cc_count(ctx.h, run, trials),
        exists=cc.cc_decide(ctx.h, run, trials),
        sizes=cc.cc_table_stats(ctx.h, run, N)[0],
        nodes=cc.cc_pattern_nodes(ctx.h, pid, nF),
        colours=cc.cc_get_colors(ctx.h, cid, trials, n),
        run=run, pid=pid, cid=cid, trials=trials,
    )
    return res


def release(ctx, r):
    cc.cc_release(ctx.h, r["run"])
    cc.cc_release_colors(ctx.h, r["cid"])


def oracle_tables(ref, nodes, trials):
    out = []
    for x, nd in enumerate(nodes):
        b = len(nd[4])
        d = {}
        for t in range(trials):
            phi, mask, cnt = ref.table(t, x, b)
            for i in range(len(mask)):
                d[(t, tuple(int(v) for v in phi[i]), int(mask[i]))] = int(cnt[i])
        out.append(d)
    return out


def gpu_table(ctx, r, x, b, cap):
    tr, phi, mask, cnt = cc.cc_table_dump(ctx.h, r["run"], x, cap, b)
    d = {}
    for i in range(len(mask)):
        key = (int(tr[i]), tuple(int(v) for v in phi[i]), int(mask[i]))
        assert key not in d, "duplicate key in a GPU table"
        d[key] = int(cnt[i])
    return d


# ------------------------------------------------------------------------------------------

def test_colouring_matches_oracle(ctx):
    for n, T, k, seed in [(1, 1, 1, 0), (200, 1, 5, 7), (20000, 3, 8, 7), (777, 64, 32, 2 ** 40 + 5),
                          (100003, 2, 9, 123456789)]:
        g = synth.csr_from_edges(n, np.zeros((0, 2), np.int64))
        cc.cc_load_graph(ctx.h, *g)
        cid = cc.cc_color(ctx.h, seed, T, k)
        got = cc.cc_get_colors(ctx.h, cid, T, n)
        cc.cc_release_colors(ctx.h, cid)
        assert np.array_equal(got, oracle.colors(n, T, k, seed)), (n, T, k, seed)


PATTERNS = {
    "P1": synth.path_pattern(1), "P2": synth.path_pattern(2), "P4": synth.path_pattern(4),
    "C4": synth.cycle_pattern(4), "C5": synth.cycle_pattern(5), "S5": synth.star_pattern(5),
    "K4": synth.clique_pattern(4), "G22": synth.grid_pattern(2, 2), "G23": synth.grid_pattern(2, 3),
    "A": synth.pattern_A(), "B": synth.pattern_B(), "C": synth.pattern_C(), "D": synth.pattern_D(),
    "T3": synth.random_partial_ktree(9, 3, 4), "T2": synth.random_partial_ktree(8, 2, 9),
}


@pytest.mark.parametrize("name", sorted(PATTERNS))
def test_nice_decomposition_matches_oracle(ctx, name):
    nF, e, td = PATTERNS[name]
    pid = cc.cc_load_pattern(ctx.h, nF, e, td)
    assert cc.cc_pattern_nodes(ctx.h, pid, nF) == oracle.nice_td(nF, e, td)


def test_min_width_decomposition(ctx):
    """With no decomposition given the library finds one of minimum width (Table 1 widths)."""
    for pat, tw in [(synth.path_pattern(6), 1), (synth.cycle_pattern(7), 2),
                    (synth.clique_pattern(5), 4), (synth.grid_pattern(3, 3), 3),
                    (synth.grid_pattern(2, 5), 2), (synth.star_pattern(6), 1),
                    (synth.pattern_A(), 1), (synth.pattern_B(), 2), (synth.pattern_C(), 2),
                    (synth.pattern_D(), 2)]:
        nF, e, _ = pat
        pid = cc.cc_load_pattern(ctx.h, nF, e, None)
        assert cc.cc_pattern_info(ctx.h, pid)[1] == tw


def _check_small(ctx, g, pat, colours, k, df, fuse, block=256, tables=True, **opt):
    nF, e, td = pat
    T = colours.shape[0]
    ref = oracle.run_dp(g, pat, colours, k, degree_filter=df)
    r = gpu_dp(ctx, g, pat, colours=colours, k=k, degree_filter=int(df), fuse=int(fuse),
               retain=1, block=block, **opt)
    try:
        assert r["nodes"] == oracle.nice_td(nF, e, td)
        assert np.array_equal(r["count"], ref.count)
        assert np.array_equal(r["exists"], ref.exists)
        assert np.array_equal(r["sizes"], ref.node_sizes.sum(axis=0))
        if tables:
            want = oracle_tables(ref, r["nodes"], T)
            dumped = 0
            for x, nd in enumerate(r["nodes"]):
                try:
                    got = gpu_table(ctx, r, x, len(nd[4]), int(r["sizes"][x]) + 1)
                except cc.CCError as ex:
                    # an introduce fused into its forget, or run in one pass with its parent
                    # introduce (planned runs), stores no table
                    assert ex.code == cc.CC_EINVAL and nd[0] == cc.INTRODUCE
                    assert fuse or cc.cc_run_mode(ctx.h, r["run"]) != "exact"
                    continue
                dumped += 1
                assert got == want[x], (x, nd)
            assert dumped >= len(r["nodes"]) // 2
    finally:
        release(ctx, r)


@pytest.mark.parametrize("name", sorted(PATTERNS))
@pytest.mark.parametrize("fuse", [0, 1, 2])
def test_dp_small_parity(ctx, name, fuse):
    pat = PATTERNS[name]
    nF = pat[0]
    g = synth.erdos_renyi(60, 0.15, 5)
    for k, df in [(nF, True), (nF + 2, False)]:
        k = min(k, 32)
        colours = oracle.colors(60, 3, k, seed=11 + k)
        _check_small(ctx, g, pat, colours, k, df, fuse)


@pytest.mark.parametrize("block", [128, 256, 512])
def test_dp_block_sizes(ctx, block):
    g = synth.barabasi_albert(500, 3, 2)
    pat = synth.grid_pattern(2, 3)
    colours = oracle.colors(500, 4, 6, seed=3)
    for fuse in (0, 1, 2):
        _check_small(ctx, g, pat, colours, 6, True, fuse, block=block)


def test_dp_wide_keys(ctx):
    """k + max_bag * ceil(log2 n) + ceil(log2 trials) > 64: 128-bit keys (14 + 3*17 + 2 bits)."""
    g = synth.erdos_renyi(100000, 2.0 / 99999, 4)
    pat = synth.cycle_pattern(5)
    colours = oracle.colors(100000, 3, 14, seed=8)
    for fuse in (0, 1, 2):
        _check_small(ctx, g, pat, colours, 14, True, fuse, tables=fuse != 1)


@pytest.mark.parametrize("name", ["C4", "C5", "G23", "K4", "T3", "B"])
def test_grouped_equals_plain(ctx, name):
    """Sorting the child by bag-neighbour images and sharing candidate lists changes nothing."""
    pat = PATTERNS[name]
    nF = pat[0]
    g = synth.barabasi_albert(2000, 4, 3)
    colours = oracle.colors(2000, 6, nF, seed=21)
    out = []
    for group in (0, 1):
        r = gpu_dp(ctx, g, pat, colours=colours, k=nF, group=group)
        out.append((r["count"].copy(), r["sizes"].copy()))
        release(ctx, r)
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    ref = oracle.run_dp(g, pat, colours, nF)
    assert np.array_equal(out[1][0], ref.count)


def test_dp_edge_cases(ctx):
    # a single vertex pattern: count = number of vertices (degree 0 passes the filter)
    g = synth.erdos_renyi(50, 0.1, 1)
    z = oracle.colors(50, 2, 1, seed=1)
    _check_small(ctx, g, synth.path_pattern(1), z, 1, True, 0)
    # a graph without edges: only edgeless patterns embed
    g0 = synth.csr_from_edges(30, np.zeros((0, 2), np.int64))
    z = oracle.colors(30, 2, 4, seed=2)
    _check_small(ctx, g0, synth.path_pattern(2), z, 4, True, 0)
    _check_small(ctx, g0, (3, np.zeros((0, 2), np.int32), ([[0], [1], [2]], [1, 2, -1])), z, 4,
                 False, 0)
    # one host vertex, more pattern vertices than host vertices
    g1 = synth.csr_from_edges(1, np.zeros((0, 2), np.int64))
    _check_small(ctx, g1, synth.path_pattern(3), np.zeros((1, 1), np.uint8), 3, True, 1)
    # complete host graph: closed form n_F! * prod(colour class sizes) when k = n_F
    gk = synth.complete_graph(12)
    z = oracle.colors(12, 4, 4, seed=5)
    r = gpu_dp(ctx, gk, synth.cycle_pattern(4), colours=z, k=4)
    for t in range(4):
        assert int(r["count"][t]) == 24 * int(np.prod(np.bincount(z[t], minlength=4)))
    release(ctx, r)


def test_invalid_inputs(ctx):
    rp = np.array([0, 1, 1], np.int32)
    with pytest.raises(cc.CCError) as e:  # asymmetric
        cc.cc_load_graph(ctx.h, rp, np.array([1], np.int32))
    assert e.value.code == cc.CC_EINVAL
    with pytest.raises(cc.CCError):  # self loop
        cc.cc_load_graph(ctx.h, np.array([0, 1], np.int32), np.array([0], np.int32))
    with pytest.raises(cc.CCError):  # unsorted row
        cc.cc_load_graph(ctx.h, *[np.array([0, 2, 3, 4], np.int32), np.array([2, 1, 0, 0], np.int32)])
    nF, e, td = synth.cycle_pattern(5)
    with pytest.raises(cc.CCError):  # decomposition misses an edge
        cc.cc_load_pattern(ctx.h, nF, e, ([[0, 1, 2], [2, 3, 4]], [1, -1]))
    with pytest.raises(cc.CCError):
        cc.cc_load_pattern(ctx.h, 33, [], None)
    g = synth.erdos_renyi(40, 0.1, 1)
    cc.cc_load_graph(ctx.h, *g)
    pid = cc.cc_load_pattern(ctx.h, nF, e, td)
    cid = cc.cc_color(ctx.h, 1, 1, 4)
    with pytest.raises(cc.CCError) as ex:  # k < n_F
        cc.cc_run_dp(ctx.h, pid, cid, cc.cc_default_opts())
    assert ex.value.code == cc.CC_EINVAL
    cc.cc_release_colors(ctx.h, cid)
    # 32 colours, bags of 4, 24-bit vertex ids and 2 trials need 129 bits
    gb = synth.csr_from_edges(1 << 24, np.zeros((0, 2), np.int64))
    cc.cc_load_graph(ctx.h, *gb)
    p4 = cc.cc_load_pattern(ctx.h, *synth.clique_pattern(4)[:2], None)
    cid = cc.cc_color(ctx.h, 1, 2, 32)
    with pytest.raises(cc.CCError) as ex:
        cc.cc_run_dp(ctx.h, p4, cid, cc.cc_default_opts())
    assert ex.value.code == cc.CC_EKEYWIDTH
    # a bag of nine vertices is beyond the kernels' largest bag
    p9 = cc.cc_load_pattern(ctx.h, *synth.clique_pattern(9)[:2], None)
    with pytest.raises(cc.CCError) as ex:
        cc.cc_run_dp(ctx.h, p9, cid, cc.cc_default_opts())
    assert ex.value.code == cc.CC_EKEYWIDTH
    cc.cc_release_colors(ctx.h, cid)


# ---- the benchmark workloads ----------------------------------------------------------------

def test_workload_er200_c5(ctx):
    """Erdos-Renyi n=200, p=0.05 (seed 1); 5-cycle; k=5; Philox seed 7; one trial."""
    w = synth.WORKLOADS["er200_c5"]
    g = synth.make_graph(w["graph"])
    pat = synth.make_pattern(w["pattern"])
    z = oracle.colors(200, 1, 5, w["seed"])
    ref = oracle.run_dp(g, pat, z, 5)
    for fuse in (0, 1, 2):
        r = gpu_dp(ctx, g, pat, seed=w["seed"], trials=1, k=5, fuse=fuse, retain=1)
        assert np.array_equal(r["colours"], z)
        assert np.array_equal(r["count"], ref.count) and int(ref.count[0]) > 0
        assert np.array_equal(r["exists"], ref.exists)
        assert np.array_equal(r["sizes"], ref.node_sizes.sum(axis=0))
        release(ctx, r)


def test_workload_ba20k_grid2x4_sampled(ctx):
    """Barabasi-Albert n=20000, m=4; 2x4 grid; k=8; 64 trials in one run (the benchmark's
    launch configuration).  Two sampled trials against the oracle; every trial's count is a
    multiple of |Aut(G_{2,4})| = 4 and exists agrees with a nonzero count."""
    w = synth.WORKLOADS["ba20k_grid2x4"]
    g = synth.make_graph(w["graph"])
    pat = synth.make_pattern(w["pattern"])
    r = gpu_dp(ctx, g, pat, seed=w["seed"], trials=64, k=8)
    z = oracle.colors(20000, 64, 8, w["seed"])
    assert np.array_equal(r["colours"], z)
    counts, exists = r["count"], r["exists"]
    assert all(int(c) % 4 == 0 for c in counts)
    assert np.array_equal(exists, (counts > 0).astype(np.uint8))
    for t in (0, 63):
        ref = oracle.run_dp(g, pat, z[t:t + 1], 8)
        assert int(counts[t]) == int(ref.count[0]), t
    release(ctx, r)
    # the same trials alone give the same counts (trial batching changes nothing)
    r1 = gpu_dp(ctx, g, pat, colours=z[[5, 40]], k=8)
    assert int(r1["count"][0]) == int(counts[5]) and int(r1["count"][1]) == int(counts[40])
    release(ctx, r1)


def test_workload_er100k_grid3x3_planted(ctx):
    """Erdos-Renyi n=100000, average degree 10 (seed 1); 3x3 grid (treewidth 3, 128-bit keys);
    k=9; 32 trials in one run, enumeration limited to 10^5.  A grid copy is planted on nine
    vertices that trial 0 colours 0..8 (otherwise the expected number of colourful copies is
    about 10^-3 and every count is 0).  Trial 0 against the oracle (count and every node's table
    size); every count is a multiple of |Aut(G_{3,3})| = 8.  The embeddings of all trials are
    those of the trials whose root table is nonempty, so the list (limit 10^5) comes from a run
    that keeps the tables of those trials only (keeping all 32 trials' tables would take about
    100 GB): it is sorted, distinct, valid, colourful in some trial and contains the oracle's
    list of trial 0."""
    w = synth.WORKLOADS["er100k_grid3x3"]
    n, T, k = 100000, 32, 9
    nF, pe, td = synth.make_pattern(w["pattern"])
    rng = np.random.default_rng(5)
    vs = rng.choice(n, size=nF, replace=False)
    g = synth.plant(synth.make_graph(w["graph"]), pe, vs)
    z = oracle.colors(n, T, k, w["seed"])
    z[0, vs] = np.arange(nF, dtype=np.uint8)
    big = cc.Context(arena_bytes=220 << 30)
    try:
        cc.cc_load_graph(big.h, *g)
        pid = cc.cc_load_pattern(big.h, nF, pe, td)
        N, width = cc.cc_pattern_info(big.h, pid)
        assert width == 3
        cid = cc.cc_set_colors(big.h, z, k)
        run = cc.cc_run_dp(big.h, pid, cid, cc.cc_default_opts())
        counts = cc.cc_count(big.h, run, T)
        exists = cc.cc_decide(big.h, run, T)
        cc.cc_release(big.h, run)
        sel = np.nonzero(exists)[0]
        cids = cc.cc_set_colors(big.h, z[sel], k)
        runs = cc.cc_run_dp(big.h, pid, cids, cc.cc_default_opts(retain=1))
        assert np.array_equal(cc.cc_count(big.h, runs, len(sel)), counts[sel])
        lst, total = cc.cc_enumerate(big.h, runs, 100000, nF)
        cc.cc_release(big.h, runs)
        cid0 = cc.cc_set_colors(big.h, z[:1], k)
        run0 = cc.cc_run_dp(big.h, pid, cid0, cc.cc_default_opts())
        sizes0 = cc.cc_table_stats(big.h, run0, N)[0]
        count0 = cc.cc_count(big.h, run0, 1)
        cc.cc_release(big.h, run0)
    finally:
        big.close()
    ref = oracle.run_dp(g, (nF, pe, td), z[:1], k)
    assert int(counts[0]) == int(ref.count[0]) == int(count0[0]) and int(counts[0]) >= 8
    assert np.array_equal(sizes0, ref.node_sizes[0])
    assert all(int(c) % 8 == 0 for c in counts)
    assert np.array_equal(exists, (counts > 0).astype(np.uint8))
    # the list: sorted, distinct, valid and colourful in some trial
    assert total == len(lst) and total >= int(counts[0])
    rows = [tuple(int(x) for x in r) for r in lst]
    assert rows == sorted(set(rows))
    row_ptr, col = g
    for phi in rows:
        assert len(set(phi)) == nF
        for a, b in np.asarray(pe).reshape(-1, 2):
            u, v = phi[a], phi[b]
            assert v in col[row_ptr[u]:row_ptr[u + 1]]
        assert any(len(set(int(z[t, x]) for x in phi)) == nF for t in sel)
    want = {tuple(int(x) for x in r) for r in ref.enumerate(100000)[0]}
    assert want <= set(rows)


def test_planned_runs_match_exact(ctx):
    """A second run of the same pattern, graph, trials and colours uses the capacities planned
    by the first (no count passes): results and table sizes are unchanged."""
    g = synth.barabasi_albert(3000, 4, 7)
    for pat in (synth.grid_pattern(2, 3), synth.pattern_B(), synth.random_partial_ktree(8, 2, 9)):
        nF = pat[0]
        pid = cc.cc_load_pattern(ctx.h, *pat)
        for rep in range(3):
            colours = oracle.colors(3000, 4, nF, seed=40 + (rep % 2))
            want = oracle.run_dp(g, pat, colours, nF)
            for fuse in (0, 1, 2):
                r = gpu_dp(ctx, g, pat, colours=colours, k=nF, fuse=fuse, pid=pid)
                assert cc.cc_run_mode(ctx.h, r["run"]) == ("exact" if rep == 0 else "planned")
                assert np.array_equal(r["count"], want.count)
                assert np.array_equal(r["sizes"], want.node_sizes.sum(axis=0))
                release(ctx, r)


def test_planned_overflow_falls_back(ctx):
    """Capacities planned on a colouring with tiny tables are too small for a random one; the
    run notices, plans again exactly and still returns the oracle's results."""
    g = synth.barabasi_albert(3000, 4, 8)
    pat = synth.grid_pattern(2, 3)
    mono = np.zeros((4, 3000), np.uint8)  # one colour: no colourful edge at all
    colours = oracle.colors(3000, 4, 6, seed=9)
    ref = oracle.run_dp(g, pat, colours, 6)
    for fuse in (1, 2, 0):
        pid = cc.cc_load_pattern(ctx.h, *pat)
        r = gpu_dp(ctx, g, pat, colours=mono, k=6, fuse=fuse, pid=pid)
        assert int(r["count"].sum()) == 0
        release(ctx, r)
        for want in ("exact", "planned"):  # the tiny plan overflows and is redone exactly
            r = gpu_dp(ctx, g, pat, colours=colours, k=6, fuse=fuse, pid=pid)
            assert cc.cc_run_mode(ctx.h, r["run"]) == want
            assert np.array_equal(r["count"], ref.count)
            assert np.array_equal(r["sizes"], ref.node_sizes.sum(axis=0))
            release(ctx, r)


@pytest.mark.parametrize("name", ["C4", "C5", "G23", "K4", "A", "B", "T3", "T2", "P4"])
@pytest.mark.parametrize("bits", [0, 1])
def test_bucketed_merge_small_parity(ctx, name, bits):
    """The bucketed forget merge (sort_sweep 3) gives the oracle's tables entry by entry, its
    counts and its enumeration (binary search in the bucketed order), both with buckets sized
    to shared memory (bits 0) and with two buckets far larger than shared memory, which are
    sorted in global scratch (bits 1)."""
    pat = PATTERNS[name]
    nF = pat[0]
    g = synth.erdos_renyi(60, 0.15, 5)
    colours = oracle.colors(60, 3, nF, seed=11 + nF)
    _check_small(ctx, g, pat, colours, nF, True, 2, sort_sweep=3, part_bits=bits)
    r = gpu_dp(ctx, g, pat, colours=colours, k=nF, fuse=2, retain=1, sort_sweep=3,
               part_bits=bits)
    ref = oracle.run_dp(g, pat, colours, nF)
    try:
        got, tot = cc.cc_enumerate(ctx.h, r["run"], 10 ** 6, nF)
        want, wtot, _ = ref.enumerate(10 ** 6)
        assert np.array_equal(got, want) and tot == wtot
    finally:
        release(ctx, r)


def test_bucketed_merge_at_scale(ctx):
    """The bucketed merge on the 64-trial Barabasi-Albert 2x4-grid step shape at reduced size
    (n=20000, 4 trials): two-level splits, exact then planned, equal to the one-sweep sort's
    tables and counts and to the oracle on two trials; and with two bucket bits, every bucket
    far beyond shared memory."""
    w = synth.WORKLOADS["ba20k_grid2x4"]
    g = synth.make_graph(w["graph"])
    pat = synth.make_pattern(w["pattern"])
    z = oracle.colors(20000, 4, 8, seed=7)
    base = gpu_dp(ctx, g, pat, colours=z, k=8)
    want = (base["count"].copy(), base["sizes"].copy())
    release(ctx, base)
    pid = cc.cc_load_pattern(ctx.h, *pat)
    for bits in (0, 0, 2):
        r = gpu_dp(ctx, g, pat, colours=z, k=8, pid=pid, sort_sweep=3, part_bits=bits)
        assert np.array_equal(r["count"], want[0])
        assert np.array_equal(r["sizes"], want[1])
        release(ctx, r)
    ref = oracle.run_dp(g, pat, z[:2], 8)
    assert np.array_equal(want[0][:2], ref.count)


@pytest.mark.parametrize("sweep", [0, 1, 2, 3])
def test_sort_variants_agree(ctx, sweep):
    """Every radix-sort schedule (separate histogram passes; one-sweep with look-back; one-sweep
    with the next tile brought in by bulk copy) gives the oracle's tables, with 64- and 128-bit
    keys."""
    g = synth.barabasi_albert(4000, 4, 12)
    for pat, k, T in ((synth.grid_pattern(2, 3), 6, 5), (synth.cycle_pattern(5), 12, 3)):
        colours = oracle.colors(4000, T, k, seed=77)
        r = gpu_dp(ctx, g, pat, colours=colours, k=k, fuse=2, sort_sweep=sweep)
        ref = oracle.run_dp(g, pat, colours, k)
        assert np.array_equal(r["count"], ref.count)
        assert np.array_equal(r["sizes"], ref.node_sizes.sum(axis=0))
        release(ctx, r)


def test_planned_at_workload_scale(ctx):
    """Planned runs on the workload's graph (hubs of degree ~500, long candidate lists, ragged
    last windows), against the oracle on two trials."""
    w = synth.WORKLOADS["ba20k_grid2x4"]
    g = synth.make_graph(w["graph"])
    pat = synth.make_pattern(w["pattern"])
    z = oracle.colors(20000, 2, 8, seed=3)
    ref = oracle.run_dp(g, pat, z, 8)
    for fuse in (2, 1):
        pid = cc.cc_load_pattern(ctx.h, *pat)
        for want in ("exact", "planned"):
            r = gpu_dp(ctx, g, pat, colours=z, k=8, fuse=fuse, pid=pid)
            assert cc.cc_run_mode(ctx.h, r["run"]) == want
            assert np.array_equal(r["count"], ref.count)
            assert np.array_equal(r["sizes"], ref.node_sizes.sum(axis=0))
            release(ctx, r)


def test_allowed_mappings_match_oracle(ctx):
    """Patterns with allowed-mapping masks (Section 3.2, masking unprofitable mappings): counts,
    table sizes, planned reruns and the enumeration equal the oracle's with the same masks, for
    every forget scheme; the masks belong to the graph they were given for."""
    n = 1500
    g = synth.barabasi_albert(n, 4, 17)
    rng = np.random.default_rng(3)
    cc.cc_load_graph(ctx.h, *g)
    fewer = False
    for pat in (synth.cycle_pattern(5), synth.pattern_B(), synth.grid_pattern(2, 3)):
        nF, e, td = pat
        bits = (rng.random((n, nF)) < 0.6).astype(np.uint32)
        allow = (bits << np.arange(nF, dtype=np.uint32)).sum(axis=1).astype(np.uint32)
        z = oracle.colors(n, 3, nF, seed=8)
        ref = oracle.run_dp(g, pat, z, nF, allow=allow)
        fewer = fewer or int(ref.count.sum()) < int(oracle.run_dp(g, pat, z, nF).count.sum())
        want_list = ref.enumerate(100000)[0]
        pid = cc.cc_load_pattern_masked(ctx.h, nF, e, td, allow)
        cid = cc.cc_set_colors(ctx.h, z, nF)
        N, _ = cc.cc_pattern_info(ctx.h, pid)
        for fuse in (2, 1, 0):
            for want_mode in ("exact", "planned"):
                run = cc.cc_run_dp(ctx.h, pid, cid, cc.cc_default_opts(fuse=fuse))
                assert cc.cc_run_mode(ctx.h, run) == want_mode
                assert np.array_equal(cc.cc_count(ctx.h, run, 3), ref.count)
                assert np.array_equal(cc.cc_table_stats(ctx.h, run, N)[0],
                                      ref.node_sizes.sum(axis=0))
                cc.cc_release(ctx.h, run)
        run = cc.cc_run_dp(ctx.h, pid, cid, cc.cc_default_opts(retain=1))
        lst, tot = cc.cc_enumerate(ctx.h, run, 100000, nF)
        assert np.array_equal(lst, want_list)
        cc.cc_release(ctx.h, run)
        cc.cc_release_colors(ctx.h, cid)
    assert fewer  # the masks removed embeddings
    # another graph: the masked pattern no longer runs
    cc.cc_load_graph(ctx.h, *synth.barabasi_albert(n, 3, 18))
    cid = cc.cc_color(ctx.h, 1, 1, 6)
    with pytest.raises(cc.CCError) as err:
        cc.cc_run_dp(ctx.h, pid, cid, cc.cc_default_opts())
    assert err.value.code == -1
    cc.cc_release_colors(ctx.h, cid)


def test_bounded_wait_times_out_and_context_survives(ctx):
    """Failure detection without a fault: a device wait on a word that nothing sets gives up
    after its bound and reports CC_ETIMEOUT through the error word; the context then runs a DP
    to the oracle's result."""
    import time

    t0 = time.time()
    assert cc.cc_probe_bounded_wait(ctx.h, 1 << 16) == -4
    assert time.time() - t0 < 30
    w = synth.WORKLOADS["er200_c5"]
    g = synth.make_graph(w["graph"])
    pat = synth.make_pattern(w["pattern"])
    r = gpu_dp(ctx, g, pat, seed=w["seed"], trials=1, k=5)
    ref = oracle.run_dp(g, pat, oracle.colors(200, 1, 5, w["seed"]), 5)
    assert np.array_equal(r["count"], ref.count)
    release(ctx, r)


@pytest.mark.parametrize("fuse", [2, 1, 0])
def test_distance_bound_matches_oracle(ctx, fuse):
    """distance_prune (Section 3.2, mapping expansion): an introduced vertex with no bag
    neighbour takes only the ball of radius dist_F(w, u) around the image of its nearest bag
    vertex w (distances 2, 3 and 4 here).  Counts, table sizes (exact and planned) and the
    enumeration equal the oracle's with the same bound; the root equals the unbounded run's."""
    n = 300
    g = synth.erdos_renyi(n, 6.0 / n, 12)
    path = lambda m: np.array([(i, i + 1) for i in range(m - 1)], np.int32)  # noqa: E731
    pats = [(3, path(3), ([[0, 2], [0, 1, 2]], [1, -1])),
            (4, path(4), ([[0, 3], [0, 1, 3], [1, 2, 3]], [1, 2, -1])),
            (5, path(5), ([[0, 4], [0, 1, 4], [1, 2, 4], [2, 3, 4]], [1, 2, 3, -1])),
            synth.random_partial_ktree(8, 3, 4), synth.random_partial_ktree(7, 3, 2)]
    cc.cc_load_graph(ctx.h, *g)
    shrunk = False
    for pat in pats:
        nF = pat[0]
        z = oracle.colors(n, 2, nF, seed=31)
        ref = oracle.run_dp(g, pat, z, nF, distance_prune=True)
        plain = oracle.run_dp(g, pat, z, nF)
        assert np.array_equal(ref.count, plain.count)
        shrunk = shrunk or int(ref.node_sizes.sum()) < int(plain.node_sizes.sum())
        pid = cc.cc_load_pattern(ctx.h, *pat)
        cid = cc.cc_set_colors(ctx.h, z, nF)
        N, _ = cc.cc_pattern_info(ctx.h, pid)
        for want in ("exact", "planned"):
            run = cc.cc_run_dp(ctx.h, pid, cid, cc.cc_default_opts(fuse=fuse, distance_prune=1))
            assert cc.cc_run_mode(ctx.h, run) == want
            assert np.array_equal(cc.cc_count(ctx.h, run, 2), ref.count)
            assert np.array_equal(cc.cc_table_stats(ctx.h, run, N)[0], ref.node_sizes.sum(axis=0))
            cc.cc_release(ctx.h, run)
        run = cc.cc_run_dp(ctx.h, pid, cid, cc.cc_default_opts(retain=1, distance_prune=1))
        lst, _ = cc.cc_enumerate(ctx.h, run, 10 ** 6, nF)
        assert np.array_equal(lst, ref.enumerate(10 ** 6)[0])
        cc.cc_release(ctx.h, run)
        cc.cc_release_colors(ctx.h, cid)
    assert shrunk
