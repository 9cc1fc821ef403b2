"""Chained introduces (run option `chain`, on by default).

An introduce x1 whose only consumer is an introduce x2 of a vertex not adjacent to x1's runs in
one pass with it in planned runs: each entry of x1's child y yields x1's entries (Section 3.1,
introduce rule), which are counted and at once extended by x2's candidates, shared by the run of
y entries with equal images of x2's bag neighbours (Section 3.2, mapping expansion).  x1's table
is never stored; its size is still counted and the reconstruction (Section 4) resolves
introduce nodes by their rule.  These tests require the chained run to give the oracle's
counts, every node's size, every stored table entry by entry and the same enumeration as the
unchained run, on patterns where x2's candidates are often present."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_1908_11248_gb300 as cc
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__

    __graft_entry__.build()
    c = cc.Context(arena_bytes=16 << 30)
    yield c
    c.close()


# (graph, pattern, k): dense Erdos-Renyi graphs with the 3x3 and 3x4 grids and two random
# partial 3-trees, each with a chainable introduce pair over a forget's (sorted) table; the upper
# introduce's entries are many (nonzero counts for the grids and the 9-vertex tree)
CASES = {
    "er200_grid33": (("er", 200, 0.08, 3), ("grid", 3, 3), 9),
    "er120_grid34": (("er", 120, 0.08, 7), ("grid", 3, 4), 12),
    "er150_ktree9": (("er", 150, 0.08, 5), ("ktree", 9, 3, 7003), 9),
    "er150_ktree8": (("er", 150, 0.08, 6), ("ktree", 8, 3, 7030), 8),
}


def chain_pairs(nodes, pat):
    """(x1, x2) pairs of the nice decomposition that the option may run together: x1 and its
    parent x2 introduce non-adjacent vertices, x1's vertex has a bag neighbour in x1's child and
    x2's has at least two."""
    nF, edges, _ = pat
    adj = [set() for _ in range(nF)]
    for a, b in np.asarray(edges).tolist():
        adj[a].add(b)
        adj[b].add(a)
    parent = {}
    for i, nd in enumerate(nodes):
        for ch in (nd[1], nd[2]):
            if ch >= 0:
                parent[ch] = i
    out = []
    for x1, (t, c0, _, u1, _) in enumerate(nodes):
        if t != cc.INTRODUCE or x1 not in parent:
            continue
        x2 = parent[x1]
        t2, _, _, u2, _ = nodes[x2]
        if t2 != cc.INTRODUCE or u1 in adj[u2]:
            continue
        ybag = nodes[c0][4]
        if sum(w in adj[u1] for w in ybag) >= 1 and sum(w in adj[u2] for w in ybag) >= 2:
            out.append((x1, x2))
    return out


def tables_of(ctx, run, nodes, sizes):
    out = {}
    for x, nd in enumerate(nodes):
        try:
            tr, phi, mask, cnt = cc.cc_table_dump(ctx.h, run, x, int(sizes[x]) + 1, len(nd[4]))
        except cc.CCError as ex:
            assert ex.code == cc.CC_EINVAL and nd[0] == cc.INTRODUCE
            out[x] = None
            continue
        out[x] = {(int(tr[i]), tuple(int(v) for v in phi[i]), int(mask[i])): int(cnt[i])
                  for i in range(len(mask))}
    return out


@pytest.mark.parametrize("name", sorted(CASES))
def test_chained_introduces_match_oracle(ctx, name):
    gspec, pspec, k = CASES[name]
    g = synth.make_graph(gspec)
    pat = synth.make_pattern(pspec)
    nF = pat[0]
    n = len(g[0]) - 1
    z = oracle.colors(n, 3, k, seed=21)
    ref = oracle.run_dp(g, pat, z, k)
    want_rows = ref.enumerate(1 << 20)[0]
    cc.cc_load_graph(ctx.h, *g)
    pid = cc.cc_load_pattern(ctx.h, *pat)
    N, _ = cc.cc_pattern_info(ctx.h, pid)
    nodes = cc.cc_pattern_nodes(ctx.h, pid, nF)
    pairs = chain_pairs(nodes, pat)
    assert pairs, "the case must have a chainable pair"
    cid = cc.cc_set_colors(ctx.h, z, k)
    got = {}
    for chain in (1, 0):
        for rep in range(2):  # the first run of a key is exact and plans the second
            o = cc.cc_default_opts(retain=1, profile=1, chain=chain)
            run = cc.cc_run_dp(ctx.h, pid, cid, o)
            mode = cc.cc_run_mode(ctx.h, run)
            counts = cc.cc_count(ctx.h, run, 3)
            sizes = cc.cc_table_stats(ctx.h, run, N)[0]
            assert np.array_equal(counts, ref.count), (chain, rep)
            assert np.array_equal(sizes, ref.node_sizes.sum(axis=0)), (chain, rep)
            if rep == 1:
                assert mode == "planned"
                node, kind, _, _ = cc.cc_run_timings(ctx.h, run)
                kinds = {(int(a), cc.KERNEL_KINDS[int(b)]) for a, b in zip(node, kind)}
                chained = {x2 for x1, x2 in pairs if (x2, "intro_chain") in kinds}
                if chain:
                    assert chained, "no introduce pair ran chained"
                else:
                    assert not chained
                tabs = tables_of(ctx, run, nodes, sizes)
                rows = cc.cc_enumerate(ctx.h, run, 1 << 20, nF)[0]
                got[chain] = (tabs, rows, chained)
            cc.cc_release(ctx.h, run)
    cc.cc_release_colors(ctx.h, cid)
    tab1, rows1, chained = got[1]
    tab0, rows0, _ = got[0]
    # every table the chained run stored equals the unchained run's and the oracle's; the
    # lower introduce of every chained pair stored none
    lower = {x1 for x1, x2 in pairs if x2 in chained}
    for x, nd in enumerate(nodes):
        if x in lower:
            assert tab1[x] is None
        if tab1[x] is None:
            continue
        want = {}
        for t in range(3):
            phi, mask, cnt = ref.table(t, x, len(nd[4]))
            for i in range(len(mask)):
                want[(t, tuple(int(v) for v in phi[i]), int(mask[i]))] = int(cnt[i])
        assert tab1[x] == want, (name, x)
        if tab0[x] is not None:
            assert tab0[x] == tab1[x]
    assert np.array_equal(rows1, rows0)
    assert np.array_equal(rows1, want_rows)


def test_chained_introduces_at_workload_scale(ctx):
    """Erdos-Renyi n=100000, average degree 10, the 3x3 grid, k=9, 4 trials with a planted grid
    copy coloured 0..8 in trial 0: chained and unchained planned runs give the same counts and
    table sizes (the unchained path is checked against the oracle by the workload tests)."""
    w = synth.WORKLOADS["er100k_grid3x3"]
    n, T, k = 100000, 4, 9
    nF, pe, td = synth.make_pattern(w["pattern"])
    rng = np.random.default_rng(5)
    vs = rng.choice(n, size=nF, replace=False)
    g = synth.plant(synth.make_graph(w["graph"]), pe, vs)
    z = oracle.colors(n, T, k, w["seed"])
    z[0, vs] = np.arange(nF, dtype=np.uint8)
    cc.cc_load_graph(ctx.h, *g)
    pid = cc.cc_load_pattern(ctx.h, nF, pe, td)
    N, _ = cc.cc_pattern_info(ctx.h, pid)
    cid = cc.cc_set_colors(ctx.h, z, k)
    res = {}
    for chain in (0, 1):
        for rep in range(2):
            run = cc.cc_run_dp(ctx.h, pid, cid, cc.cc_default_opts(chain=chain, profile=1))
            if rep == 1:
                node, kind, _, _ = cc.cc_run_timings(ctx.h, run)
                used = any(cc.KERNEL_KINDS[int(b)] == "intro_chain" for b in kind)
                assert used == bool(chain)
                res[chain] = (cc.cc_count(ctx.h, run, T), cc.cc_table_stats(ctx.h, run, N)[0])
            cc.cc_release(ctx.h, run)
    cc.cc_release_colors(ctx.h, cid)
    assert np.array_equal(res[0][0], res[1][0])
    assert np.array_equal(res[0][1], res[1][1])
    assert int(res[1][0][0]) > 0  # the planted copy
    assert all(int(c) % 8 == 0 for c in res[1][0])  # |Aut(G_{3,3})| = 8 divides every count
