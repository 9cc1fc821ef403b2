"""GPU reconstruction (Section 4) against the oracle: the sorted, repeat-free union over trials of
all colourful embeddings, truncated to a limit, must equal the oracle's list row for row."""
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


def gpu_enum(ctx, g, pat, colours, k, limit, **opt):
    nF, e, td = pat
    cc.cc_load_graph(ctx.h, *g)
    pid = cc.cc_load_pattern(ctx.h, nF, e, td)
    cid = cc.cc_set_colors(ctx.h, colours, k)
    run = cc.cc_run_dp(ctx.h, pid, cid, cc.cc_default_opts(retain=1, **opt))
    try:
        rows, total = cc.cc_enumerate(ctx.h, run, limit, nF)
        counts = cc.cc_count(ctx.h, run, colours.shape[0])
    finally:
        cc.cc_release(ctx.h, run)
        cc.cc_release_colors(ctx.h, cid)
    return rows, total, counts


PATS = {
    "C4": synth.cycle_pattern(4), "C5": synth.cycle_pattern(5), "P4": synth.path_pattern(4),
    "S5": synth.star_pattern(5), "G23": synth.grid_pattern(2, 3), "K4": synth.clique_pattern(4),
    "A": synth.pattern_A(), "B": synth.pattern_B(), "D": synth.pattern_D(),
    "T3": synth.random_partial_ktree(8, 3, 4), "T2": synth.random_partial_ktree(8, 2, 9),
    "P1": synth.path_pattern(1),
}


@pytest.mark.parametrize("name", sorted(PATS))
@pytest.mark.parametrize("fuse", [0, 1, 2])
def test_enumerate_small(ctx, name, fuse):
    pat = PATS[name]
    nF = pat[0]
    g = synth.erdos_renyi(36, 0.22, 3)
    colours = oracle.colors(36, 3, nF, seed=5 + nF)
    ref = oracle.run_dp(g, pat, colours, nF)
    want, want_total, _ = ref.enumerate(10 ** 7)
    rows, total, counts = gpu_enum(ctx, g, pat, colours, nF, 10 ** 6, fuse=fuse)
    assert np.array_equal(counts, ref.count)
    assert total == want_total
    assert np.array_equal(rows, want)
    # truncation keeps the lexicographically smallest
    rows5, total5, _ = gpu_enum(ctx, g, pat, colours, nF, 5, fuse=fuse)
    assert total5 == want_total and np.array_equal(rows5, want[:5])


def test_enumerate_with_more_colours_and_no_filter(ctx):
    pat = synth.pattern_B()
    g = synth.erdos_renyi(30, 0.25, 8)
    colours = oracle.colors(30, 2, 9, seed=3)
    ref = oracle.run_dp(g, pat, colours, 9, degree_filter=False)
    want, want_total, _ = ref.enumerate(10 ** 7)
    rows, total, _ = gpu_enum(ctx, g, pat, colours, 9, 10 ** 6, degree_filter=0)
    assert total == want_total and np.array_equal(rows, want)


def test_enumerate_workload_er200_c5(ctx):
    """Erdos-Renyi n=200, p=0.05; 5-cycle; k=5; Philox seed 7: the full sorted list."""
    g = synth.erdos_renyi(200, 0.05, 1)
    pat = synth.cycle_pattern(5)
    colours = oracle.colors(200, 1, 5, 7)
    ref = oracle.run_dp(g, pat, colours, 5)
    want, want_total, _ = ref.enumerate(10 ** 6)
    rows, total, counts = gpu_enum(ctx, g, pat, colours, 5, 10 ** 5)
    assert total == want_total == int(counts[0]) == 4000
    assert np.array_equal(rows, want)


def test_enumerate_requires_kept_tables(ctx):
    g = synth.erdos_renyi(30, 0.2, 1)
    nF, e, td = synth.cycle_pattern(4)
    cc.cc_load_graph(ctx.h, *g)
    pid = cc.cc_load_pattern(ctx.h, nF, e, td)
    cid = cc.cc_color(ctx.h, 1, 1, 4)
    run = cc.cc_run_dp(ctx.h, pid, cid, cc.cc_default_opts(retain=0))
    with pytest.raises(cc.CCError) as ex:
        cc.cc_enumerate(ctx.h, run, 10, nF)
    assert ex.value.code == cc.CC_EINVAL
    cc.cc_release(ctx.h, run)
    cc.cc_release_colors(ctx.h, cid)


@pytest.mark.parametrize("name", ["C4", "C5", "G23", "K4", "B", "T2"])
def test_enumerate_vertex_sets(ctx, name):
    """Occurrences counted by vertex set (Section 5.2's switch): the distinct image sets of the
    oracle's embeddings, sorted; fewer than the embeddings whenever F has automorphisms."""
    pat = PATS[name]
    nF, e, td = pat
    g = synth.erdos_renyi(36, 0.3, 11)
    colours = oracle.colors(36, 4, nF, seed=17)
    ref = oracle.run_dp(g, pat, colours, nF)
    emb, total, _ = ref.enumerate(10 ** 7)
    want = sorted({tuple(sorted(int(v) for v in r)) for r in emb})
    cc.cc_load_graph(ctx.h, *g)
    pid = cc.cc_load_pattern(ctx.h, nF, e, td)
    cid = cc.cc_set_colors(ctx.h, colours, nF)
    run = cc.cc_run_dp(ctx.h, pid, cid, cc.cc_default_opts(retain=1))
    try:
        sets, nsets = cc.cc_enumerate_sets(ctx.h, run, 10 ** 6, nF)
        assert nsets == len(want) and [tuple(int(v) for v in r) for r in sets] == want
        if len(want) > 3:
            few, n2 = cc.cc_enumerate_sets(ctx.h, run, 3, nF)
            assert n2 == len(want) and [tuple(int(v) for v in r) for r in few] == want[:3]
        if total:
            assert nsets < total  # every pattern here has a nontrivial automorphism
    finally:
        cc.cc_release(ctx.h, run)
        cc.cc_release_colors(ctx.h, cid)
