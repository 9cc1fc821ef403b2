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


def test_noalloc_allocates_nothing(built):
    """The point of the entry point: once a first call on the device has run (it looks up the
    array's address and loads its kernels), further calls leave the device's free memory as it
    was."""
    import torch

    stream = torch.cuda.current_stream().cuda_stream
    g, pat = synth.erdos_renyi(200, 0.05, 1), synth.cycle_pattern(5)
    first = cc.cc_count_noalloc(0, stream, *g, pat[0], pat[1], pat[2], 7, 3, 5)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(0)[0]
    for _ in range(3):
        again = cc.cc_count_noalloc(0, stream, *g, pat[0], pat[1], pat[2], 7, 3, 5)
        assert np.array_equal(again[0], first[0]) and np.array_equal(again[1], first[1])
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(0)[0] == free0


def test_noalloc_refuses_a_capturing_stream(built):
    """The call copies from host memory and waits for its stream, which a stream being captured
    into a CUDA graph cannot do: it returns CC_EINVAL at once and leaves the capture intact."""
    import torch

    g, pat = synth.erdos_renyi(200, 0.05, 1), synth.cycle_pattern(5)
    x = torch.zeros(16, device="cuda")
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        x.add_(1.0)
        with pytest.raises(cc.CCError) as ex:
            cc.cc_count_noalloc(0, side.cuda_stream, *g, pat[0], pat[1], pat[2], 7, 3, 5)
    assert ex.value.code == cc.CC_EINVAL
    graph.replay()
    torch.cuda.synchronize()
    assert float(x[0]) == 1.0


def test_noalloc_rejects_oversized_input(built):
    import torch

    stream = torch.cuda.current_stream().cuda_stream
    empty = np.zeros((0, 2), np.int32)
    # n = 4 Mi isolated vertices and 16 trials: row pointers 16 MiB, degree bytes 4 MiB and
    # colours 64 MiB exceed the 64 MiB array before any table is made
    g = synth.csr_from_edges(1 << 22, np.zeros((0, 2), np.int64))
    with pytest.raises(cc.CCError) as ex:
        cc.cc_count_noalloc(0, stream, *g, 1, empty, None, 1, 16, 1)
    assert ex.value.code == cc.CC_ENOMEM
    # with 8 trials the graph and colours fit (52 MiB), but the leaf table (16 bytes per vertex
    # and trial, 512 MiB) does not: the dynamic programme reports CC_ENOMEM
    with pytest.raises(cc.CCError) as ex:
        cc.cc_count_noalloc(0, stream, *g, 1, empty, None, 1, 8, 1)
    assert ex.value.code == cc.CC_ENOMEM
    # the array is still usable afterwards
    g2, pat = synth.erdos_renyi(200, 0.05, 1), synth.cycle_pattern(5)
    want_c, want_e = allocating_count(g2, pat, 7, 3, 5)
    got_c, got_e = cc.cc_count_noalloc(0, stream, *g2, pat[0], pat[1], pat[2], 7, 3, 5)
    assert np.array_equal(got_c, want_c) and np.array_equal(got_e, want_e)
