"""The serving loop: queries submitted while others run give, bit for bit, what the same query
gives alone through the plain calls (cc_color, cc_run_dp, cc_count, cc_decide) and what the CPU
oracle gives for the same Philox colouring; admission keeps the memory held under the budget.
"""
from __future__ import annotations

import time

import numpy as np
import pytest

import oracle
import synth

cc = pytest.importorskip("paper_1908_11248_gb300")
pytestmark = pytest.mark.gpu

N = 3000


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__

    __graft_entry__.build()
    c = cc.Context(arena_bytes=8 << 30)
    yield c
    c.close()


@pytest.fixture(scope="module")
def graph():
    return synth.barabasi_albert(N, 4, 11)


PATTERNS = [synth.path_pattern(4), synth.cycle_pattern(5), synth.grid_pattern(2, 3),
            synth.pattern_B(), synth.star_pattern(5), synth.random_partial_ktree(6, 2, 4)]


def _queries(nq, seed):
    """A seeded mix: (pattern index, colouring seed, trials, k)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(nq):
        p = int(rng.integers(0, len(PATTERNS)))
        nF = PATTERNS[p][0]
        k = nF + int(rng.integers(0, 2))
        out.append((p, int(rng.integers(1, 1 << 40)), int(rng.integers(1, 3)), k))
    return out


def _wait(ctx, tickets, trials, timeout=120.0):
    res, t0 = {}, time.time()
    while len(res) < len(tickets):
        for i, t in enumerate(tickets):
            if i in res:
                continue
            done, status, counts, exists, lat, _ = cc.cc_serve_poll(ctx.h, t, trials[i])
            if done:
                res[i] = (status, counts, exists, lat)
        assert time.time() - t0 < timeout, "served queries did not finish"
        time.sleep(0.001)
    return [res[i] for i in range(len(tickets))]


def _plain(ctx, pid, seed, trials, k):
    cid = cc.cc_color(ctx.h, seed, trials, k)
    run = cc.cc_run_dp(ctx.h, pid, cid, cc.cc_default_opts())
    out = cc.cc_count(ctx.h, run, trials), cc.cc_decide(ctx.h, run, trials)
    cc.cc_release(ctx.h, run)
    cc.cc_release_colors(ctx.h, cid)
    return out


def test_served_equals_alone_and_oracle(ctx, graph):
    """Two bursts of 48 queries: the first plans every (pattern, trials, k), the second runs
    planned with several queries at once.  Every result equals the same query run alone through
    the plain calls, and a sample equals the oracle."""
    cc.cc_load_graph(ctx.h, *graph)
    pids = [cc.cc_load_pattern(ctx.h, *p) for p in PATTERNS]
    first = _queries(48, 1)
    second = [(p, s + 7, T, k) for p, s, T, k in first]
    cc.cc_serve_start(ctx.h, 0, 6)
    res = []
    for qs in (first, second):
        tickets = [cc.cc_serve_submit(ctx.h, pids[p], s, T, k) for p, s, T, k in qs]
        res += _wait(ctx, tickets, [q[2] for q in qs])
    stats = cc.cc_serve_stats(ctx.h)
    cc.cc_serve_stop(ctx.h)
    assert stats["submitted"] == stats["completed"] == 96
    assert stats["inflight_max"] >= 2  # queries overlapped on the device
    assert stats["exact_runs"] <= 48
    qs = first + second
    for (p, s, T, k), (status, counts, exists, lat) in zip(qs, res):
        assert status == 0 and lat > 0
        want_c, want_e = _plain(ctx, pids[p], s, T, k)
        assert np.array_equal(counts, want_c) and np.array_equal(exists, want_e)
    for (p, s, T, k), (status, counts, exists, lat) in list(zip(qs, res))[40:56]:
        ref = oracle.run_dp(graph, PATTERNS[p], oracle.colors(N, T, k, s), k)
        assert np.array_equal(counts, ref.count) and np.array_equal(exists, ref.exists)


def test_budget_bounds_reserved_memory(ctx, graph):
    """With a budget a few times one query's tables, admission keeps the memory held at once
    under it and the results stay those of the plain calls."""
    cc.cc_load_graph(ctx.h, *graph)
    pat = synth.grid_pattern(2, 3)
    pid = cc.cc_load_pattern(ctx.h, *pat)
    budget = 256 << 20
    cc.cc_serve_start(ctx.h, budget, 8)
    seeds = list(range(100, 124))
    tickets = [cc.cc_serve_submit(ctx.h, pid, s, 2, 6) for s in seeds]
    res = _wait(ctx, tickets, [2] * len(seeds))
    stats = cc.cc_serve_stats(ctx.h)
    cc.cc_serve_stop(ctx.h)
    assert stats["reserved_max"] <= budget
    for s, (status, counts, exists, _) in zip(seeds, res):
        assert status == 0
        want_c, want_e = _plain(ctx, pid, s, 2, 6)
        assert np.array_equal(counts, want_c) and np.array_equal(exists, want_e)


def test_serving_errors_and_busy(ctx, graph):
    """Bad queries fail alone with their status; other calls on a serving context are refused;
    tickets are handed out once; stopping twice is harmless."""
    cc.cc_load_graph(ctx.h, *graph)
    pid = cc.cc_load_pattern(ctx.h, *synth.cycle_pattern(5))
    cc.cc_serve_start(ctx.h, 0, 2)
    with pytest.raises(cc.CCError) as e:
        cc.cc_serve_start(ctx.h, 0, 2)
    assert e.value.code == -8
    with pytest.raises(cc.CCError) as e:
        cc.cc_color(ctx.h, 1, 1, 5)
    assert e.value.code == -8
    pid2 = cc.cc_load_pattern(ctx.h, *synth.path_pattern(3))  # allowed while serving
    t_bad = cc.cc_serve_submit(ctx.h, 999999, 1, 1, 5)
    t_k = cc.cc_serve_submit(ctx.h, pid, 1, 1, 4)  # k < n_F
    t_ok = cc.cc_serve_submit(ctx.h, pid2, 3, 2, 3)
    res = _wait(ctx, [t_bad, t_k, t_ok], [1, 1, 2])
    assert res[0][0] == -6 and res[1][0] == -1 and res[2][0] == 0
    with pytest.raises(cc.CCError):
        cc.cc_serve_poll(ctx.h, t_ok, 2)  # already handed out
    with pytest.raises(cc.CCError):
        cc.cc_serve_submit(ctx.h, pid, 1, 0, 5)  # trials < 1
    cc.cc_serve_stop(ctx.h)
    cc.cc_serve_stop(ctx.h)
    with pytest.raises(cc.CCError):
        cc.cc_serve_submit(ctx.h, pid, 1, 1, 5)
    want_c, _ = _plain(ctx, pid2, 3, 2, 3)
    assert np.array_equal(res[2][1], want_c)


def test_served_enumeration_equals_alone_and_oracle(ctx, graph):
    """Queries with a limit reconstruct their embeddings (Section 4) inside the server: the rows
    equal cc_enumerate of the same query run alone with its tables kept, and the oracle's."""
    cc.cc_load_graph(ctx.h, *graph)
    pats = [synth.cycle_pattern(4), synth.path_pattern(3), synth.grid_pattern(2, 2)]
    pids = [cc.cc_load_pattern(ctx.h, *p) for p in pats]
    qs = [(i % 3, 500 + i, 1 + i % 2, pats[i % 3][0], [0, 50, 10 ** 6][i % 3]) for i in range(9)]
    cc.cc_serve_start(ctx.h, 0, 4)
    tickets = [cc.cc_serve_submit(ctx.h, pids[p], s, T, k, lim) for p, s, T, k, lim in qs]
    got, t0 = {}, time.time()
    while len(got) < len(qs):
        for i, (t, (p, s, T, k, lim)) in enumerate(zip(tickets, qs)):
            if i not in got:
                r = cc.cc_serve_poll(ctx.h, t, T, lim, pats[p][0])
                if r[0]:
                    got[i] = r
        assert time.time() - t0 < 120
        time.sleep(0.001)
    cc.cc_serve_stop(ctx.h)
    for i, (p, s, T, k, lim) in enumerate(qs):
        done, status, counts, exists, lat, rows = got[i]
        assert status == 0
        cid = cc.cc_color(ctx.h, s, T, k)
        run = cc.cc_run_dp(ctx.h, pids[p], cid, cc.cc_default_opts(retain=1))
        assert np.array_equal(counts, cc.cc_count(ctx.h, run, T))
        if lim:
            want, _ = cc.cc_enumerate(ctx.h, run, lim, pats[p][0])
            assert np.array_equal(rows, want) and len(rows) > 0
            ref = oracle.run_dp(graph, pats[p], oracle.colors(N, T, k, s), k)
            assert np.array_equal(rows, ref.enumerate(lim)[0])
        else:
            assert len(rows) == 0
        cc.cc_release(ctx.h, run)
        cc.cc_release_colors(ctx.h, cid)


def test_big_query_runs_split_alone_and_in_the_mix(ctx, graph):
    """A query whose tables exceed the serving budget is not refused: it runs split (one trial
    in slices by the image of one pattern vertex), alone and among smaller queries, and its
    counts equal those of the same query run in the whole arena."""
    g = synth.barabasi_albert(3000, 4, 13)
    cc.cc_load_graph(ctx.h, *g)
    big = cc.cc_load_pattern(ctx.h, *synth.cycle_pattern(6))
    small = cc.cc_load_pattern(ctx.h, *synth.path_pattern(4))
    want = _plain(ctx, big, 77, 1, 6)
    want_s = [_plain(ctx, small, 900 + i, 1, 4) for i in range(6)]
    cc.cc_serve_start(ctx.h, 256 << 20, 4)
    alone = _wait(ctx, [cc.cc_serve_submit(ctx.h, big, 77, 1, 6)], [1])
    mix_t = [cc.cc_serve_submit(ctx.h, small, 900 + i, 1, 4) for i in range(3)]
    mix_t.append(cc.cc_serve_submit(ctx.h, big, 77, 1, 6))
    mix_t += [cc.cc_serve_submit(ctx.h, small, 903 + i, 1, 4) for i in range(3)]
    mix = _wait(ctx, mix_t, [1] * 7)
    stats = cc.cc_serve_stats(ctx.h)
    cc.cc_serve_stop(ctx.h)
    assert stats["sliced"] >= 1
    for status, counts, exists, _ in alone + [mix[3]]:
        assert status == 0
        assert np.array_equal(counts, want[0]) and np.array_equal(exists, want[1])
    for (status, counts, exists, _), w in zip(mix[:3] + mix[4:], want_s):
        assert status == 0 and np.array_equal(counts, w[0])


def test_cancel_drops_unstarted_queries(ctx, graph):
    """cc_serve_cancel right after a burst: every query ends, either with its result (equal to
    the same query run alone) or with CC_ECANCELED; queries submitted after the cancel run."""
    cc.cc_load_graph(ctx.h, *graph)
    pids = [cc.cc_load_pattern(ctx.h, *p) for p in PATTERNS]
    qs = _queries(64, 5)
    cc.cc_serve_start(ctx.h, 0, 2)
    tickets = [cc.cc_serve_submit(ctx.h, pids[p], s, T, k) for p, s, T, k in qs]
    dropped = cc.cc_serve_cancel(ctx.h)
    after = [cc.cc_serve_submit(ctx.h, pids[p], s + 1, T, k) for p, s, T, k in qs[:4]]
    res = _wait(ctx, tickets + after, [q[2] for q in qs] + [q[2] for q in qs[:4]])
    cc.cc_serve_stop(ctx.h)
    statuses = [r[0] for r in res[:64]]
    assert set(statuses) <= {0, cc.CC_ECANCELED}
    assert statuses.count(cc.CC_ECANCELED) >= dropped >= 1
    for (p, s, T, k), (status, counts, exists, _) in zip(qs, res[:64]):
        if status == 0:
            want_c, want_e = _plain(ctx, pids[p], s, T, k)
            assert np.array_equal(counts, want_c) and np.array_equal(exists, want_e)
    for (p, s, T, k), (status, counts, exists, _) in zip(qs[:4], res[64:]):
        assert status == 0
        want_c, want_e = _plain(ctx, pids[p], s + 1, T, k)
        assert np.array_equal(counts, want_c) and np.array_equal(exists, want_e)
    with pytest.raises(cc.CCError):
        cc.cc_serve_cancel(ctx.h)  # not serving
