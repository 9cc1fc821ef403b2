"""Pins of the CPU oracle against facts that do not come from the oracle itself.

* Philox4x32-10 against the published known-answer vectors (tests/golden).
* Nice tree decompositions against the definitions of Section 1.2 (checked independently).
* Every node table D_x against its definition (Section 2.1), by brute force on tiny graphs.
* Root counts against brute force, closed forms, the sum over all colourings, and invariants
  (decomposition choice, relabelling, automorphisms, degree filter, second oracle).
* Reconstruction (Section 4) against the count and a direct check of every embedding.
"""
from __future__ import annotations

import math
import os
from itertools import product

import numpy as np
import pytest

import oracle
import synth
from tests import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------------------------------
# Philox
# ------------------------------------------------------------------------------------------

def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(x, 16) for x in line.split()])
    return rows


def test_philox_known_answers():
    rows = _kat()
    assert len(rows) == 3
    for r in rows:
        out = oracle.philox4x32_10(r[0:4], r[4:6])
        assert [int(x) for x in out] == r[6:10]


@pytest.mark.parametrize("k", [2, 5, 8, 9, 12, 32])
def test_colouring_uniform_chi2(k):
    n, T = 20000, 2
    z = oracle.colors(n, T, k, seed=12345)
    assert z.max() < k
    for t in range(T):
        obs = np.bincount(z[t], minlength=k).astype(np.float64)
        exp = n / k
        chi2 = ((obs - exp) ** 2 / exp).sum()
        # 99.9% quantile of chi^2 with k-1 dof is below 3*(k-1) + 25 for these k
        assert chi2 < 3 * (k - 1) + 25, (k, chi2)
    # trials are different streams, and the seed matters
    assert (z[0] != z[1]).mean() > 0.3
    z2 = oracle.colors(n, 1, k, seed=54321)
    assert (z2[0] != z[0]).mean() > 0.3


def test_colouring_is_counter_based():
    """colour(v, t) depends only on (seed, v, t): a shorter run is a prefix."""
    a = oracle.colors(1000, 3, 7, seed=99)
    b = oracle.colors(500, 2, 7, seed=99)
    assert np.array_equal(a[:2, :500], b)
    # and equals the documented mapping of the first Philox word
    for v, t in [(0, 0), (17, 2), (999, 1)]:
        x = int(oracle.philox4x32_10([v, t, 0, 0], [99, 0])[0])
        assert a[t, v] == (x * 7) >> 32


# ------------------------------------------------------------------------------------------
# nice tree decompositions, checked against the definitions of Section 1.2
# ------------------------------------------------------------------------------------------

def check_nice(nF, edges, td, nodes):
    assert nodes is not None
    N = len(nodes)
    parents = [[] for _ in range(N)]
    for i, (ty, c0, c1, u, bag) in enumerate(nodes):
        assert bag == sorted(bag) and len(set(bag)) == len(bag)
        for c in (c0, c1):
            if c >= 0:
                assert c < i  # post-order
                parents[c].append(i)
        if ty == oracle.LEAF:
            assert c0 < 0 and c1 < 0 and bag == [u]
        elif ty == oracle.INTRODUCE:
            cb = nodes[c0][4]
            assert c1 < 0 and u not in cb and sorted(cb + [u]) == bag
        elif ty == oracle.FORGET:
            cb = nodes[c0][4]
            assert c1 < 0 and u in cb and [w for w in cb if w != u] == bag
        else:
            assert ty == oracle.JOIN and c0 >= 0 and c1 >= 0
            assert nodes[c0][4] == bag == nodes[c1][4]
    # root: last, empty bag, degree 1; every other node has one parent
    assert nodes[-1][4] == [] and nodes[-1][0] == oracle.FORGET
    assert all(len(parents[i]) == 1 for i in range(N - 1)) and parents[-1] == []
    # it is a tree decomposition of F
    for u in range(nF):
        hold = [i for i in range(N) if u in nodes[i][4]]
        assert hold
        tops = [i for i in hold if not (parents[i] and u in nodes[parents[i][0]][4])]
        assert len(tops) == 1
    for a, b in np.asarray(edges).reshape(-1, 2):
        assert any(a in nd[4] and b in nd[4] for nd in nodes)
    # built from the given decomposition: every bag lies inside one of its bags (so the width
    # is at most the given width; forgetting a vertex early can make it smaller)
    assert all(any(set(nd[4]) <= set(b) for b in td[0]) for nd in nodes)
    assert max(len(nd[4]) for nd in nodes) <= max(len(b) for b in td[0])


PATTERNS = [
    synth.path_pattern(1), synth.path_pattern(2), synth.path_pattern(5), synth.cycle_pattern(3),
    synth.cycle_pattern(5), synth.star_pattern(5), synth.clique_pattern(4),
    synth.grid_pattern(2, 4), synth.grid_pattern(3, 3), synth.pattern_A(), synth.pattern_B(),
    synth.pattern_C(), synth.pattern_D(), synth.random_partial_ktree(11, 3, 5),
    synth.random_partial_ktree(8, 2, 6),
]


@pytest.mark.parametrize("pi", range(len(PATTERNS)))
def test_nice_td_definitions(pi):
    nF, e, td = PATTERNS[pi]
    nodes = oracle.nice_td(nF, e, td)
    check_nice(nF, e, td, nodes)


def test_nice_td_rejects_invalid():
    nF, e, td = synth.cycle_pattern(5)
    bags, parent = td
    assert oracle.nice_td(nF, e, ([[0, 1, 2], [0, 2, 3]], [1, -1])) is None  # vertex 4 missing
    assert oracle.nice_td(nF, e, ([[0, 1, 2], [2, 3, 4], [0, 4]], [1, 2, -1])) is None  # edge
    # vertex 0 in two disconnected parts of the tree
    assert oracle.nice_td(4, [(0, 1), (1, 2), (2, 3)], ([[0, 1], [1, 2], [2, 3, 0]], [1, 2, -1])) \
        is None
    assert oracle.nice_td(nF, e, (bags, [-1] * len(bags))) is None  # two roots


# ------------------------------------------------------------------------------------------
# node tables against the definition of D (Section 2.1), by brute force
# ------------------------------------------------------------------------------------------

TINY = [
    (synth.path_pattern(3), "er", 7, 0.5),
    (synth.cycle_pattern(4), "er", 7, 0.6),
    (synth.star_pattern(4), "er", 7, 0.5),
    (synth.grid_pattern(2, 2), "complete", 5, None),
    ((4, np.array([(0, 1), (2, 3)], np.int32),
      ([[0, 1], [1, 2], [2, 3]], [1, 2, -1])), "er", 6, 0.5),  # disconnected: bare introduce
    ((4, np.array([(0, 1), (1, 2), (2, 0), (0, 3)], np.int32),
      ([[0, 1, 2], [0, 3]], [-1, 0])), "er", 7, 0.6),  # triangle + pendant, a join in the TD
    ((5, np.array([(0, 1), (0, 2), (0, 3), (3, 4)], np.int32),
      ([[0, 1], [0, 2], [0, 3], [3, 4]], [-1, 0, 0, 2])), "er", 7, 0.6),  # tree with joins
]


def _graph(kind, n, p, seed):
    if kind == "complete":
        return synth.complete_graph(n)
    return synth.erdos_renyi(n, p, seed)


@pytest.mark.parametrize("ci", range(len(TINY)))
@pytest.mark.parametrize("dfilter", [False, True])
def test_node_tables_match_definition(ci, dfilter):
    (nF, e, td), kind, n, p = TINY[ci]
    g = _graph(kind, n, p, 3 + ci)
    G = brute.adj_sets(*g)
    degG = np.diff(g[0])
    degF = np.zeros(nF, int)
    for a, b in np.asarray(e).reshape(-1, 2):
        degF[a] += 1
        degF[b] += 1
    nodes = oracle.nice_td(nF, e, td)
    vs = brute.vstar(nodes)
    for k in (nF, nF + 1):
        zeta = np.random.default_rng(ci * 7 + k).integers(0, k, size=(2, n)).astype(np.uint8)
        run = oracle.run_dp(g, (nF, e, td), zeta, k, degree_filter=dfilter)
        for t in range(2):
            for x, nd in enumerate(nodes):
                bag = nd[4]
                want = brute.node_table(G, nF, e, zeta[t], bag, vs[x],
                                        degG if dfilter else None, degF if dfilter else None)
                phi, mask, cnt = run.table(t, x, len(bag))
                got = {(tuple(int(v) for v in phi[i]), int(mask[i])): int(cnt[i])
                       for i in range(len(mask))}
                assert got == dict(want), (x, nd)


@pytest.mark.parametrize("ci", range(len(TINY)))
def test_node_tables_with_allowed_mappings(ci):
    """Per-host-vertex masks of the pattern vertices that may map there (Section 3.2, masking
    unprofitable mappings): every node table equals the definition restricted to allowed maps;
    a full mask changes nothing."""
    (nF, e, td), kind, n, p = TINY[ci]
    g = _graph(kind, n, p, 3 + ci)
    G = brute.adj_sets(*g)
    nodes = oracle.nice_td(nF, e, td)
    vs = brute.vstar(nodes)
    rng = np.random.default_rng(50 + ci)
    zeta = rng.integers(0, nF, size=(2, n)).astype(np.uint8)
    allow = np.zeros(n, np.uint32)
    for v in range(n):
        for y in range(nF):
            if rng.random() < 0.7:
                allow[v] |= np.uint32(1 << y)
    run = oracle.run_dp(g, (nF, e, td), zeta, nF, degree_filter=False, allow=allow)
    full = oracle.run_dp(g, (nF, e, td), zeta, nF, degree_filter=False,
                         allow=np.full(n, (1 << nF) - 1, np.uint32))
    plain = oracle.run_dp(g, (nF, e, td), zeta, nF, degree_filter=False)
    assert np.array_equal(full.node_sizes, plain.node_sizes)
    assert np.array_equal(full.count, plain.count)
    for t in range(2):
        for x, nd in enumerate(nodes):
            bag = nd[4]
            want = brute.node_table(G, nF, e, zeta[t], bag, vs[x], allow=allow)
            phi, mask, cnt = run.table(t, x, len(bag))
            got = {(tuple(int(v) for v in phi[i]), int(mask[i])): int(cnt[i])
                   for i in range(len(mask))}
            assert got == dict(want), (x, nd)


@pytest.mark.parametrize("ci", range(len(TINY)))
def test_degree_filter_is_an_allowed_mask(ci):
    """The degree filter is the mask {y : deg_G(x) >= deg_F(y)} (the paragraph derives it from
    the extended input): both give the same tables."""
    (nF, e, td), kind, n, p = TINY[ci]
    g = _graph(kind, n, p, 3 + ci)
    degG = np.diff(g[0])
    degF = np.zeros(nF, int)
    for a, b in np.asarray(e).reshape(-1, 2):
        degF[a] += 1
        degF[b] += 1
    allow = np.array([sum(1 << y for y in range(nF) if degG[v] >= degF[y]) for v in range(n)],
                     np.uint32)
    zeta = np.random.default_rng(ci).integers(0, nF, size=(2, n)).astype(np.uint8)
    a = oracle.run_dp(g, (nF, e, td), zeta, nF, degree_filter=True)
    b = oracle.run_dp(g, (nF, e, td), zeta, nF, degree_filter=False, allow=allow)
    assert np.array_equal(a.node_sizes, b.node_sizes) and np.array_equal(a.count, b.count)
    for t in range(2):
        for x, nd in enumerate(oracle.nice_td(nF, e, td)):
            ta, tb = a.table(t, x, len(nd[4])), b.table(t, x, len(nd[4]))
            assert all(np.array_equal(u, w) for u, w in zip(ta, tb))


# ------------------------------------------------------------------------------------------
# root counts: brute force, closed forms, sum over colourings
# ------------------------------------------------------------------------------------------

SMALL_PATTERNS = [synth.path_pattern(4), synth.cycle_pattern(4), synth.cycle_pattern(5),
                  synth.star_pattern(4), synth.grid_pattern(2, 2), synth.clique_pattern(3),
                  (5, np.array([(0, 1), (2, 3), (3, 4)], np.int32),
                   ([[0, 1], [1, 2], [2, 3], [3, 4]], [1, 2, 3, -1]))]


@pytest.mark.parametrize("pi", range(len(SMALL_PATTERNS)))
def test_root_count_brute_force(pi):
    nF, e, td = SMALL_PATTERNS[pi]
    for gi in range(3):
        g = synth.erdos_renyi(8, 0.55, 100 + gi)
        G = brute.adj_sets(*g)
        for k in (nF, nF + 2):
            zeta = np.random.default_rng(gi * 31 + k).integers(0, k, size=(3, 8)).astype(np.uint8)
            run = oracle.run_dp(g, (nF, e, td), zeta, k)
            for t in range(3):
                want = brute.count_embeddings(G, nF, e, zeta[t])
                assert int(run.count[t]) == want
                assert int(run.exists[t]) == int(want > 0)


def _esym(vals, r):
    """Elementary symmetric polynomial e_r(vals)."""
    e = [1] + [0] * r
    for v in vals:
        for j in range(r, 0, -1):
            e[j] += e[j - 1] * v
    return e[r]


@pytest.mark.parametrize("pat", [synth.cycle_pattern(4), synth.path_pattern(4),
                                 synth.star_pattern(4), synth.grid_pattern(2, 2),
                                 synth.clique_pattern(4), synth.pattern_B()])
def test_closed_form_complete_host(pat):
    """G = K_n: every injective map is an embedding, so count = n_F! * e_{n_F}(c_1..c_k) with
    c_i the size of colour class i (n_F! * prod c_i when k = n_F)."""
    nF, e, td = pat
    n = 9
    g = synth.complete_graph(n)
    for k in (nF, nF + 1):
        zeta = np.random.default_rng(k).integers(0, k, size=(4, n)).astype(np.uint8)
        run = oracle.run_dp(g, pat, zeta, k)
        for t in range(4):
            c = np.bincount(zeta[t], minlength=k)
            assert int(run.count[t]) == math.factorial(nF) * _esym(list(c), nF)


def test_closed_form_cycle_host_paths_and_cycles():
    """G = C_n: P_j has 2 * #(windows of j consecutive cycle vertices with distinct colours)
    embeddings; C_j has 2n if j = n and the colouring is a bijection, else 0."""
    n = 12
    g = synth.cycle_graph(n)
    rng = np.random.default_rng(5)
    for j in range(2, 8):
        pat = synth.path_pattern(j)
        zeta = rng.integers(0, j, size=(6, n)).astype(np.uint8)
        zeta[0, :j] = np.arange(j)  # make sure some window is colourful
        run = oracle.run_dp(g, pat, zeta, j)
        for t in range(6):
            w = sum(len({int(zeta[t][(i + s) % n]) for s in range(j)}) == j for i in range(n))
            assert int(run.count[t]) == 2 * w
    for j in (3, 5, 8):
        for nn in (j, j + 3):
            gc = synth.cycle_graph(nn)
            z = np.stack([rng.permutation(nn) % j, np.arange(nn) % j]).astype(np.uint8)
            if nn == j:
                z[1] = rng.permutation(j)
            run = oracle.run_dp(gc, synth.cycle_pattern(j), z, j)
            for t in range(2):
                bij = len(set(z[t].tolist())) == nn
                assert int(run.count[t]) == (2 * nn if (nn == j and bij) else 0)


def test_closed_form_star():
    """F = S_j (centre + j-1 leaves): count = sum_v (j-1)! e_{j-1}(neighbour colour classes of v
    other than the colour of v)."""
    g = synth.erdos_renyi(60, 0.15, 9)
    rp, col = g
    for j in (3, 4, 5):
        for k in (j, j + 1):
            zeta = np.random.default_rng(j * 10 + k).integers(0, k, size=(2, 60)).astype(np.uint8)
            run = oracle.run_dp(g, synth.star_pattern(j), zeta, k)
            for t in range(2):
                tot = 0
                for v in range(60):
                    nb = col[rp[v]:rp[v + 1]]
                    cls = np.bincount(zeta[t][nb], minlength=k)
                    cls[zeta[t][v]] = 0
                    tot += math.factorial(j - 1) * _esym(list(cls), j - 1)
                assert int(run.count[t]) == tot


def test_closed_form_single_edge():
    """F = K_2: twice the number of edges whose endpoints differ in colour."""
    g = synth.barabasi_albert(300, 3, 4)
    e = synth.edges_from_csr(*g)
    zeta = oracle.colors(300, 3, 2, seed=4)
    run = oracle.run_dp(g, synth.path_pattern(2), zeta, 2)
    for t in range(3):
        assert int(run.count[t]) == 2 * int((zeta[t][e[:, 0]] != zeta[t][e[:, 1]]).sum())


@pytest.mark.parametrize("pat", [synth.path_pattern(3), synth.cycle_pattern(3),
                                 synth.star_pattern(4), synth.cycle_pattern(4)])
def test_sum_over_all_colourings(pat):
    """Summed over all k^n colourings, count = inj(F, G) * (k)_{n_F} * k^(n - n_F)."""
    nF, e, td = pat
    n = 6
    g = synth.erdos_renyi(n, 0.7, 21)
    G = brute.adj_sets(*g)
    inj = len(brute.embeddings(G, nF, e, None))
    for k in (nF, nF + 1):
        allz = np.array(list(product(range(k), repeat=n)), dtype=np.uint8)
        run = oracle.run_dp(g, pat, allz, k)
        falling = math.prod(range(k - nF + 1, k + 1))
        assert int(run.count.astype(object).sum()) == inj * falling * k ** (n - nF)


# ------------------------------------------------------------------------------------------
# invariants and the second oracle
# ------------------------------------------------------------------------------------------

def test_invariant_under_decomposition_and_relabelling():
    g = synth.erdos_renyi(120, 0.08, 2)
    rng = np.random.default_rng(0)
    for pat in (synth.cycle_pattern(5), synth.grid_pattern(2, 3), synth.pattern_B(),
                synth.pattern_D()):
        nF, e, td = pat
        zeta = oracle.colors(120, 3, nF, seed=11)
        base = oracle.run_dp(g, pat, zeta, nF).count
        # the one-bag decomposition
        assert np.array_equal(oracle.run_dp(g, (nF, e, synth.trivial_td(nF)), zeta, nF).count,
                              base)
        # relabelled pattern with its relabelled decomposition
        perm = rng.permutation(nF)
        assert np.array_equal(oracle.run_dp(g, synth.relabel_pattern(nF, e, td, perm), zeta,
                                            nF).count, base)
        # relabelled host graph with colours moved along
        gp = rng.permutation(120)
        g2 = synth.relabel_csr(*g, gp)
        z2 = np.zeros_like(zeta)
        z2[:, gp] = zeta
        assert np.array_equal(oracle.run_dp(g2, pat, z2, nF).count, base)
        # the degree filter never changes the root
        assert np.array_equal(oracle.run_dp(g, pat, zeta, nF, degree_filter=False).count, base)


@pytest.mark.parametrize("pat,aut", [(synth.cycle_pattern(5), 10), (synth.path_pattern(4), 2),
                                     (synth.grid_pattern(2, 4), 4), (synth.grid_pattern(3, 3), 8),
                                     (synth.star_pattern(4), 6), (synth.clique_pattern(4), 24)])
def test_count_divisible_by_automorphisms(pat, aut):
    g = synth.barabasi_albert(400, 4, 1)
    nF = pat[0]
    zeta = oracle.colors(400, 2, nF, seed=3)
    run = oracle.run_dp(g, pat, zeta, nF)
    assert all(int(c) % aut == 0 for c in run.count)


@pytest.mark.parametrize("pat", [synth.cycle_pattern(5), synth.pattern_A(), synth.pattern_B(),
                                 synth.pattern_C(), synth.pattern_D(), synth.grid_pattern(2, 3)])
def test_dp_matches_backtracking(pat):
    nF, e, td = pat
    g = synth.barabasi_albert(250, 3, 8)
    zeta = oracle.colors(250, 2, nF, seed=17)
    run = oracle.run_dp(g, pat, zeta, nF)
    for t in range(2):
        c, _ = oracle.backtrack(g, pat, zeta[t])
        assert int(run.count[t]) == c


def test_workload_er200_c5_matches_backtracking():
    g = synth.erdos_renyi(200, 0.05, 1)
    pat = synth.cycle_pattern(5)
    zeta = oracle.colors(200, 1, 5, seed=7)
    run = oracle.run_dp(g, pat, zeta, 5)
    c, lst = oracle.backtrack(g, pat, zeta[0], limit=10 ** 6)
    assert int(run.count[0]) == c and c > 0
    L, tot, per = run.enumerate(10 ** 6)
    assert tot == per == c
    assert np.array_equal(L, lst)


def _check_embedding(G, e, zeta_rows, Phi):
    assert len(set(Phi.tolist())) == len(Phi)
    for a, b in np.asarray(e).reshape(-1, 2):
        assert int(Phi[b]) in G[int(Phi[a])]
    assert any(len({int(z[v]) for v in Phi}) == len(Phi) for z in zeta_rows)


@pytest.mark.parametrize("pat", [synth.cycle_pattern(4), synth.pattern_A(), synth.pattern_B(),
                                 synth.pattern_D(), synth.star_pattern(5)])
def test_reconstruction(pat):
    """Section 4: per trial the reconstructed list has exactly count entries; the union over
    trials is sorted, repeat-free, and every row is a colourful embedding."""
    nF, e, td = pat
    g = synth.erdos_renyi(40, 0.2, 6)
    G = brute.adj_sets(*g)
    zeta = oracle.colors(40, 3, nF, seed=2)
    run = oracle.run_dp(g, pat, zeta, nF)
    L, tot, per = run.enumerate(10 ** 6)
    assert per == int(run.count.astype(object).sum())
    assert tot == len(L) <= per
    assert all(tuple(L[i]) < tuple(L[i + 1]) for i in range(len(L) - 1))
    for Phi in L:
        _check_embedding(G, e, zeta, Phi)
    # union over trials equals the union of the per-trial backtracking lists
    want = set()
    for t in range(3):
        _, lst = oracle.backtrack(g, pat, zeta[t], limit=10 ** 6)
        want |= {tuple(r) for r in lst}
    assert {tuple(r) for r in L} == want
    # truncation keeps the lexicographically smallest
    L5, tot5, _ = run.enumerate(5)
    assert tot5 == tot and np.array_equal(L5, L[:5])


# ------------------------------------------------------------------------------------------
# the distance bound of Section 3.2 (mapping expansion)
# ------------------------------------------------------------------------------------------

def _gdist(g, a, r):
    """Host vertices within distance r of a (plain breadth-first search)."""
    G = brute.adj_sets(*g)
    seen, frontier = {a}, {a}
    for _ in range(r):
        frontier = {y for x in frontier for y in G[x]} - seen
        seen |= frontier
    return seen


def test_distance_bound_table_by_definition():
    """Path 0-1-2 with bags {0,2} under {0,1,2}: vertex 2 is introduced next to 0 at F-distance
    2 with no bag neighbour, so the pruned table is the definition's table restricted to
    phi(2) within distance 2 of phi(0); the root is unchanged."""
    e = np.array([(0, 1), (1, 2)], np.int32)
    td = ([[0, 2], [0, 1, 2]], [1, -1])
    nodes = oracle.nice_td(3, e, td)
    x = next(i for i, nd in enumerate(nodes) if nd[0] == 1 and nd[3] == 2 and len(nd[4]) == 2)
    vs = brute.vstar(nodes)
    for seed in range(3):
        g = synth.erdos_renyi(12, 0.25, 40 + seed)
        G = brute.adj_sets(*g)
        zeta = np.random.default_rng(seed).integers(0, 3, size=(2, 12)).astype(np.uint8)
        plain = oracle.run_dp(g, (3, e, td), zeta, 3, degree_filter=False)
        pruned = oracle.run_dp(g, (3, e, td), zeta, 3, degree_filter=False, distance_prune=True)
        assert np.array_equal(plain.count, pruned.count)
        assert pruned.node_sizes[:, x].sum() < plain.node_sizes[:, x].sum()
        for t in range(2):
            want = brute.node_table(G, 3, e, zeta[t], nodes[x][4], vs[x])
            want = {k: v for k, v in want.items() if k[0][1] in _gdist(g, k[0][0], 2)}
            phi, mask, cnt = pruned.table(t, x, 2)
            got = {(tuple(int(v) for v in phi[i]), int(mask[i])): int(cnt[i])
                   for i in range(len(mask))}
            assert got == want


def test_distance_bound_at_distance_three_by_definition():
    """Path 0-1-2-3 with bags {0,3} under {0,1,3} under {1,2,3}: vertex 3 is introduced next to
    0 at F-distance 3 with no bag neighbour, so the pruned table is the definition's table
    restricted to phi(3) within distance 3 of phi(0) (a breadth-first ball, not the radius-2
    one); the root is unchanged."""
    e = np.array([(0, 1), (1, 2), (2, 3)], np.int32)
    td = ([[0, 3], [0, 1, 3], [1, 2, 3]], [1, 2, -1])
    nodes = oracle.nice_td(4, e, td)
    x = next(i for i, nd in enumerate(nodes) if nd[0] == 1 and nd[3] == 3 and len(nd[4]) == 2)
    vs = brute.vstar(nodes)
    shrunk = beyond2 = False
    for seed in range(4):
        g = synth.erdos_renyi(16, 0.13, 60 + seed)
        G = brute.adj_sets(*g)
        zeta = np.random.default_rng(seed).integers(0, 4, size=(2, 16)).astype(np.uint8)
        plain = oracle.run_dp(g, (4, e, td), zeta, 4, degree_filter=False)
        pruned = oracle.run_dp(g, (4, e, td), zeta, 4, degree_filter=False, distance_prune=True)
        assert np.array_equal(plain.count, pruned.count)
        shrunk = shrunk or pruned.node_sizes[:, x].sum() < plain.node_sizes[:, x].sum()
        for t in range(2):
            full = brute.node_table(G, 4, e, zeta[t], nodes[x][4], vs[x])
            want = {k: v for k, v in full.items() if k[0][1] in _gdist(g, k[0][0], 3)}
            near2 = {k for k in full if k[0][1] in _gdist(g, k[0][0], 2)}
            phi, mask, cnt = pruned.table(t, x, 2)
            got = {(tuple(int(v) for v in phi[i]), int(mask[i])): int(cnt[i])
                   for i in range(len(mask))}
            assert got == want
            beyond2 = beyond2 or len(set(want) - near2) > 0  # radius 3, not 2
    assert shrunk and beyond2


@pytest.mark.parametrize("pat", [synth.random_partial_ktree(7, 3, 2),
                                 synth.random_partial_ktree(8, 2, 9),
                                 synth.random_partial_ktree(8, 3, 4), synth.pattern_D(),
                                 (4, np.array([(0, 1), (1, 2), (2, 3)], np.int32),
                                  ([[0, 3], [0, 1, 3], [1, 2, 3]], [1, 2, -1]))])
def test_distance_bound_keeps_root_and_shrinks_tables(pat):
    """On patterns whose decompositions introduce vertices away from their bag: root counts
    and enumerations are those without the bound, and every table is a subset (counts no
    larger) of the unbounded one."""
    nF = pat[0]
    g = synth.erdos_renyi(30, 0.2, 8)
    zeta = oracle.colors(30, 3, nF, seed=4)
    a = oracle.run_dp(g, pat, zeta, nF)
    b = oracle.run_dp(g, pat, zeta, nF, distance_prune=True)
    assert np.array_equal(a.count, b.count) and np.array_equal(a.exists, b.exists)
    assert np.array_equal(a.enumerate(10 ** 6)[0], b.enumerate(10 ** 6)[0])
    assert (b.node_sizes <= a.node_sizes).all()
    nodes = oracle.nice_td(*pat)
    for t in range(3):
        for x, nd in enumerate(nodes):
            pa, ma, ca = a.table(t, x, len(nd[4]))
            pb, mb, cb = b.table(t, x, len(nd[4]))
            A = {(tuple(int(v) for v in pa[i]), int(ma[i])): int(ca[i]) for i in range(len(ma))}
            for i in range(len(mb)):
                k = (tuple(int(v) for v in pb[i]), int(mb[i]))
                assert k in A and int(cb[i]) <= A[k]


def test_masks_and_distance_bound_together():
    """Allowed mappings and the distance bound compose: on a path whose decomposition
    introduces 2 next to 0 (F-distance 2), the bounded run's tables are smaller, its root and
    enumeration are those of the masks alone, and its counts are the brute-force counts of
    allowed colourful embeddings."""
    e = np.array([(0, 1), (1, 2), (2, 3)], np.int32)
    pat = (4, e, ([[0, 2], [0, 1, 2], [2, 3]], [1, -1, 1]))
    g = synth.erdos_renyi(9, 0.6, 1)
    G = brute.adj_sets(*g)
    rng = np.random.default_rng(1)
    allow = np.array([sum(1 << y for y in range(4) if rng.random() < 0.85) for _ in range(9)],
                     np.uint32)
    zeta = rng.integers(0, 4, size=(2, 9)).astype(np.uint8)
    a = oracle.run_dp(g, pat, zeta, 4, allow=allow, degree_filter=False)
    b = oracle.run_dp(g, pat, zeta, 4, allow=allow, degree_filter=False, distance_prune=True)
    assert b.node_sizes.sum() < a.node_sizes.sum()
    assert np.array_equal(a.count, b.count) and int(b.count.min()) > 0
    assert np.array_equal(a.enumerate(10 ** 6)[0], b.enumerate(10 ** 6)[0])
    for t in range(2):
        want = sum(1 for m in brute.embeddings(G, 4, e, zeta[t])
                   if all((int(allow[m[y]]) >> y) & 1 for y in m))
        assert int(b.count[t]) == want
