"""Seeded synthetic inputs: host graphs G, pattern graphs F and tree decompositions of F.

This module only builds inputs.  It holds none of the colour-coding arithmetic (no colouring,
no dynamic programme, no nice-decomposition construction): both the CPU oracle and the GPU
library consume what it returns, and neither is imported here.

Graphs are simple and undirected (paper Section 1.2) and returned as CSR arrays
``(row_ptr int32[n+1], col int32[2m])`` with every row sorted and duplicate-free, no self loops.
Patterns are ``(n_F, edges int32[m_F, 2])``.  A tree decomposition is returned as
``(bags: list[list[int]], parent: list[int])`` with parent -1 at the root; it satisfies the three
conditions of the paper's tree-decomposition definition (Section 1.2).
"""
from __future__ import annotations

import numpy as np

# ----------------------------------------------------------------------------------------------
# host graphs
# ----------------------------------------------------------------------------------------------


def csr_from_edges(n: int, edges: np.ndarray):
    """Symmetric CSR from an undirected edge list; drops self loops and duplicate edges."""
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    e = e[e[:, 0] != e[:, 1]]
    a = np.minimum(e[:, 0], e[:, 1])
    b = np.maximum(e[:, 0], e[:, 1])
    key = np.unique(a * n + b)
    a = key // n
    b = key % n
    src = np.concatenate([a, b])
    dst = np.concatenate([b, a])
    order = np.lexsort((dst, src))
    src = src[order]
    dst = dst[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, src + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return row_ptr.astype(np.int32), dst.astype(np.int32)


def plant(graph, pattern_edges, vertices):
    """The graph with a copy of a pattern added: pattern vertex i becomes graph vertex
    vertices[i] and every pattern edge becomes an edge (existing ones are kept once)."""
    row_ptr, col = graph
    n = len(row_ptr) - 1
    v = np.asarray(vertices, dtype=np.int64)
    pe = np.asarray(pattern_edges, dtype=np.int64).reshape(-1, 2)
    extra = np.stack([v[pe[:, 0]], v[pe[:, 1]]], axis=1)
    return csr_from_edges(n, np.concatenate([edges_from_csr(row_ptr, col), extra]))


def edges_from_csr(row_ptr, col):
    """Each undirected edge once, as (u, v) with u < v, in CSR order."""
    n = len(row_ptr) - 1
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(row_ptr))
    m = src < col
    return np.stack([src[m], np.asarray(col, dtype=np.int64)[m]], axis=1)


def erdos_renyi(n: int, p: float, seed: int):
    """G(n, p).  Small n: one uniform draw per pair i<j in lexicographic order.  Large n:
    geometric skipping over the same pair order (Batagelj and Brandes)."""
    rng = np.random.default_rng(seed)
    npairs = n * (n - 1) // 2
    if npairs <= 5_000_000:
        iu, ju = np.triu_indices(n, k=1)
        keep = rng.random(npairs) < p
        return csr_from_edges(n, np.stack([iu[keep], ju[keep]], axis=1))
    # geometric skipping: gaps between successive kept pair indices are Geometric(p)
    idx = []
    pos = -1
    chunk = max(1024, int(npairs * p * 1.1 / 8) + 1024)
    while True:
        gaps = rng.geometric(p, size=chunk).astype(np.int64)
        c = pos + np.cumsum(gaps)
        c = c[c < npairs]
        idx.append(c)
        if len(c) < chunk:
            break
        pos = int(c[-1])
    k = np.concatenate(idx)
    # pair index -> (i, j), i < j, lexicographic: row i holds n-1-i pairs
    nn = float(n)
    i = np.floor(((2 * nn - 1) - np.sqrt((2 * nn - 1) ** 2 - 8.0 * k)) / 2).astype(np.int64)
    start = i * (2 * n - i - 1) // 2
    # fix up rounding at row boundaries
    over = start > k
    while over.any():
        i[over] -= 1
        start = i * (2 * n - i - 1) // 2
        over = start > k
    nxt = (i + 1) * (2 * n - i - 2) // 2
    under = nxt <= k
    while under.any():
        i[under] += 1
        start = i * (2 * n - i - 1) // 2
        nxt = (i + 1) * (2 * n - i - 2) // 2
        under = nxt <= k
    j = k - start + i + 1
    return csr_from_edges(n, np.stack([i, j], axis=1))


def barabasi_albert(n: int, m: int, seed: int):
    """Preferential attachment: start from K_{m+1}; every new vertex attaches to m distinct
    earlier vertices drawn proportionally to degree (uniform draws from the list of edge
    endpoints; a repeated target is redrawn)."""
    rng = np.random.default_rng(seed)
    m0 = m + 1
    edges = [(i, j) for i in range(m0) for j in range(i + 1, m0)]
    ends = np.empty(2 * (len(edges) + (n - m0) * m), dtype=np.int64)
    ne = 0
    for a, b in edges:
        ends[ne] = a
        ends[ne + 1] = b
        ne += 2
    out = np.empty(((n - m0) * m, 2), dtype=np.int64)
    oe = 0
    for v in range(m0, n):
        chosen = []
        while len(chosen) < m:
            t = int(ends[int(rng.integers(0, ne))])
            if t not in chosen:
                chosen.append(t)
        for t in chosen:
            out[oe, 0] = v
            out[oe, 1] = t
            oe += 1
            ends[ne] = v
            ends[ne + 1] = t
            ne += 2
    all_e = np.concatenate([np.array(edges, dtype=np.int64).reshape(-1, 2), out[:oe]])
    return csr_from_edges(n, all_e)


def power_law_config(n: int, mean_deg: float, exponent: float, seed: int):
    """Erased configuration model: i.i.d. degrees from a discrete power law P(d) ~ d^-exponent on
    [d_min, d_max = n^(1/(exponent-1))]; d_min is a seeded mix of the two integers around the
    value that gives the requested mean; stubs are matched uniformly; self loops and multi-edges
    are erased."""
    rng = np.random.default_rng(seed)
    d_max = int(n ** (1.0 / (exponent - 1.0)))

    def mean_for(dmin):
        d = np.arange(dmin, d_max + 1, dtype=np.float64)
        w = d ** (-exponent)
        return float((d * w).sum() / w.sum())

    # integer d_min bracketing the target mean, mixed to hit it
    lo = 1
    while lo + 1 <= d_max and mean_for(lo + 1) <= mean_deg:
        lo += 1
    m_lo, m_hi = mean_for(lo), mean_for(lo + 1)
    frac = 0.0 if m_hi == m_lo else min(1.0, max(0.0, (mean_deg - m_lo) / (m_hi - m_lo)))

    def draw(dmin, size):
        d = np.arange(dmin, d_max + 1, dtype=np.float64)
        w = d ** (-exponent)
        w /= w.sum()
        return rng.choice(np.arange(dmin, d_max + 1), size=size, p=w)

    use_hi = rng.random(n) < frac
    deg = np.empty(n, dtype=np.int64)
    deg[~use_hi] = draw(lo, int((~use_hi).sum()))
    deg[use_hi] = draw(lo + 1, int(use_hi.sum()))
    if deg.sum() % 2:
        deg[int(rng.integers(0, n))] += 1
    stubs = np.repeat(np.arange(n, dtype=np.int64), deg)
    rng.shuffle(stubs)
    return csr_from_edges(n, stubs.reshape(-1, 2))


def complete_graph(n: int):
    iu, ju = np.triu_indices(n, k=1)
    return csr_from_edges(n, np.stack([iu, ju], axis=1))


def cycle_graph(n: int):
    e = np.stack([np.arange(n), (np.arange(n) + 1) % n], axis=1)
    return csr_from_edges(n, e)


def relabel_csr(row_ptr, col, perm):
    """Graph with vertex v renamed perm[v]."""
    n = len(row_ptr) - 1
    e = edges_from_csr(row_ptr, col)
    perm = np.asarray(perm, dtype=np.int64)
    return csr_from_edges(n, perm[e])


# ----------------------------------------------------------------------------------------------
# patterns (Table 1 families and Fig. 1 patterns) with tree decompositions
# ----------------------------------------------------------------------------------------------


def _chain_parent(nb):
    """Parents for a path of bags: bag i's parent is bag i+1, last bag is the root."""
    return [i + 1 for i in range(nb - 1)] + [-1]


def path_pattern(n):
    """P_n, treewidth 1 (Table 1)."""
    e = np.array([(i, i + 1) for i in range(n - 1)], dtype=np.int32).reshape(-1, 2)
    bags = [[i, i + 1] for i in range(n - 1)] if n > 1 else [[0]]
    return n, e, (bags, _chain_parent(len(bags)))


def cycle_pattern(n):
    """C_n, treewidth 2 (Table 1); bags {0, i, i+1}."""
    e = np.array([(i, (i + 1) % n) for i in range(n)], dtype=np.int32)
    bags = [[0, i, i + 1] for i in range(1, n - 1)]
    return n, e, (bags, _chain_parent(len(bags)))


def star_pattern(n):
    """S_n: a centre 0 and n-1 leaves, treewidth 1 (Table 1)."""
    e = np.array([(0, i) for i in range(1, n)], dtype=np.int32).reshape(-1, 2)
    bags = [[0, i] for i in range(1, n)] if n > 1 else [[0]]
    return n, e, (bags, _chain_parent(len(bags)))


def clique_pattern(n):
    """K_n, treewidth n-1 (Table 1); a single bag."""
    e = np.array([(i, j) for i in range(n) for j in range(i + 1, n)], dtype=np.int32).reshape(-1, 2)
    return n, e, ([list(range(n))], [-1])


def grid_pattern(r, c):
    """G_{r,c}: vertex (i, j) is i*c + j; treewidth min(r, c) (Table 1).  The decomposition sweeps
    along the longer side, a bag holding one cross-section plus the next vertex."""
    e = []
    for i in range(r):
        for j in range(c):
            v = i * c + j
            if j + 1 < c:
                e.append((v, v + 1))
            if i + 1 < r:
                e.append((v, v + c))
    e = np.array(e, dtype=np.int32).reshape(-1, 2)
    # order vertices so that consecutive windows of width min(r,c)+1 cover every edge
    if r <= c:
        order = [i * c + j for j in range(c) for i in range(r)]  # column-major sweep
        w = r
    else:
        order = [i * c + j for i in range(r) for j in range(c)]  # row-major sweep
        w = c
    n = r * c
    if n <= w + 1:
        return n, e, ([list(range(n))], [-1])
    bags = [sorted(order[s:s + w + 1]) for s in range(n - w)]
    return n, e, (bags, _chain_parent(len(bags)))


# Fig. 1: patterns A-D as drawn in the paper's TikZ (vertex names are the node labels).
PATTERN_A_EDGES = [(0, 1), (1, 2), (2, 3), (2, 4), (5, 4), (6, 4), (6, 7), (7, 8)]
PATTERN_B_EDGES = [(0, 1), (1, 2), (0, 2), (1, 6), (1, 5), (2, 3), (3, 4)]
PATTERN_C_EDGES = [(0, 3), (0, 4), (1, 3), (1, 5), (2, 4), (2, 5), (6, 1), (6, 2), (7, 0), (7, 2),
                   (8, 0), (8, 1)]
# D: the isolated edge p1-p2 becomes 0-1, the 5-cycle 1..5 becomes 2..6
PATTERN_D_EDGES = [(0, 1), (2, 3), (3, 4), (4, 5), (5, 6), (2, 6)]


def pattern_A():
    """Fig. 1 (a): a tree on 9 vertices, 8 edges, treewidth 1."""
    e = np.array(PATTERN_A_EDGES, dtype=np.int32)
    bags = [[0, 1], [1, 2], [2, 3], [2, 4], [4, 5], [4, 6], [6, 7], [7, 8]]
    parent = [1, 3, 3, -1, 3, 3, 5, 6]
    return 9, e, (bags, parent)


def pattern_B():
    """Fig. 1 (b): 7 vertices, 7 edges, treewidth 2."""
    e = np.array(PATTERN_B_EDGES, dtype=np.int32)
    bags = [[0, 1, 2], [1, 5], [1, 6], [2, 3], [3, 4]]
    parent = [-1, 0, 0, 0, 3]
    return 7, e, (bags, parent)


def pattern_C():
    """Fig. 1 (c): 9 vertices, 12 edges, treewidth 2 (0,1,2 with paths of length 2 between
    every pair, doubled)."""
    e = np.array(PATTERN_C_EDGES, dtype=np.int32)
    bags = [[0, 1, 2], [0, 1, 3], [0, 1, 8], [0, 2, 4], [0, 2, 7], [1, 2, 5], [1, 2, 6]]
    parent = [-1, 0, 0, 0, 0, 0, 0]
    return 9, e, (bags, parent)


def pattern_D():
    """Fig. 1 (d): disconnected, an edge plus a 5-cycle; 7 vertices, 6 edges, treewidth 2."""
    e = np.array(PATTERN_D_EDGES, dtype=np.int32)
    bags = [[0, 1], [1, 2], [2, 3, 4], [2, 4, 5], [2, 5, 6]]
    parent = [1, 2, 3, 4, -1]
    return 7, e, (bags, parent)


def random_partial_ktree(n, k, seed, keep=0.5):
    """Random partial k-tree on n >= k+1 vertices: start with K_{k+1}; each new vertex is joined
    to a uniformly random k-clique of the k-tree built so far; then a random spanning tree of the
    k-tree is kept together with every other edge with probability ``keep``.  The tree
    decomposition is the construction's (k+1)-cliques."""
    rng = np.random.default_rng(seed)
    cliques = [tuple(range(k + 1))]  # bags, in creation order
    parent = [-1]
    kcl = []  # (k-clique, bag index that contains it)
    from itertools import combinations
    for c in combinations(range(k + 1), k):
        kcl.append((c, 0))
    edges = set((i, j) for i in range(k + 1) for j in range(i + 1, k + 1))
    for v in range(k + 1, n):
        c, b = kcl[int(rng.integers(0, len(kcl)))]
        bag = tuple(sorted(c + (v,)))
        cliques.append(bag)
        parent.append(b)
        bi = len(cliques) - 1
        for w in c:
            edges.add((min(v, w), max(v, w)))
        for sub in combinations(c, k - 1):
            kcl.append((tuple(sorted(sub + (v,))), bi))
    edges = sorted(edges)
    # random spanning tree (random edge order, union-find), plus each other edge w.p. keep
    perm = rng.permutation(len(edges))
    uf = list(range(n))

    def find(x):
        while uf[x] != x:
            uf[x] = uf[uf[x]]
            x = uf[x]
        return x

    kept = []
    for i in perm:
        a, b = edges[i]
        ra, rb = find(a), find(b)
        if ra != rb:
            uf[ra] = rb
            kept.append((a, b))
        elif rng.random() < keep:
            kept.append((a, b))
    e = np.array(sorted(kept), dtype=np.int32)
    # root the decomposition at bag 0 (parents point towards bag 0 already)
    return n, e, ([list(b) for b in cliques], parent)


def relabel_pattern(nF, edges, td, perm):
    """Pattern with vertex u renamed perm[u] (decomposition relabelled alike)."""
    perm = list(perm)
    e = np.array([(perm[a], perm[b]) for a, b in np.asarray(edges)], dtype=np.int32).reshape(-1, 2)
    bags, parent = td
    return nF, e, ([sorted(perm[u] for u in bag) for bag in bags], list(parent))


def trivial_td(nF):
    """The one-bag decomposition (width n_F - 1); valid for every pattern."""
    return [list(range(nF))], [-1]


# ----------------------------------------------------------------------------------------------
# the benchmark workloads (seeded)
# ----------------------------------------------------------------------------------------------

WORKLOADS = {
    # Erdos-Renyi n=200, p=0.05 (seed 1); 5-cycle; k=5; Philox seed 7; 1 trial
    "er200_c5": dict(graph=("er", 200, 0.05, 1), pattern=("cycle", 5), k=5, seed=7, trials=1),
    # Barabasi-Albert n=20000, m=4 (seed 1); 2x4 grid; k=8; 64 trials
    "ba20k_grid2x4": dict(graph=("ba", 20000, 4, 1), pattern=("grid", 2, 4), k=8, seed=7,
                          trials=64),
    # Erdos-Renyi n=100000, average degree 10 (seed 1); 3x3 grid; k=9; 32 trials
    "er100k_grid3x3": dict(graph=("er", 100000, 10.0 / 99999.0, 1), pattern=("grid", 3, 3), k=9,
                           seed=7, trials=32),
    # erased power-law configuration model n=10^6, mean degree 8, exponent 2.5 (seed 1); a batch
    # of 64 random partial 3-trees of 10-12 vertices (pattern seeds 7000..7063); k = n_F; 16
    # trials each
    "pl1m_ktree3": dict(graph=("pl", 1_000_000, 8.0, 2.5, 1), patterns=64, sizes=(10, 12),
                        width=3, pattern_seed=7000, trials=16, seed=7),
    # serving: Barabasi-Albert n=200000, m=5 (seed 1) resident; 2000 queries, Poisson arrivals
    # at 200/s (seed 1); families path, cycle, grid, random partial k-tree (k <= 3); n_F = k
    # uniform in 4..10; one trial per query
    "serve_ba200k": dict(graph=("ba", 200000, 5, 1), queries=2000, rate=200.0, seed=1,
                         sizes=(4, 10), trials=1, ktree_pool=2),
}

GRID_SHAPES = {4: (2, 2), 6: (2, 3), 8: (2, 4), 9: (3, 3), 10: (2, 5)}

# Erdos-Renyi phase-transition study (paper Section 5.4): target G(150, p) against pattern
# G(10, q), p and q from 0 in steps of 0.03; ten colourings (iterations) per point, k = 10
ER_PHASE = dict(n_target=150, n_pattern=10, step=0.03, iterations=10, seed=1)


def er_phase_probs(step=ER_PHASE["step"]):
    """Edge probabilities 0, step, 2*step, ... up to 1 (the axes of the study)."""
    m = int(np.floor(1.0 / step + 1e-9))
    return [round(i * step, 10) for i in range(m + 1)]


def er_phase_instance(ip, iq, spec=ER_PHASE):
    """Point (ip, iq) of the study: (p, q, target CSR, pattern (n_F, edges, None), colouring
    seed).  Every point has its own seeded target and pattern; td None asks the library for a
    minimum-width decomposition, as the paper computes one (Section 3)."""
    probs = er_phase_probs(spec["step"])
    p, q = probs[ip], probs[iq]
    base = spec["seed"] * 1_000_003
    g = erdos_renyi(spec["n_target"], p, base + 1000 * ip + iq)
    pg = erdos_renyi(spec["n_pattern"], q, base + 500_000 + 1000 * iq + ip)
    edges = edges_from_csr(*pg).astype(np.int32)
    return p, q, g, (spec["n_pattern"], edges, None), base + 7 * (1000 * ip + iq) + 1


def ktree_batch(spec):
    """The pattern batch of a batched workload: `patterns` random partial k-trees (k = width) with
    n_F uniform in sizes (numpy seed 1), pattern i from seed pattern_seed + i."""
    rng = np.random.default_rng(1)
    lo, hi = spec["sizes"]
    return [random_partial_ktree(int(rng.integers(lo, hi + 1)), spec["width"],
                                 spec["pattern_seed"] + i) for i in range(spec["patterns"])]


def serve_stream(spec, count=None):
    """The query stream of a serving workload: a list of dicts with the arrival time (s), the
    pattern spec (as make_pattern takes it), k and the colouring seed.  Families are uniform over
    path, cycle, grid and random partial k-tree; n_F = k is uniform in sizes; a grid family
    drawn for a size no grid has is drawn again.  Random partial k-trees take k (their width)
    uniform in 1..min(3, n_F - 1) and a pattern seed from a pool of `ktree_pool` per (n_F, k),
    so that queries repeat patterns as a served population would."""
    rng = np.random.default_rng(spec["seed"])
    lo, hi = spec["sizes"]
    n = spec["queries"] if count is None else min(count, spec["queries"])
    out, t = [], 0.0
    for _ in range(n):
        t += float(rng.exponential(1.0 / spec["rate"]))
        nF = int(rng.integers(lo, hi + 1))
        while True:
            fam = ("path", "cycle", "grid", "ktree")[int(rng.integers(0, 4))]
            if fam != "grid" or nF in GRID_SHAPES:
                break
        if fam == "grid":
            pat = ("grid",) + GRID_SHAPES[nF]
        elif fam == "ktree":
            w = int(rng.integers(1, min(3, nF - 1) + 1))
            pat = ("ktree", nF, w, 1000 * nF + 10 * w + int(rng.integers(0, spec["ktree_pool"])))
        else:
            pat = (fam, nF)
        out.append(dict(t=t, pattern=pat, k=nF, seed=int(rng.integers(1, 1 << 62)),
                        trials=spec["trials"]))
    return out


def make_graph(spec):
    kind = spec[0]
    if kind == "er":
        return erdos_renyi(spec[1], spec[2], spec[3])
    if kind == "ba":
        return barabasi_albert(spec[1], spec[2], spec[3])
    if kind == "pl":
        return power_law_config(spec[1], spec[2], spec[3], spec[4])
    if kind == "complete":
        return complete_graph(spec[1])
    if kind == "cycle":
        return cycle_graph(spec[1])
    raise ValueError(kind)


def make_pattern(spec):
    kind = spec[0]
    if kind == "path":
        return path_pattern(spec[1])
    if kind == "cycle":
        return cycle_pattern(spec[1])
    if kind == "star":
        return star_pattern(spec[1])
    if kind == "clique":
        return clique_pattern(spec[1])
    if kind == "grid":
        return grid_pattern(spec[1], spec[2])
    if kind == "ktree":
        return random_partial_ktree(spec[1], spec[2], spec[3])
    if kind in ("A", "B", "C", "D"):
        return {"A": pattern_A, "B": pattern_B, "C": pattern_C, "D": pattern_D}[kind]()
    raise ValueError(kind)


def random_colors(n, trials, k, seed):
    """Explicit colourings (uint8[trials, n]) from numpy, for inputs given as colours."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, k, size=(trials, n), dtype=np.uint8)
