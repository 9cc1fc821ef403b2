"""Brute-force definitions used to pin the oracle on tiny inputs (pure Python, no oracle code).

Everything here is the plain definition, enumerated exhaustively:
  * a colourful embedding (Section 1, SubIso; Section 2.1, colourful copy) is an injective map
    Phi: V(F) -> V(G) that keeps every edge of F and gives its image distinct colours;
  * the table value D(x, phi, C) (Section 2.1, semantics of the table) counted: the number of
    colourful embeddings of F[V*_x] that agree with phi on the bag V_x and use exactly colours C.
"""
from __future__ import annotations

from collections import Counter
from itertools import permutations

import numpy as np


def adj_sets(row_ptr, col):
    n = len(row_ptr) - 1
    return [set(int(c) for c in col[row_ptr[v]:row_ptr[v + 1]]) for v in range(n)]


def embeddings(G, nF, edges, zeta=None, verts=None):
    """All colourful embeddings of F[verts] (default: all of F) as dicts u -> v.  zeta=None
    drops the colour condition (plain injective homomorphisms)."""
    adj = G
    n = len(adj)
    verts = list(range(nF)) if verts is None else sorted(verts)
    vs = set(verts)
    E = [(int(a), int(b)) for a, b in np.asarray(edges).reshape(-1, 2) if a in vs and b in vs]
    out = []
    for img in permutations(range(n), len(verts)):
        m = dict(zip(verts, img))
        if any(m[b] not in adj[m[a]] for a, b in E):
            continue
        if zeta is not None and len({int(zeta[v]) for v in img}) != len(img):
            continue
        out.append(m)
    return out


def count_embeddings(G, nF, edges, zeta):
    return len(embeddings(G, nF, edges, zeta))


def vstar(nodes):
    """V*_x for every node of a nice decomposition given as (type, c0, c1, vertex, bag)."""
    vs = []
    for (ty, c0, c1, u, bag) in nodes:
        s = set(bag)
        for c in (c0, c1):
            if c >= 0:
                s |= vs[c]
        vs.append(s)
    return vs


def node_table(G, nF, edges, zeta, bag, verts, degG=None, degF=None, allow=None):
    """D(x, ., .) by definition: Counter over (phi tuple in bag order, colour set) of colourful
    embeddings of F[verts].  With degG/degF given, only maps with deg_G(Phi(y)) >= deg_F(y)
    for every y are counted (the degree filter of Section 3.2); with allow given, only maps with
    bit y of allow[Phi(y)] set for every y (the extended input of the same paragraph)."""
    tab = Counter()
    for m in embeddings(G, nF, edges, zeta, verts):
        if degG is not None and any(degG[m[y]] < degF[y] for y in m):
            continue
        if allow is not None and any(not (int(allow[m[y]]) >> y) & 1 for y in m):
            continue
        C = 0
        for v in m.values():
            C |= 1 << int(zeta[v])
        tab[(tuple(m[u] for u in bag), C)] += 1
    return tab


def _reach_through(adj, S, v):
    """Q(S, v): the vertices outside S and v that some path from v reaches with every inner
    vertex in S."""
    seen, stack, out = {v}, [v], set()
    while stack:
        x = stack.pop()
        for y in adj[x]:
            if y in seen:
                continue
            seen.add(y)
            if y in S:
                stack.append(y)
            else:
                out.add(y)
    return out


def exact_treewidth(n, edges):
    """Treewidth by definition through elimination orderings: TW(S) = min over v in S of
    max(TW(S - v), |Q(S - v, v)|) over all vertex subsets S (Bodlaender, Fomin, Koster, Kratsch,
    Thilikos), tw = TW(V); plain dictionary over frozensets, for n up to about 12."""
    adj = [set() for _ in range(n)]
    for a, b in np.asarray(edges).reshape(-1, 2):
        adj[int(a)].add(int(b))
        adj[int(b)].add(int(a))
    tw = {frozenset(): -1}
    for size in range(1, n + 1):
        for S in map(frozenset, __import__("itertools").combinations(range(n), size)):
            tw[S] = min(max(tw[S - {v}], len(_reach_through(adj, S - {v}, v))) for v in S)
    return max(0, tw[frozenset(range(n))])


def elimination_td(n, edges):
    """A tree decomposition (bags, parent) from the greedy minimum-degree elimination ordering:
    bag(v) = v and its neighbours when v is eliminated (which then become a clique); the parent
    of bag(v) is the bag of the first-eliminated of those neighbours; bags whose vertex has no
    later neighbour (one per connected component) are chained under the last one."""
    adj = [set() for _ in range(n)]
    for a, b in np.asarray(edges).reshape(-1, 2):
        adj[int(a)].add(int(b))
        adj[int(b)].add(int(a))
    left, order, nbrs = set(range(n)), [], {}
    while left:
        v = min(left, key=lambda x: (len(adj[x] & left), x))
        nb = adj[v] & left - {v}
        nbrs[v] = nb
        for a in nb:
            adj[a] |= nb - {a}
        left.remove(v)
        order.append(v)
    pos = {v: i for i, v in enumerate(order)}
    bags = [sorted({v} | nbrs[v]) for v in order]
    parent, roots = [], []
    for i, v in enumerate(order):
        if nbrs[v]:
            parent.append(pos[min(nbrs[v], key=lambda a: pos[a])])
        else:
            parent.append(-1)
            roots.append(i)
    for a, b in zip(roots, roots[1:]):
        parent[a] = b
    return bags, parent
