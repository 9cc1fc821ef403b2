// CPU oracle for the colour-coding dynamic programme of Malik, Suchy and Valla (arXiv 1908.11248).
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct restatement of the
// paper's method that the GPU library is checked against.  Only the test suite, the smoke check
// and the CPU-baseline leg of the benchmark load it.  It shares no code, header, table or helper
// with the GPU library, and the GPU library never calls it.
//
// What it computes (all integer, no floating point):
//   * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel random numbers: as easy as
//     1, 2, 3"), restated from the published round function and key schedule, and the random
//     k-colouring drawn from it (Section 2.1: a uniform colour per host vertex).
//   * The nice tree decomposition built from a given tree decomposition (Section 1.2, Definition
//     of a nice tree decomposition, with leaf bags of size one; Section 3).
//   * The bottom-up table D_x of every node (Section 3.1, "Dynamic Programming Description"),
//     one std::map per node keyed by (ordered bag tuple phi, colour set C), extended from the
//     paper's Boolean table to a count of colourful embeddings of F[V*_x] (mod 2^64).
//   * The root test (Section 3.1, last paragraph) and result reconstruction R(x, M) (Section 4).
//   * A second, independent oracle: plain backtracking over V(F) in breadth-first order.
//
// Conventions (readings of the paper):
//   * colours are 0-based; bit i of a colour set is colour i (Section 3.2, colour sets).
//   * bags are ordered by increasing F-vertex id (Section 3.2, representation of mappings).
//   * the degree filter deg_G(x) >= deg_F(y) (Section 3.2, masking unprofitable mappings) is a
//     switch; it never changes the root result.
//   * the extended input of that paragraph, per host vertex the set of pattern vertices that may
//     be mapped to it, is an optional mask array (bit y of allow[x]: y may map to x); maps that
//     break it are not counted anywhere.
//   * the distance bound of Section 3.2 (mapping expansion) is a switch: an introduced vertex u
//     with no neighbour in the bag takes only the host vertices within distance d of phi(w),
//     where w is the bag vertex nearest to u in F (the first in bag order among the nearest) and
//     d = dist_F(w, u); a vertex with no bag vertex in its F-component takes every host vertex.
//     It never changes the root result.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <utility>
#include <vector>

namespace {

// ------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11, Section 5: the Philox S-box and its Weyl key schedule)
// ------------------------------------------------------------------------------------------
const uint32_t PHILOX_M0 = 0xD2511F53u;
const uint32_t PHILOX_M1 = 0xCD9E8D57u;
const uint32_t PHILOX_W0 = 0x9E3779B9u;  // golden ratio
const uint32_t PHILOX_W1 = 0xBB67AE85u;  // sqrt(3) - 1

void philox_round(uint32_t x[4], const uint32_t k[2]) {
  uint64_t p0 = (uint64_t)PHILOX_M0 * x[0];
  uint64_t p1 = (uint64_t)PHILOX_M1 * x[2];
  uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  uint32_t y0 = hi1 ^ x[1] ^ k[0];
  uint32_t y1 = lo1;
  uint32_t y2 = hi0 ^ x[3] ^ k[1];
  uint32_t y3 = lo0;
  x[0] = y0; x[1] = y1; x[2] = y2; x[3] = y3;
}

void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k[2] = {key[0], key[1]};
  for (int r = 0; r < 10; ++r) {
    philox_round(x, k);
    k[0] += PHILOX_W0;
    k[1] += PHILOX_W1;
  }
  for (int i = 0; i < 4; ++i) out[i] = x[i];
}

// colour of host vertex v in trial t: first Philox word of counter (v, t, 0, 0) under key
// (seed low word, seed high word), scaled to [0, k) by a 32-bit fixed-point multiply.
uint8_t colour_of(uint64_t seed, uint32_t v, uint32_t t, uint32_t k) {
  uint32_t ctr[4] = {v, t, 0u, 0u};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t out[4];
  philox4x32_10(ctr, key, out);
  return (uint8_t)(((uint64_t)out[0] * k) >> 32);
}

// ------------------------------------------------------------------------------------------
// graphs
// ------------------------------------------------------------------------------------------
struct Graph {
  int32_t n = 0;
  std::vector<int32_t> row_ptr, col;
  int32_t deg(int32_t v) const { return row_ptr[v + 1] - row_ptr[v]; }
  bool adjacent(int32_t a, int32_t b) const {  // rows are sorted
    return std::binary_search(col.begin() + row_ptr[a], col.begin() + row_ptr[a + 1], b);
  }
  // the host vertices within distance r of a (a itself included), increasing: breadth-first
  // search stopped at depth r
  std::vector<int32_t> ball(int32_t a, int32_t r) const {
    std::vector<int32_t> depth(n, -1), q{a};
    depth[a] = 0;
    for (size_t h = 0; h < q.size(); ++h) {
      const int32_t x = q[h];
      if (depth[x] == r) continue;
      for (int32_t i = row_ptr[x]; i < row_ptr[x + 1]; ++i)
        if (depth[col[i]] < 0) {
          depth[col[i]] = depth[x] + 1;
          q.push_back(col[i]);
        }
    }
    std::sort(q.begin(), q.end());
    return q;
  }
};

struct Pattern {
  int32_t n = 0;
  std::vector<std::vector<char>> adj;  // adjacency matrix of F
  std::vector<int32_t> deg;
  // breadth-first distances from a in F (-1: another component)
  std::vector<int32_t> dist(int32_t a) const {
    std::vector<int32_t> d(n, -1), q{a};
    d[a] = 0;
    for (size_t h = 0; h < q.size(); ++h)
      for (int32_t b = 0; b < n; ++b)
        if (adj[q[h]][b] && d[b] < 0) {
          d[b] = d[q[h]] + 1;
          q.push_back(b);
        }
    return d;
  }
};

Pattern make_pattern(int32_t nF, int32_t mF, const int32_t *edges) {
  Pattern F;
  F.n = nF;
  F.adj.assign(nF, std::vector<char>(nF, 0));
  F.deg.assign(nF, 0);
  for (int32_t i = 0; i < mF; ++i) {
    int32_t a = edges[2 * i], b = edges[2 * i + 1];
    if (a != b && !F.adj[a][b]) {
      F.adj[a][b] = F.adj[b][a] = 1;
      F.deg[a]++;
      F.deg[b]++;
    }
  }
  return F;
}

// ------------------------------------------------------------------------------------------
// nice tree decomposition (Section 1.2 definitions; Section 3, conversion after Cygan et al.)
// ------------------------------------------------------------------------------------------
enum NodeType { LEAF = 0, INTRODUCE = 1, FORGET = 2, JOIN = 3 };

struct NiceNode {
  int32_t type;
  int32_t child0 = -1, child1 = -1;
  int32_t vertex = -1;          // leaf vertex, introduced or forgotten vertex
  std::vector<int32_t> bag;     // sorted
};

struct NiceTD {
  std::vector<NiceNode> nodes;  // post-order; the root (empty bag) is last
};

int32_t push_forget(NiceTD &T, int32_t top, int32_t u) {
  NiceNode f;
  f.type = FORGET;
  f.child0 = top;
  f.vertex = u;
  for (int32_t w : T.nodes[top].bag)
    if (w != u) f.bag.push_back(w);
  T.nodes.push_back(f);
  return (int32_t)T.nodes.size() - 1;
}

bool in_bag(const NiceTD &T, int32_t node, int32_t u) {
  const std::vector<int32_t> &b = T.nodes[node].bag;
  return std::find(b.begin(), b.end(), u) != b.end();
}

// Introduces the vertices `add` on top of node `top`, one introduce node each, while the
// decomposition bag `target` is being built.  The paper does not fix their order; we take, each
// time, the smallest remaining vertex that has an F-neighbour in the current bag, or the
// smallest remaining vertex if none has, so that an introduce finds its candidates in adjacency
// lists whenever F allows (Section 3.2, mapping expansion).  Nor does it fix where forgets go:
// a vertex of `drop` (vertices of `target` absent from the next bag up) is forgotten, in
// increasing vertex order, as soon as every F-neighbour it has in `target` has been in the bag,
// except when that would empty the bag before an introduce.
int32_t introduce_all(NiceTD &T, const Pattern &F, int32_t top, std::vector<int32_t> add,
                      const std::vector<int32_t> &drop, const std::vector<int32_t> &target) {
  std::sort(add.begin(), add.end());
  std::vector<char> gone(F.n, 0);
  auto forget_ripe = [&](int32_t t) {
    for (int32_t q : drop) {
      if (!in_bag(T, t, q)) continue;
      bool waiting = false;  // an F-neighbour of q in the target bag not yet in the bag
      for (int32_t w : target)
        if (F.adj[q][w] && !in_bag(T, t, w) && !gone[w]) waiting = true;
      if (waiting) continue;
      if (T.nodes[t].bag.size() == 1 && !add.empty()) continue;
      t = push_forget(T, t, q);
      gone[q] = 1;
    }
    return t;
  };
  top = forget_ripe(top);
  while (!add.empty()) {
    size_t pick = 0;
    for (size_t j = 0; j < add.size(); ++j) {
      bool anchored = false;
      for (int32_t w : T.nodes[top].bag) anchored = anchored || F.adj[add[j]][w];
      if (anchored) {
        pick = j;
        break;
      }
    }
    int32_t u = add[pick];
    add.erase(add.begin() + pick);
    NiceNode in;
    in.type = INTRODUCE;
    in.child0 = top;
    in.vertex = u;
    in.bag = T.nodes[top].bag;
    in.bag.push_back(u);
    std::sort(in.bag.begin(), in.bag.end());
    T.nodes.push_back(in);
    top = forget_ripe((int32_t)T.nodes.size() - 1);
  }
  return top;
}

// Vertices of decomposition bag i that its parent's bag lacks (all of them at the root).
std::vector<int32_t> leaving_bag(const std::vector<std::vector<int32_t>> &bags,
                                 const std::vector<int32_t> &parent, int32_t i) {
  std::vector<int32_t> d;
  for (int32_t u : bags[i])
    if (parent[i] < 0 ||
        std::find(bags[parent[i]].begin(), bags[parent[i]].end(), u) == bags[parent[i]].end())
      d.push_back(u);
  return d;
}

// Builds the nice decomposition rooted at decomposition node i: its top node has bag B_i minus
// the vertices of B_i that left early (those B_i does not pass to its parent).  Children of a
// decomposition node are taken in increasing id; going from a child's bag to B_i first forgets
// what remains of B_c \ B_i in increasing vertex order, then introduces B_i \ B_c (order of
// introduce_all, with early forgets unless several children must be joined at B_i); several
// children are combined by left-deep joins.  A leaf bag becomes a size-one leaf node holding its
// smallest vertex followed by introductions of the rest.
int32_t nice_build(NiceTD &T, const Pattern &F, const std::vector<std::vector<int32_t>> &bags,
                   const std::vector<int32_t> &parent,
                   const std::vector<std::vector<int32_t>> &kids, int32_t i) {
  const std::vector<int32_t> &B = bags[i];
  const std::vector<int32_t> none;
  if (kids[i].empty()) {
    NiceNode leaf;
    leaf.type = LEAF;
    leaf.vertex = B[0];
    leaf.bag = {B[0]};
    T.nodes.push_back(leaf);
    int32_t top = (int32_t)T.nodes.size() - 1;
    return introduce_all(T, F, top, std::vector<int32_t>(B.begin() + 1, B.end()),
                         leaving_bag(bags, parent, i), B);
  }
  std::vector<int32_t> tops;
  for (int32_t c : kids[i]) {
    int32_t top = nice_build(T, F, bags, parent, kids, c);
    const std::vector<int32_t> &Bc = bags[c];
    for (int32_t u : Bc) {
      if (std::find(B.begin(), B.end(), u) != B.end()) continue;
      if (in_bag(T, top, u)) top = push_forget(T, top, u);
    }
    std::vector<int32_t> add;
    for (int32_t u : B)
      if (std::find(Bc.begin(), Bc.end(), u) == Bc.end()) add.push_back(u);
    top = introduce_all(T, F, top, add,
                        kids[i].size() == 1 ? leaving_bag(bags, parent, i) : none, B);
    tops.push_back(top);
  }
  int32_t top = tops[0];
  for (size_t j = 1; j < tops.size(); ++j) {
    NiceNode jn;
    jn.type = JOIN;
    jn.child0 = top;
    jn.child1 = tops[j];
    jn.bag = T.nodes[top].bag;
    T.nodes.push_back(jn);
    top = (int32_t)T.nodes.size() - 1;
  }
  return top;
}

// returns false when (bags, parent) is not a tree decomposition of F with nonempty bags
bool make_nice(const Pattern &F, int32_t nbags, const int32_t *bag_ptr, const int32_t *bag_vtx,
               const int32_t *parent, NiceTD &T) {
  if (nbags <= 0) return false;
  std::vector<std::vector<int32_t>> bags(nbags), kids(nbags);
  int32_t root = -1;
  for (int32_t i = 0; i < nbags; ++i) {
    for (int32_t j = bag_ptr[i]; j < bag_ptr[i + 1]; ++j) {
      int32_t u = bag_vtx[j];
      if (u < 0 || u >= F.n) return false;
      bags[i].push_back(u);
    }
    std::sort(bags[i].begin(), bags[i].end());
    if (bags[i].empty()) return false;
    if (std::adjacent_find(bags[i].begin(), bags[i].end()) != bags[i].end()) return false;
    if (parent[i] < 0) {
      if (root >= 0) return false;
      root = i;
    } else {
      if (parent[i] >= nbags) return false;
      kids[parent[i]].push_back(i);
    }
  }
  if (root < 0) return false;
  // the parent pointers must form one tree: every node reaches the root
  for (int32_t i = 0; i < nbags; ++i) {
    int32_t x = i, steps = 0;
    while (parent[x] >= 0 && steps <= nbags) { x = parent[x]; ++steps; }
    if (x != root) return false;
  }
  // (i) every vertex in a bag; (ii) every edge in a bag; (iii) bags holding u are connected
  for (int32_t u = 0; u < F.n; ++u) {
    int32_t holders = 0, tops = 0;
    for (int32_t i = 0; i < nbags; ++i) {
      bool in = std::binary_search(bags[i].begin(), bags[i].end(), u);
      if (!in) continue;
      ++holders;
      bool pin = parent[i] >= 0 &&
                 std::binary_search(bags[parent[i]].begin(), bags[parent[i]].end(), u);
      if (!pin) ++tops;
    }
    if (holders == 0 || tops != 1) return false;
  }
  for (int32_t a = 0; a < F.n; ++a)
    for (int32_t b = a + 1; b < F.n; ++b) {
      if (!F.adj[a][b]) continue;
      bool ok = false;
      for (int32_t i = 0; i < nbags && !ok; ++i)
        ok = std::binary_search(bags[i].begin(), bags[i].end(), a) &&
             std::binary_search(bags[i].begin(), bags[i].end(), b);
      if (!ok) return false;
    }
  T.nodes.clear();
  std::vector<int32_t> par(parent, parent + nbags);
  int32_t top = nice_build(T, F, bags, par, kids, root);
  for (int32_t u : bags[root])
    if (in_bag(T, top, u)) top = push_forget(T, top, u);
  return true;
}

int32_t pos_in(const std::vector<int32_t> &bag, int32_t u) {
  return (int32_t)(std::lower_bound(bag.begin(), bag.end(), u) - bag.begin());
}

// ------------------------------------------------------------------------------------------
// the dynamic programme (Section 3.1), counting colourful embeddings mod 2^64
// ------------------------------------------------------------------------------------------
typedef std::pair<std::vector<int32_t>, uint32_t> Key;  // (phi as ordered bag tuple, colour set C)
typedef std::map<Key, uint64_t> Table;

struct Run {
  Graph G;
  Pattern F;
  NiceTD T;
  int32_t k = 0, trials = 0;
  bool degree_filter = true;
  bool distance_prune = false;
  std::vector<uint32_t> allow;           // empty: every mapping allowed
  std::vector<uint8_t> colours;          // trials * n
  std::vector<std::vector<Table>> D;     // [trial][node]
  std::vector<uint8_t> exists;
  std::vector<uint64_t> count;
};

void run_trial(Run &R, int32_t t) {
  const Graph &G = R.G;
  const Pattern &F = R.F;
  const uint8_t *zeta = &R.colours[(size_t)t * G.n];
  std::vector<Table> &D = R.D[t];
  D.assign(R.T.nodes.size(), Table());
  for (size_t x = 0; x < R.T.nodes.size(); ++x) {
    const NiceNode &nd = R.T.nodes[x];
    Table &Dx = D[x];
    if (nd.type == LEAF) {
      // every host vertex, with the singleton colour set of its colour
      int32_t u = nd.vertex;
      for (int32_t v = 0; v < G.n; ++v) {
        if (R.degree_filter && G.deg(v) < F.deg[u]) continue;
        if (!R.allow.empty() && !((R.allow[v] >> u) & 1u)) continue;
        Dx[Key({v}, 1u << zeta[v])] += 1;
      }
    } else if (nd.type == INTRODUCE) {
      // extend phi' by u -> v: the colour of v is new to C', and every edge of F[V_x] at u
      // is realised in G.  Candidates are the neighbours of the image of one bag neighbour of
      // u when u has one (Section 3.2, mapping expansion), all of V(G) otherwise.
      const NiceNode &ch = R.T.nodes[nd.child0];
      int32_t u = nd.vertex;
      int32_t p = pos_in(nd.bag, u);
      std::vector<int32_t> nb_slots;  // slots in the child tuple of u's bag neighbours
      for (size_t s = 0; s < ch.bag.size(); ++s)
        if (F.adj[u][ch.bag[s]]) nb_slots.push_back((int32_t)s);
      // distance bound: the bag vertex w of u's component nearest to u (first in bag order
      // among the nearest) and its F-distance to u
      int32_t near_slot = -1, near_dist = -1;
      if (nb_slots.empty() && R.distance_prune) {
        const std::vector<int32_t> du = F.dist(u);
        for (size_t s = 0; s < ch.bag.size(); ++s) {
          const int32_t d = du[ch.bag[s]];
          if (d >= 0 && (near_dist < 0 || d < near_dist)) {
            near_dist = d;
            near_slot = (int32_t)s;
          }
        }
      }
      for (const auto &e : D[nd.child0]) {
        const std::vector<int32_t> &phi_c = e.first.first;
        uint32_t Cc = e.first.second;
        std::vector<int32_t> cand;
        if (!nb_slots.empty()) {
          int32_t a = phi_c[nb_slots[0]];
          cand.assign(G.col.begin() + G.row_ptr[a], G.col.begin() + G.row_ptr[a + 1]);
        } else if (near_slot >= 0) {  // the host vertices within distance d of phi(w)
          cand = G.ball(phi_c[near_slot], near_dist);
        } else {
          cand.resize(G.n);
          for (int32_t v = 0; v < G.n; ++v) cand[v] = v;
        }
        for (int32_t v : cand) {
          if ((Cc >> zeta[v]) & 1u) continue;
          if (R.degree_filter && G.deg(v) < F.deg[u]) continue;
          if (!R.allow.empty() && !((R.allow[v] >> u) & 1u)) continue;
          bool ok = true;
          for (int32_t s : nb_slots)
            if (!G.adjacent(phi_c[s], v)) { ok = false; break; }
          if (!ok) continue;
          std::vector<int32_t> phi(phi_c);
          phi.insert(phi.begin() + p, v);
          Dx[Key(phi, Cc | (1u << zeta[v]))] += e.second;
        }
      }
    } else if (nd.type == FORGET) {
      // restrict phi' to V_x; colour sets carry over; equal results are merged (summed)
      const NiceNode &ch = R.T.nodes[nd.child0];
      int32_t p = pos_in(ch.bag, nd.vertex);
      for (const auto &e : D[nd.child0]) {
        std::vector<int32_t> phi(e.first.first);
        phi.erase(phi.begin() + p);
        Dx[Key(phi, e.first.second)] += e.second;
      }
    } else {  // JOIN
      // equal mappings in both children; C' and C'' may share exactly the bag's colours
      const Table &Dy = D[nd.child0];
      const Table &Dz = D[nd.child1];
      for (const auto &ey : Dy) {
        const std::vector<int32_t> &phi = ey.first.first;
        uint32_t bagc = 0;
        for (int32_t v : phi) bagc |= 1u << zeta[v];
        for (auto it = Dz.lower_bound(Key(phi, 0u)); it != Dz.end() && it->first.first == phi;
             ++it) {
          uint32_t C1 = ey.first.second, C2 = it->first.second;
          if ((C1 & C2) != bagc) continue;
          Dx[Key(phi, C1 | C2)] += ey.second * it->second;
        }
      }
    }
  }
  // root: empty bag; a solution exists iff its table is nonempty (Section 3.1)
  const Table &Dr = D.back();
  R.exists[t] = Dr.empty() ? 0 : 1;
  uint64_t c = 0;
  for (const auto &e : Dr) c += e.second;
  R.count[t] = c;
}

// ------------------------------------------------------------------------------------------
// result reconstruction R(x, M) (Section 4), per trial
// ------------------------------------------------------------------------------------------
typedef std::vector<int32_t> Phi;  // full map V(F) -> V(G), -1 where unassigned

std::vector<std::vector<Phi>> reconstruct(const Run &R, int32_t t, int32_t x,
                                          const std::vector<Key> &M) {
  const NiceNode &nd = R.T.nodes[x];
  const uint8_t *zeta = &R.colours[(size_t)t * R.G.n];
  const std::vector<Table> &D = R.D[t];
  std::vector<std::vector<Phi>> L(M.size());
  if (nd.type == LEAF) {
    for (size_t i = 0; i < M.size(); ++i) {
      Phi P(R.F.n, -1);
      P[nd.vertex] = M[i].first[0];
      L[i].push_back(P);
    }
  } else if (nd.type == INTRODUCE) {
    int32_t p = pos_in(nd.bag, nd.vertex);
    std::vector<Key> Mh(M.size());
    for (size_t i = 0; i < M.size(); ++i) {
      std::vector<int32_t> phi(M[i].first);
      int32_t v = phi[p];
      phi.erase(phi.begin() + p);
      Mh[i] = Key(phi, M[i].second & ~(1u << zeta[v]));
    }
    std::vector<std::vector<Phi>> Lh = reconstruct(R, t, nd.child0, Mh);
    for (size_t i = 0; i < M.size(); ++i)
      for (Phi P : Lh[i]) {
        P[nd.vertex] = M[i].first[p];
        L[i].push_back(P);
      }
  } else if (nd.type == FORGET) {
    const NiceNode &ch = R.T.nodes[nd.child0];
    int32_t p = pos_in(ch.bag, nd.vertex);
    // scan D_y once, grouping its pairs by (restriction to V_x, colour set)
    std::map<Key, std::vector<Key>> by_restriction;
    for (const auto &e : D[nd.child0]) {
      std::vector<int32_t> phi(e.first.first);
      phi.erase(phi.begin() + p);
      by_restriction[Key(phi, e.first.second)].push_back(e.first);
    }
    std::vector<Key> Mh;
    std::vector<std::pair<size_t, size_t>> range(M.size());
    for (size_t i = 0; i < M.size(); ++i) {
      size_t b = Mh.size();
      auto it = by_restriction.find(M[i]);
      if (it != by_restriction.end())
        for (const Key &k2 : it->second) Mh.push_back(k2);
      range[i] = {b, Mh.size()};
    }
    std::vector<std::vector<Phi>> Lh = reconstruct(R, t, nd.child0, Mh);
    for (size_t i = 0; i < M.size(); ++i)
      for (size_t j = range[i].first; j < range[i].second; ++j)
        for (const Phi &P : Lh[j]) L[i].push_back(P);
  } else {  // JOIN
    const Table &Dy = D[nd.child0];
    const Table &Dz = D[nd.child1];
    std::vector<Key> M1, M2;
    std::vector<std::pair<size_t, size_t>> range(M.size());
    for (size_t i = 0; i < M.size(); ++i) {
      const std::vector<int32_t> &phi = M[i].first;
      uint32_t bagc = 0;
      for (int32_t v : phi) bagc |= 1u << zeta[v];
      size_t b = M1.size();
      for (auto iy = Dy.lower_bound(Key(phi, 0u)); iy != Dy.end() && iy->first.first == phi; ++iy)
        for (auto iz = Dz.lower_bound(Key(phi, 0u)); iz != Dz.end() && iz->first.first == phi;
             ++iz) {
          uint32_t C1 = iy->first.second, C2 = iz->first.second;
          if ((C1 | C2) == M[i].second && (C1 & C2) == bagc) {
            M1.push_back(iy->first);
            M2.push_back(iz->first);
          }
        }
      range[i] = {b, M1.size()};
    }
    std::vector<std::vector<Phi>> L1 = reconstruct(R, t, nd.child0, M1);
    std::vector<std::vector<Phi>> L2 = reconstruct(R, t, nd.child1, M2);
    for (size_t i = 0; i < M.size(); ++i)
      for (size_t j = range[i].first; j < range[i].second; ++j)
        for (const Phi &P1 : L1[j])
          for (const Phi &P2 : L2[j]) {
            Phi P(P1);
            for (int32_t u = 0; u < R.F.n; ++u)
              if (P2[u] >= 0) P[u] = P2[u];
            L[i].push_back(P);
          }
  }
  return L;
}

// ------------------------------------------------------------------------------------------
// second oracle: backtracking over V(F) in breadth-first order
// ------------------------------------------------------------------------------------------
struct Backtrack {
  const Graph *G;
  const Pattern *F;
  const uint8_t *zeta;
  std::vector<int32_t> order, anchor;  // anchor[i]: an earlier neighbour of order[i], or -1
  std::vector<int32_t> img;
  uint64_t count = 0;
  uint64_t limit = 0;
  std::vector<Phi> found;
  bool degree_filter = false;

  void rec(size_t i, uint32_t used) {
    if (i == order.size()) {
      ++count;
      if (found.size() < limit) found.push_back(img);
      return;
    }
    int32_t u = order[i];
    auto try_v = [&](int32_t v) {
      if ((used >> zeta[v]) & 1u) return;
      if (degree_filter && G->deg(v) < F->deg[u]) return;
      for (size_t j = 0; j < i; ++j) {
        int32_t w = order[j];
        if (F->adj[u][w] && !G->adjacent(img[w], v)) return;
      }
      img[u] = v;
      rec(i + 1, used | (1u << zeta[v]));
      img[u] = -1;
    };
    if (anchor[i] >= 0) {
      int32_t a = img[anchor[i]];
      for (int32_t j = G->row_ptr[a]; j < G->row_ptr[a + 1]; ++j) try_v(G->col[j]);
    } else {
      for (int32_t v = 0; v < G->n; ++v) try_v(v);
    }
  }
};

Graph make_graph(int32_t n, const int32_t *row_ptr, const int32_t *col) {
  Graph G;
  G.n = n;
  G.row_ptr.assign(row_ptr, row_ptr + n + 1);
  G.col.assign(col, col + row_ptr[n]);
  return G;
}

}  // namespace

extern "C" {

void or_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out) {
  philox4x32_10(ctr, key, out);
}

void or_color(int32_t n, int32_t trials, int32_t k, uint64_t seed, uint8_t *out) {
  for (int32_t t = 0; t < trials; ++t)
    for (int32_t v = 0; v < n; ++v) out[(size_t)t * n + v] = colour_of(seed, v, t, k);
}

// Nice decomposition of F from (bag_ptr, bag_vtx, parent).  Writes node arrays in post-order
// (root last) and returns the node count, -1 for an invalid decomposition, -2 if max_nodes is
// too small.  bag_out_ptr has max_nodes+1 entries; bag_out_vtx holds up to max_nodes*n_F.
int32_t or_nice_td(int32_t nF, int32_t mF, const int32_t *edges, int32_t nbags,
                   const int32_t *bag_ptr, const int32_t *bag_vtx, const int32_t *parent,
                   int32_t max_nodes, int32_t *type, int32_t *child0, int32_t *child1,
                   int32_t *vertex, int32_t *bag_out_ptr, int32_t *bag_out_vtx) {
  Pattern F = make_pattern(nF, mF, edges);
  NiceTD T;
  if (!make_nice(F, nbags, bag_ptr, bag_vtx, parent, T)) return -1;
  if ((int32_t)T.nodes.size() > max_nodes) return -2;
  int32_t off = 0;
  for (size_t i = 0; i < T.nodes.size(); ++i) {
    type[i] = T.nodes[i].type;
    child0[i] = T.nodes[i].child0;
    child1[i] = T.nodes[i].child1;
    vertex[i] = T.nodes[i].vertex;
    bag_out_ptr[i] = off;
    for (int32_t u : T.nodes[i].bag) bag_out_vtx[off++] = u;
  }
  bag_out_ptr[T.nodes.size()] = off;
  return (int32_t)T.nodes.size();
}

// Runs the DP for every trial.  Returns an opaque handle, or nullptr for an invalid input.
void *or_dp_run(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t nF, int32_t mF,
                const int32_t *edges, int32_t nbags, const int32_t *bag_ptr,
                const int32_t *bag_vtx, const int32_t *parent, const uint8_t *colours,
                int32_t trials, int32_t k, int32_t degree_filter, const uint32_t *allow,
                int32_t distance_prune) {
  if (nF < 1 || nF > 32 || k < nF || k > 32 || trials < 1 || n < 0) return nullptr;
  Run *R = new Run();
  R->G = make_graph(n, row_ptr, col);
  R->F = make_pattern(nF, mF, edges);
  if (!make_nice(R->F, nbags, bag_ptr, bag_vtx, parent, R->T)) {
    delete R;
    return nullptr;
  }
  R->k = k;
  R->trials = trials;
  R->degree_filter = degree_filter != 0;
  R->distance_prune = distance_prune != 0;
  if (allow) R->allow.assign(allow, allow + n);
  R->colours.assign(colours, colours + (size_t)trials * n);
  R->D.resize(trials);
  R->exists.assign(trials, 0);
  R->count.assign(trials, 0);
  for (int32_t t = 0; t < trials; ++t) run_trial(*R, t);
  return R;
}

void or_dp_free(void *h) { delete (Run *)h; }

int32_t or_dp_num_nodes(void *h) { return (int32_t)((Run *)h)->T.nodes.size(); }

void or_dp_results(void *h, uint8_t *exists, uint64_t *count, uint64_t *node_sizes) {
  Run *R = (Run *)h;
  size_t N = R->T.nodes.size();
  for (int32_t t = 0; t < R->trials; ++t) {
    exists[t] = R->exists[t];
    count[t] = R->count[t];
    for (size_t x = 0; x < N; ++x) node_sizes[(size_t)t * N + x] = R->D[t][x].size();
  }
}

// Table of (trial, node) in key order: per entry the bag tuple (bag size int32), then the colour
// set and the count.  Arrays must hold node_sizes entries.
void or_dp_table(void *h, int32_t t, int32_t x, int32_t *phi, uint32_t *mask, uint64_t *cnt) {
  Run *R = (Run *)h;
  size_t b = R->T.nodes[x].bag.size(), i = 0;
  for (const auto &e : R->D[t][x]) {
    for (size_t s = 0; s < b; ++s) phi[i * b + s] = e.first.first[s];
    mask[i] = e.first.second;
    cnt[i] = e.second;
    ++i;
  }
}

// Every embedding of the run's trials reconstructed from the root (Section 4), as the
// lexicographically sorted union over trials without repeats, truncated to `limit` rows of
// n_F ints.  Returns the number of distinct embeddings before truncation; *n_per_trial_sum
// gets the sum over trials of the per-trial list lengths.
uint64_t or_enumerate(void *h, uint64_t limit, int32_t *out, uint64_t *n_per_trial_sum) {
  Run *R = (Run *)h;
  std::vector<Phi> all;
  uint64_t per_trial = 0;
  for (int32_t t = 0; t < R->trials; ++t) {
    const Table &Dr = R->D[t].back();
    std::vector<Key> M;
    for (const auto &e : Dr) M.push_back(e.first);
    std::vector<std::vector<Phi>> L = reconstruct(*R, t, (int32_t)R->T.nodes.size() - 1, M);
    for (const auto &l : L)
      for (const Phi &P : l) {
        all.push_back(P);
        ++per_trial;
      }
  }
  std::sort(all.begin(), all.end());
  all.erase(std::unique(all.begin(), all.end()), all.end());
  if (n_per_trial_sum) *n_per_trial_sum = per_trial;
  uint64_t m = std::min<uint64_t>(limit, all.size());
  for (uint64_t i = 0; i < m; ++i)
    for (int32_t u = 0; u < R->F.n; ++u) out[i * R->F.n + u] = all[i][u];
  return all.size();
}

// Second oracle: the number of colourful embeddings of F in G under one colouring, by plain
// backtracking, and the first `limit` of them in lexicographic order.  Returns the count.
uint64_t or_backtrack(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t nF,
                      int32_t mF, const int32_t *edges, const uint8_t *colours,
                      int32_t degree_filter, uint64_t limit, int32_t *out, uint64_t *n_out) {
  Graph G = make_graph(n, row_ptr, col);
  Pattern F = make_pattern(nF, mF, edges);
  Backtrack B;
  B.G = &G;
  B.F = &F;
  B.zeta = colours;
  B.degree_filter = degree_filter != 0;
  B.limit = limit ? ~0ull : 0ull;
  // breadth-first order over F, component by component
  std::vector<char> seen(nF, 0);
  for (int32_t s = 0; s < nF; ++s) {
    if (seen[s]) continue;
    seen[s] = 1;
    B.order.push_back(s);
    B.anchor.push_back(-1);
    for (size_t q = B.order.size() - 1; q < B.order.size(); ++q) {
      int32_t u = B.order[q];
      for (int32_t w = 0; w < nF; ++w)
        if (F.adj[u][w] && !seen[w]) {
          seen[w] = 1;
          B.order.push_back(w);
          B.anchor.push_back(u);
        }
    }
  }
  B.img.assign(nF, -1);
  B.rec(0, 0u);
  std::sort(B.found.begin(), B.found.end());
  uint64_t m = std::min<uint64_t>(limit, B.found.size());
  for (uint64_t i = 0; i < m; ++i)
    for (int32_t u = 0; u < nF; ++u) out[i * nF + u] = B.found[i][u];
  if (n_out) *n_out = m;
  return B.count;
}

}  // extern "C"
