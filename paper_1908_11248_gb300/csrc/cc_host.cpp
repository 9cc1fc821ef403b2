// Host runtime of the colour-coding library: the C ABI of include/cc.h.
//
// It owns the device arena, validates and uploads the host graph, turns a pattern and its tree
// decomposition into a nice decomposition (Section 1.2, Section 3), plans every node's table and
// issues the node kernels of cc_kernels.cu in post-order (Section 3.1).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/cc.h"
#include "cc_internal.h"
#include "cc_runtime.h"

using cc::DevInfo;
using cc::KeyLayout;
using cc::TableDesc;
using cc::u64;
using cc::Arena;
using cc::Ctx;
using cc::NiceNode;
using cc::Pattern;
using cc::Run;

namespace cc {
namespace rt {

#define CUDA_OK(expr)                               \
  do {                                              \
    cudaError_t e_ = (expr);                        \
    if (e_ != cudaSuccess) return CC_ECUDA;         \
  } while (0)

int check_launch(int r) { return r == 0 ? CC_OK : CC_ECUDA; }

int bits_for(u64 x) {  // bits to hold values 0..x
  int b = 0;
  while ((x >> b) != 0) ++b;
  return b;
}

// capacity for `entries` keys at fill `lf`, rounded up to a whole 256-byte line of records
u64 hash_cap(u64 entries, float lf) {
  double want = (double)std::max<u64>(entries, 1) / (double)lf;
  u64 c = (u64)want + 16;
  return (c + 15) & ~u64(15);
}

// ---- nice tree decomposition (Section 1.2; Section 3, after Cygan et al.) ------------------
bool valid_td(const std::vector<uint32_t> &adj, int nF, const std::vector<std::vector<int>> &bags,
              const std::vector<int> &parent, int &root) {
  int nb = (int)bags.size();
  if (nb == 0) return false;
  root = -1;
  for (int i = 0; i < nb; ++i) {
    if (bags[i].empty()) return false;
    if (parent[i] < 0) {
      if (root >= 0) return false;
      root = i;
    } else if (parent[i] >= nb || parent[i] == i) {
      return false;
    }
  }
  if (root < 0) return false;
  for (int i = 0; i < nb; ++i) {  // acyclic, reaches the root
    int x = i, steps = 0;
    while (parent[x] >= 0 && steps <= nb) {
      x = parent[x];
      ++steps;
    }
    if (x != root) return false;
  }
  std::vector<uint32_t> bm(nb, 0);
  for (int i = 0; i < nb; ++i)
    for (int u : bags[i]) {
      if (u < 0 || u >= nF || (bm[i] >> u & 1u)) return false;
      bm[i] |= 1u << u;
    }
  for (int u = 0; u < nF; ++u) {  // (i) covered, (iii) connected: exactly one topmost bag
    int tops = 0, holders = 0;
    for (int i = 0; i < nb; ++i) {
      if (!(bm[i] >> u & 1u)) continue;
      ++holders;
      if (parent[i] < 0 || !(bm[parent[i]] >> u & 1u)) ++tops;
    }
    if (holders == 0 || tops != 1) return false;
  }
  for (int a = 0; a < nF; ++a)  // (ii) every edge in some bag
    for (int b = a + 1; b < nF; ++b) {
      if (!(adj[a] >> b & 1u)) continue;
      bool ok = false;
      for (int i = 0; i < nb && !ok; ++i) ok = (bm[i] >> a & 1u) && (bm[i] >> b & 1u);
      if (!ok) return false;
    }
  return true;
}

void build_nice(const std::vector<uint32_t> &adj, const std::vector<std::vector<int>> &bags_in,
                const std::vector<int> &parent, int root, std::vector<NiceNode> &out) {
  int nb = (int)bags_in.size();
  std::vector<std::vector<int>> bags(bags_in), kids(nb);
  for (auto &b : bags) std::sort(b.begin(), b.end());
  for (int i = 0; i < nb; ++i)
    if (parent[i] >= 0) kids[parent[i]].push_back(i);  // increasing id
  out.clear();
  auto push = [&](NiceNode nd) {
    out.push_back(nd);
    return (int)out.size() - 1;
  };
  auto contains = [](const std::vector<int> &v, int u) {
    return std::binary_search(v.begin(), v.end(), u);
  };
  auto forget_node = [&](int t, int u) {
    NiceNode f;
    f.type = 2;
    f.child0 = t;
    f.vertex = u;
    for (int w : out[t].bag)
      if (w != u) f.bag.push_back(w);
    return push(f);
  };
  // Introduces `todo` (increasing) on top of node t while building decomposition bag `target`:
  // each step takes the smallest vertex with an F-neighbour already in the bag, else the
  // smallest, so introduces are anchored in adjacency lists whenever the pattern allows.  A
  // vertex of `drop` (vertices of `target` that the next bag up no longer holds) is forgotten as
  // soon as all its F-neighbours in `target` are in the bag (increasing order, never emptying
  // the bag while introduces remain): no later node needs it, and a forget taken before an
  // introduce of a non-neighbour shrinks that introduce's table
  auto introduce_all = [&](int t, std::vector<int> todo, const std::vector<int> &drop,
                           const std::vector<int> &target) {
    uint32_t tmask = 0, gone = 0;  // gone: forgotten early in this chain
    for (int w : target) tmask |= 1u << w;
    auto early_forgets = [&](int t0) {
      for (int q : drop) {
        uint32_t bagmask = 0;
        for (int w : out[t0].bag) bagmask |= 1u << w;
        if (!(bagmask >> q & 1u)) continue;
        if ((adj[q] & tmask & ~(bagmask | gone)) != 0) continue;  // a neighbour still to come
        if (out[t0].bag.size() == 1 && !todo.empty()) continue;
        t0 = forget_node(t0, q);
        gone |= 1u << q;
      }
      return t0;
    };
    t = early_forgets(t);
    while (!todo.empty()) {
      uint32_t bagmask = 0;
      for (int w : out[t].bag) bagmask |= 1u << w;
      size_t pick = 0;
      for (size_t j = 0; j < todo.size(); ++j)
        if (adj[todo[j]] & bagmask) {
          pick = j;
          break;
        }
      int u = todo[pick];
      todo.erase(todo.begin() + pick);
      NiceNode in;
      in.type = 1;
      in.child0 = t;
      in.vertex = u;
      in.bag = out[t].bag;
      in.bag.insert(std::upper_bound(in.bag.begin(), in.bag.end(), u), u);
      t = push(in);
      t = early_forgets(t);
    }
    return t;
  };
  // the vertices of bag i that the next bag up no longer holds (all of them at the root)
  auto leaving = [&](int i) {
    std::vector<int> d;
    for (int u : bags[i])
      if (parent[i] < 0 || !contains(bags[parent[i]], u)) d.push_back(u);
    return d;
  };
  // chain from child bag `c` to its parent bag p on top of node t: forgets (increasing vertex
  // order) of what is still in the bag and not in B_p, then the introduces of B_p \ B_c, with
  // early forgets of B_p's leaving vertices when p has no other child (a join needs all of B_p)
  auto transition = [&](int t, int c, int p) {
    const std::vector<int> &from = bags[c], &to = bags[p];
    for (int u : from)
      if (!contains(to, u) && contains(out[t].bag, u)) t = forget_node(t, u);
    std::vector<int> todo;
    for (int u : to)
      if (!contains(from, u)) todo.push_back(u);
    const std::vector<int> none;
    return kids[p].size() == 1 ? introduce_all(t, todo, leaving(p), to)
                               : introduce_all(t, todo, none, to);
  };
  // explicit post-order walk of the decomposition tree; a finished child's subtree is followed
  // at once by its transition to the parent's bag, and a node with several children joins their
  // transitioned tops left-deep
  std::vector<int> top(nb, -1);
  std::vector<std::pair<int, size_t>> stack{{root, 0}};
  while (!stack.empty()) {
    int i = stack.back().first;
    size_t &next = stack.back().second;
    if (next < kids[i].size()) {
      int c = kids[i][next++];
      stack.push_back({c, 0});
      continue;
    }
    stack.pop_back();
    const std::vector<int> &B = bags[i];
    int t = -1;
    if (kids[i].empty()) {
      NiceNode leaf;
      leaf.type = 0;
      leaf.vertex = B[0];
      leaf.bag = {B[0]};
      t = introduce_all(push(leaf), std::vector<int>(B.begin() + 1, B.end()), leaving(i), B);
    } else {
      for (int c : kids[i]) {
        if (t < 0) {
          t = top[c];
        } else {
          NiceNode j;
          j.type = 3;
          j.child0 = t;
          j.child1 = top[c];
          j.bag = out[t].bag;
          t = push(j);
        }
      }
    }
    top[i] = (parent[i] >= 0) ? transition(t, i, parent[i]) : t;
  }
  int t = top[root];
  for (int u : bags[root])  // empty-bag root of degree one
    if (contains(out[t].bag, u)) t = forget_node(t, u);
  for (size_t i = 0; i < out.size(); ++i) {
    if (out[i].child0 >= 0) out[out[i].child0].parent = (int)i;
    if (out[i].child1 >= 0) out[out[i].child1].parent = (int)i;
  }
}

// ---- minimum-width decomposition from elimination orderings (Section 3) -------------------
// Exact dynamic programme over vertex subsets (Bodlaender, Fomin, Koster, Kratsch, Thilikos):
// TW(S) = min over v in S of max(TW(S - v), |Q(S - v, v)|), where Q(S, v) holds the vertices
// outside S + v reachable from v through S; the minimiser gives the elimination order.
uint32_t q_set(const std::vector<uint32_t> &adj, uint32_t S, int v) {
  uint32_t seen = 1u << v, reach = adj[v];
  uint32_t inner = reach & S & ~seen;
  while (inner) {
    int x = __builtin_ctz(inner);
    seen |= 1u << x;
    reach |= adj[x];
    inner = reach & S & ~seen;
  }
  return reach & ~S & ~(1u << v);
}

std::vector<int> exact_order(const std::vector<uint32_t> &adj, int n) {
  size_t N = size_t(1) << n;
  std::vector<int8_t> tw(N);
  std::vector<uint8_t> arg(N);
  tw[0] = -1;
  for (size_t S = 1; S < N; ++S) {
    int best = 127, bv = 0;
    for (uint32_t rest = (uint32_t)S; rest; rest &= rest - 1) {
      int v = __builtin_ctz(rest);
      uint32_t Sm = (uint32_t)S & ~(1u << v);
      int val = std::max<int>(tw[Sm], __builtin_popcount(q_set(adj, Sm, v)));
      if (val < best) {
        best = val;
        bv = v;
      }
    }
    tw[S] = (int8_t)best;
    arg[S] = (uint8_t)bv;
  }
  std::vector<int> order(n);
  uint32_t S = (uint32_t)(N - 1);
  for (int i = n - 1; i >= 0; --i) {
    order[i] = arg[S];
    S &= ~(1u << arg[S]);
  }
  return order;
}

std::vector<int> min_fill_order(std::vector<uint32_t> adj, int n) {
  std::vector<int> order;
  uint32_t left = n == 32 ? ~0u : ((1u << n) - 1u);
  while (left) {
    int best = -1, bf = INT32_MAX;
    for (uint32_t r = left; r; r &= r - 1) {
      int v = __builtin_ctz(r);
      uint32_t nb = adj[v] & left;
      int fill = 0;
      for (uint32_t a = nb; a; a &= a - 1) {
        int x = __builtin_ctz(a);
        fill += __builtin_popcount(nb & ~adj[x] & ~(1u << x));
      }
      if (fill < bf) {
        bf = fill;
        best = v;
      }
    }
    uint32_t nb = adj[best] & left;
    for (uint32_t a = nb; a; a &= a - 1) {
      int x = __builtin_ctz(a);
      adj[x] |= nb & ~(1u << x);
    }
    left &= ~(1u << best);
    order.push_back(best);
  }
  return order;
}

void td_from_order(std::vector<uint32_t> adj, int n, const std::vector<int> &order,
                   std::vector<std::vector<int>> &bags, std::vector<int> &parent) {
  std::vector<int> pos(n);
  for (int i = 0; i < n; ++i) pos[order[i]] = i;
  std::vector<uint32_t> later(n);
  for (int i = 0; i < n; ++i) {
    int v = order[i];
    uint32_t hi = 0;
    for (uint32_t a = adj[v]; a; a &= a - 1) {
      int x = __builtin_ctz(a);
      if (pos[x] > i) hi |= 1u << x;
    }
    later[i] = hi;
    for (uint32_t a = hi; a; a &= a - 1) {  // fill: the later neighbours become a clique
      int x = __builtin_ctz(a);
      adj[x] |= hi & ~(1u << x);
    }
  }
  bags.assign(n, {});
  parent.assign(n, -1);
  int root = -1;
  for (int i = 0; i < n; ++i) {
    bags[i].push_back(order[i]);
    int first = n;
    for (uint32_t a = later[i]; a; a &= a - 1) {
      int x = __builtin_ctz(a);
      bags[i].push_back(x);
      first = std::min(first, pos[x]);
    }
    parent[i] = first < n ? first : -1;
  }
  // bags without a parent belong to different components: hang them under the last one
  for (int i = n - 1; i >= 0; --i)
    if (parent[i] < 0) {
      if (root < 0) root = i;
      else parent[i] = root;
    }
}

// ---- helpers ------------------------------------------------------------------------------
Arena &active_arena(Ctx *c) { return c->active ? *c->active : c->arena; }

void free_run(Ctx *c, Run *r) {
  Arena &H = r->home ? *r->home : c->arena;
  for (auto &t : r->timings) {
    cudaEventDestroy(t.start);
    cudaEventDestroy(t.stop);
  }
  r->timings.clear();
  for (auto &t : r->tables)
    if (t.slots) H.release(t.slots);
  r->tables.clear();
  H.release(r->d_counters);
  H.release(r->d_exists);
  H.release(r->d_count);
  H.release(r->d_blk);
  H.release(r->d_err);
  r->d_blk = nullptr;
  r->d_err = nullptr;
  auto it = c->colorings.find(r->coloring);
  if (it != c->colorings.end() && --it->second.refs == 0) {
    c->arena.release(it->second.d_colors);
    c->colorings.erase(it);
  }
}

int ensure_scratch(Ctx *c, size_t words) {
  if (c->scratch_words >= words) return CC_OK;
  c->arena.release(c->d_scratch);
  c->d_scratch = arena_alloc<u64>(c, words);
  c->scratch_words = c->d_scratch ? words : 0;
  return c->d_scratch ? CC_OK : CC_ENOMEM;
}

int read_u64(Ctx *c, const u64 *d, u64 *h) {
  CUDA_OK(cudaMemcpyAsync(h, d, sizeof(u64), cudaMemcpyDeviceToHost, c->stream));
  CUDA_OK(cudaStreamSynchronize(c->stream));
  return CC_OK;
}

int pos_in(const std::vector<int32_t> &bag, int u) {
  return (int)(std::lower_bound(bag.begin(), bag.end(), u) - bag.begin());
}

// ---- the planner: node by node in post-order, exact capacities ----------------------------
int finish_run(Ctx *c, Run *R);
int near_slot(const Pattern &P, int u, const std::vector<int32_t> &child_bag, int *dist);

// Runs every node of the nice decomposition in post-order (Section 3.1).
//
// Exact mode (plan == nullptr): introduces first count their entries and joins their colour-set
// pairs; every table gets exactly the room it needs, and sizes are read back node by node.
// Planned mode: capacities come from earlier exact runs of the same pattern, graph, trials,
// colours and options (a little larger); there are no count passes and no host reads until the
// end, introduces append in chunks (leaving holes that consumers skip), and all sizes stay on
// the device.  If any table outgrew its planned room the run reports CC_ECAPACITY and the
// caller repeats it in exact mode.
int run_nodes(Ctx *c, Run *R, const Pattern &P, const cc::Coloring &col, const cc::Plan *plan) {
  const int N = (int)P.nodes.size();
  const int32_t n = c->n;
  const float lf = R->opts.load_factor;
  const int block = R->opts.block;
  const int df = R->opts.degree_filter;
  const bool planned = plan != nullptr;
  cc::GraphDev G{c->d_row_ptr, c->d_col, col.d_colors, n, c->d_deg8, P.d_allow};
  R->tables.assign(N, {});
  R->sizes.assign(N, 0);
  R->pairs.assign(N, 0);
  R->checks.clear();
  std::vector<bool> made(N, false);
  const int grid = cc::intro_grid(c->dev, block);
  Arena &A = active_arena(c);
  // per-run scratch (a captured graph's branches must not share it)
  if (!R->d_blk) R->d_blk = arena_alloc<u64>(c, 2 * (size_t)std::max(grid, cc::sort_grid(c->dev)) + 8);
  if (!R->d_err) R->d_err = arena_alloc<int>(c, 1);
  if (!R->d_blk || !R->d_err) return CC_ENOMEM;
  int rc = CC_OK;
  u64 *blk = R->d_blk;
  u64 *cursor = R->d_counters + N;      // per node: chunked-append cursor (scan bound)
  u64 *pairs_dev = R->d_counters + 2 * N;  // per join: matching colour-set pairs
  CUDA_OK(cudaMemsetAsync(R->d_err, 0, sizeof(int), c->stream));
  const size_t rb = cc::slot_bytes(R->kw);
  // planned room for a quantity last seen at v (plus slack for chunked appends)
  const u64 chunk_slack = (u64)grid * 2048;
  auto room = [&](u64 v) { return v + v / 4 + 4096; };

  // every launch goes through `timed`: it counts the launch and, when profiling, brackets it
  // with CUDA events on the context's stream
  auto timed = [&](int node, int kind, int kernels, auto &&launch) -> int {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (R->opts.profile) {
      if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return CC_ECUDA;
      if (cudaEventRecord(e0, c->stream) != cudaSuccess) return CC_ECUDA;
    }
    int r = check_launch(launch());
    c->launches += kernels;
    if (R->opts.profile) {
      if (cudaEventRecord(e1, c->stream) != cudaSuccess) return CC_ECUDA;
      R->timings.push_back({node, kind, e0, e1, 0});
    }
    return r;
  };
  auto release_child = [&](int y) {
    if (R->opts.retain || y < 0) return;
    A.release(R->tables[y].slots);
    R->tables[y] = {};
  };
  auto desc = [&](int x) {
    TableDesc t;
    t.slots = R->tables[x].slots;
    t.cap = R->tables[x].cap;
    t.count = R->tables[x].bound ? R->tables[x].bound : R->d_counters + x;
    t.hashed = R->tables[x].hashed;
    return t;
  };
  // entries of node x: exact size, or planned room
  auto entries = [&](int x) { return planned ? room(plan->entries[x]) : R->sizes[x]; };
  auto new_hash = [&](int x, u64 keys) -> int {
    u64 cap = hash_cap(keys, lf);
    void *p = A.alloc(cap * rb);
    if (!p) return CC_ENOMEM;
    CUDA_OK(cudaMemsetAsync(p, 0, cap * rb, c->stream));
    R->tables[x] = {p, cap, 1, true};
    return CC_OK;
  };
  // true if table t is sorted with exactly the slots sl[0..n) (in any order) most significant
  auto sorted_by = [&](const cc::NodeTable &t, int m, const int *sl) {
    if (t.hashed || t.sort_n < m || m < t.sort_min) return false;
    for (int j = 0; j < m; ++j) {
      bool in = false;
      for (int i = 0; i < m; ++i) in = in || t.sort_slots[i] == sl[j];
      if (!in) return false;
    }
    return true;
  };
  // true if table t comes in runs of equal images of exactly the slots sl[0..m), sorted or
  // clustered (a grouped introduce then shares candidate lists without sorting it; its results
  // do not depend on the runs being whole)
  auto grouped_by = [&](const cc::NodeTable &t, int m, const int *sl) {
    if (sorted_by(t, m, sl)) return true;
    if (t.hashed || t.cluster_n < m || m < t.cluster_min) return false;
    for (int j = 0; j < m; ++j) {
      bool in = false;
      for (int i = 0; i < m; ++i) in = in || t.cluster_slots[i] == sl[j];
      if (!in) return false;
    }
    return true;
  };
  // chained introduces (option chain): introduce x1 with a bag neighbour, under an introduce
  // x2 of a vertex not adjacent to x1's that has >= 2 bag neighbours (all of them in x1's child
  // y) and whose table is not added into a forget's hash; returns x2 and fills x2's
  // bag-neighbour slots counted in y's bag, else -1 (structure only: y's order is checked when
  // x1 is reached)
  auto chain_parent = [&](int x1, int *nb2, int *nnb2) -> int {
    if (!R->opts.chain || !R->opts.group) return -1;
    const NiceNode &n1 = P.nodes[x1];
    if (n1.type != 1 || n1.parent < 0) return -1;
    const int x2 = n1.parent;
    const NiceNode &n2 = P.nodes[x2];
    if (n2.type != 1 || (P.adj[n2.vertex] >> n1.vertex & 1u)) return -1;
    const NiceNode &ny = P.nodes[n1.child0];
    int k1 = 0, k2 = 0;
    for (size_t s = 0; s < ny.bag.size(); ++s) {
      if (P.adj[n1.vertex] >> ny.bag[s] & 1u) ++k1;
      if (P.adj[n2.vertex] >> ny.bag[s] & 1u) nb2[k2++] = (int)s;
    }
    if (k1 < 1 || k2 < 2 || k2 * R->L.nb > 64) return -1;
    const int f = n2.parent;
    if (f >= 0 && P.nodes[f].type == 2 && R->opts.fuse == 1) return -1;
    *nnb2 = k2;
    return x2;
  };
  std::vector<int> chain_from(N, -1);  // x2 -> the x1 it runs together with
  // full sort order for the table of forget node f: when the next node introduces a vertex
  // with bag neighbours, their slots come first so that its runs are contiguous (when that
  // introduce runs chained with its parent, the parent's bag neighbours come first)
  auto forget_order = [&](int f) {
    const NiceNode &fn = P.nodes[f];
    cc::SortSpec sp{};
    sp.L = R->L;
    sp.b = (int)fn.bag.size();
    sp.full = 1;
    sp.nsl = 0;
    bool used[cc::kMaxBag] = {};
    const int g = fn.parent;
    int nb2[cc::kMaxBag], nnb2 = 0;
    if (g >= 0 && chain_parent(g, nb2, &nnb2) >= 0)
      for (int j = 0; j < nnb2; ++j) {
        sp.order[sp.nsl++] = nb2[j];
        used[nb2[j]] = true;
      }
    if (g >= 0 && P.nodes[g].type == 1)
      for (int s = 0; s < sp.b; ++s)
        if (!used[s] && (P.adj[P.nodes[g].vertex] >> fn.bag[s] & 1u)) {
          sp.order[sp.nsl++] = s;
          used[s] = true;
        }
    int o = sp.nsl;
    for (int s = 0; s < sp.b; ++s)
      if (!used[s]) sp.order[o++] = s;
    sp.bits = sp.b * R->L.nb + R->L.tb + R->L.k;
    return sp;
  };
  // sorts the records of src (scan bound *n_src, at most src_cap slots, *n of them nonempty,
  // at most cap) into a new buffer *out of cap records
  auto sort_records = [&](int node, const cc::SortSpec &sp, const void *src, const u64 *n_src,
                          u64 src_cap, const u64 *nn, u64 cap, void **out) -> int {
    void *ba = A.alloc(std::max<u64>(1, cap) * rb);
    void *bb = A.alloc(std::max<u64>(1, cap) * rb);
    u64 *hist = arena_alloc<u64>(c, 256 * (size_t)cc::sort_grid(c->dev) + 512);
    // one-sweep scratch: tiles of the largest pass input (the scanned source or the buffers)
    cc::SweepScratch sw{};
    sw.max_tiles = std::max(src_cap, cap) / cc::sweep_tile(R->kw) + 2;
    sw.ghist = arena_alloc<u64>(c, 256 * 16);
    sw.tile_ctr = arena_alloc<unsigned>(c, 16);
    sw.status = arena_alloc<u64>(c, 256 * sw.max_tiles);
    sw.err = R->d_err;
    sw.tma = R->opts.sort_sweep == 2;
    if (!ba || !bb || !hist || !sw.ghist || !sw.tile_ctr || !sw.status) {
      A.release(ba);
      A.release(bb);
      A.release(hist);
      A.release(sw.ghist);
      A.release(sw.tile_ctr);
      A.release(sw.status);
      return CC_ENOMEM;
    }
    int which = 0;
    const bool sweep = R->opts.sort_sweep != 0;
    int r = timed(node, CC_K_SORT, sweep ? 2 + cc::sort_passes(sp) : 4 * cc::sort_passes(sp), [&] {
      return cc::launch_sort_records(c->stream, c->dev, R->kw, sp, src, n_src, src_cap, nn, cap,
                                     ba, bb, hist, &which, sweep ? &sw : nullptr);
    });
    A.release(hist);
    A.release(sw.ghist);
    A.release(sw.tile_ctr);
    A.release(sw.status);
    A.release(which ? ba : bb);
    *out = which ? bb : ba;
    return r;
  };
  // in planned mode, device word `w` must end at most `cap`
  auto check = [&](const u64 *w, u64 cap) {
    if (planned) R->checks.push_back({w, cap});
  };

  for (int x = 0; x < N; ++x) {
    if (made[x]) continue;
    const NiceNode &nd = P.nodes[x];
    if (nd.type == 0) {  // leaf
      u64 cap = std::max<u64>(1, (u64)n * (u64)R->trials);
      void *p = A.alloc(cap * rb);
      if (!p) return CC_ENOMEM;
      R->tables[x] = {p, cap, 1, true};
      cc::LeafArgs a{G, R->L, R->trials, df ? P.deg[nd.vertex] : 0, desc(x), R->d_err,
                     1u << nd.vertex};
      if (n == 0) CUDA_OK(cudaMemsetAsync(p, 0, rb, c->stream));
      rc = timed(x, CC_K_LEAF, 1, [&] { return cc::launch_leaf(c->stream, c->dev, R->kw, a); });
      if (rc) return rc;
    } else if (nd.type == 1) {  // introduce
      if (planned) {
        // the lower introduce of a chain: nothing runs now, its parent runs both
        int nb2[cc::kMaxBag], nnb2 = 0;
        const int x2 = chain_parent(x, nb2, &nnb2);
        if (x2 >= 0 && grouped_by(R->tables[nd.child0], nnb2, nb2)) {
          chain_from[x2] = x;
          made[x] = true;
          continue;
        }
      }
      // chained: the input is the lower introduce's child, whose bag lacks that introduce's
      // vertex (slot c_p of the lower bag); this introduce's bag neighbours are all in it
      const int x1 = chain_from[x];
      const int y = x1 >= 0 ? P.nodes[x1].child0 : nd.child0;
      const NiceNode &ch = P.nodes[nd.child0];
      cc::IntroArgs a{};
      a.G = G;
      a.L = R->L;
      a.in = desc(y);
      a.b_in = (int)P.nodes[y].bag.size();
      a.p = pos_in(nd.bag, nd.vertex);
      a.nnb = 0;
      for (size_t s = 0; s < ch.bag.size(); ++s)
        if (P.adj[nd.vertex] >> ch.bag[s] & 1u) a.nb_slot[a.nnb++] = (int)s;
      if (x1 >= 0) {
        const NiceNode &n1 = P.nodes[x1];
        const NiceNode &ny = P.nodes[y];
        a.c_p = pos_in(n1.bag, n1.vertex);
        for (int j = 0; j < a.nnb; ++j) a.nb_slot[j] -= a.nb_slot[j] > a.c_p ? 1 : 0;
        a.c_nnb = 0;
        for (size_t s = 0; s < ny.bag.size(); ++s)
          if (P.adj[n1.vertex] >> ny.bag[s] & 1u) a.c_nb_slot[a.c_nnb++] = (int)s;
        a.c_degF = df ? P.deg[n1.vertex] : 0;
        a.c_ubit = 1u << n1.vertex;
        a.c_valid = R->d_counters + x1;
      }
      if (a.nnb == 0 && R->opts.distance_prune) {
        // distance bound: candidates are the ball of radius dist_F(w, u) around the image of
        // the nearest bag vertex w, walked like an adjacency list (no other bag neighbour is
        // then checked)
        int dist = 0;
        const int s = near_slot(P, nd.vertex, ch.bag, &dist);
        auto bl = c->balls.find(dist);
        if (s >= 0 && bl != c->balls.end()) {
          a.nnb = 1;
          a.nb_slot[0] = s;
          a.G.row_ptr = bl->second.first;
          a.G.col = bl->second.second;
        }
      }
      a.degF = df ? P.deg[nd.vertex] : 0;
      a.ubit = 1u << nd.vertex;
      a.err = R->d_err;
      a.cand = R->d_counters + 3 * N + x;  // candidates examined (count pass, or planned)
      a.proj_q = -1;
      a.q = -1;
      // several bag neighbours: the child must come in runs of equal images of those slots so
      // that a run shares one candidate list; sort it unless its order already starts with them
      const int grouped = R->opts.group && a.nnb >= 2 && a.nnb * R->L.nb <= 64;
      void *sorted = nullptr;
      if (grouped && !grouped_by(R->tables[y], a.nnb, a.nb_slot)) {
        cc::SortSpec sp{};
        sp.L = R->L;
        sp.b = a.b_in;
        sp.nsl = a.nnb;
        for (int j = 0; j < a.nnb; ++j) sp.order[j] = a.nb_slot[j];
        sp.full = 0;
        sp.bits = a.nnb * R->L.nb;
        const cc::NodeTable &ty = R->tables[y];
        const u64 m = entries(y);
        check(R->d_counters + y, m);
        rc = sort_records(x, sp, ty.slots, ty.hashed ? c->d_ones : desc(y).count, ty.cap,
                          R->d_counters + y, m, &sorted);
        if (rc) return rc;
        a.in = TableDesc{sorted, std::max<u64>(1, m), R->d_counters + y, 0};
      }
      struct SortedGuard {
        Arena &a;
        void *p;
        ~SortedGuard() { a.release(p); }
      } sorted_guard{A, sorted};
      u64 total = 0, cand = 0;
      if (!planned) {
        rc = timed(x, CC_K_INTRO_COUNT, 2, [&] {
          return cc::launch_intro_blk(c->stream, c->dev, R->kw, 0, grouped, block, a, blk);
        });
        if (rc) return rc;
        rc = read_u64(c, blk + 2 * grid, &total);
        if (!rc) rc = read_u64(c, a.cand, &cand);
        if (rc) return rc;
        if (R->opts.profile) R->timings.back().candidates = cand;
        R->sizes[x] = total;
      }
      // room for this introduce's entries: exact, or planned plus the holes chunked appends
      // may leave (one partial chunk per warp, or per block for the block kernel); a warp's
      // chunk shrinks for small tables so that those holes stay under a quarter of the entries
      const bool warp_path = planned && (a.nnb <= 1 || grouped);
      a.chunk = 256;
      u64 slack = chunk_slack;
      if (warp_path) {
        const u64 warps = (u64)c->dev.sms * c->dev.blocks_per_sm * 8;
        while (a.chunk > 32 && warps * a.chunk * 4 > plan->entries[x]) a.chunk >>= 1;
        slack = warps * a.chunk;
      }
      const u64 raw = planned ? room(plan->entries[x]) + slack : std::max<u64>(1, total);
      if (planned) check(R->d_counters + x, room(plan->entries[x]));
      auto write_dense = [&](void *buf, u64 cap, int proj) -> int {
        a.out = TableDesc{buf, cap, nullptr, 0};
        a.proj_q = proj;
        a.valid = R->d_counters + x;
        a.cursor = planned ? cursor + x : nullptr;
        a.cand = planned ? R->d_counters + 3 * N + x : nullptr;
        if (planned) check(cursor + x, cap);
        // planned runs: lean warp kernels (expanding, or grouped by bag-neighbour images, or
        // two introduces chained)
        const bool warp = planned && a.nnb <= 1, gwarp = planned && grouped;
        // chained, the lower introduce with one bag neighbour: colour counts of every host
        // vertex's neighbours let entries whose runs have no upper candidate count their lower
        // extensions without walking the adjacency
        u64 *hist = nullptr;
        if (x1 >= 0 && a.c_nnb == 1 && R->L.k <= 16 && c->max_deg < 65536)
          hist = arena_alloc<u64>(c, (size_t)R->trials * (size_t)n * 4);
        a.c_hist = hist;
        int r = timed(x, x1 >= 0 ? CC_K_INTRO_CHAIN : CC_K_INTRO_WRITE, hist ? 2 : 1, [&] {
          if (hist) {
            const int h = cc::launch_nb_colour_hist(c->stream, c->dev, a.G, R->trials, a.c_degF,
                                                    a.c_ubit, hist, a.cand);
            if (h) return h;
          }
          return x1 >= 0 ? cc::launch_intro_chain(c->stream, c->dev, R->kw, a)
                 : warp  ? cc::launch_intro_warp(c->stream, c->dev, R->kw, 1, a)
                 : gwarp ? cc::launch_intro_group_warp(c->stream, c->dev, R->kw, 1, a)
                         : cc::launch_intro_blk(c->stream, c->dev, R->kw, 1, grouped, block, a,
                                                blk);
        });
        A.release(hist);
        if (R->opts.profile && !r) R->timings.back().candidates = cand;
        return r;
      };
      const int f = nd.parent;
      const int fuse = (f >= 0 && P.nodes[f].type == 2) ? R->opts.fuse : 0;
      if (fuse == 1) {  // add projected entries into the forget's hash table
        rc = new_hash(f, planned ? room(plan->entries[f]) : total);
        if (rc) return rc;
        a.out = desc(f);
        a.q = pos_in(nd.bag, P.nodes[f].vertex);
        a.valid = R->d_counters + x;
        a.cand = planned ? R->d_counters + 3 * N + x : nullptr;
        const bool warp = planned && a.nnb <= 1, gwarp = planned && grouped;
        rc = timed(x, CC_K_INTRO_FUSED, 1, [&] {
          return warp    ? cc::launch_intro_warp(c->stream, c->dev, R->kw, 2, a)
                 : gwarp ? cc::launch_intro_group_warp(c->stream, c->dev, R->kw, 2, a)
                         : cc::launch_intro_blk(c->stream, c->dev, R->kw, 2, grouped, block, a,
                                                blk);
        });
        if (rc) return rc;
        if (R->opts.profile) R->timings.back().candidates = cand;
        made[f] = true;
        release_child(y);
        if (!planned) {
          rc = read_u64(c, R->d_counters + f, &R->sizes[f]);
          if (rc) return rc;
        }
        if (f == N - 1) break;
        continue;
      }
      if (fuse == 2 && R->opts.sort_sweep == 3) {
        // write projected entries densely, then the bucketed merge: split by a hash of the next
        // introduce's bag-neighbour images, sort and merge each bucket in shared memory
        void *buf = A.alloc(raw * rb);
        if (!buf) return CC_ENOMEM;
        rc = write_dense(buf, raw, pos_in(nd.bag, P.nodes[f].vertex));
        if (!rc) release_child(y);
        cc::SortSpec sp = forget_order(f);
        const u64 records = planned ? room(plan->entries[x]) : std::max<u64>(1, total);
        sp.hbits = R->opts.part_bits > 0 ? std::min(20, R->opts.part_bits)
                                         : cc::part_bucket_bits(records, R->kw);
        // buckets by the images of all bag slots: equal images stay in one run (so do those of
        // any prefix of the order that holds them all) while the records sharing them are few
        // (colour sets times trials); a one-slot bag hashes the whole key
        sp.hslots = sp.b >= 2 ? sp.b : 0;
        const u64 F = 1ull << sp.hbits;
        const u64 *bound = planned ? cursor + x : R->d_counters + x;
        void *mid = A.alloc(raw * rb);
        void *spare = sp.hbits > 10 ? A.alloc(raw * rb) : nullptr;
        void *out = A.alloc(raw * rb);
        cc::PartScratch ps{};
        ps.hist = arena_alloc<unsigned>(c, F);
        ps.base = arena_alloc<u64>(c, F + 1);
        ps.cur1 = arena_alloc<u64>(c, 1024);
        ps.cur2 = arena_alloc<u64>(c, F);
        ps.status = arena_alloc<u64>(c, F);
        ps.claim = arena_alloc<unsigned>(c, 1);
        ps.scan = arena_alloc<u64>(c, cc::scan_scratch_words(c->dev) + 8);
        ps.err = R->d_err;
        auto give_back = [&]() {
          A.release(buf);
          A.release(mid);
          A.release(spare);
          A.release(ps.hist);
          A.release(ps.base);
          A.release(ps.cur1);
          A.release(ps.cur2);
          A.release(ps.status);
          A.release(ps.claim);
          A.release(ps.scan);
        };
        if (!mid || (sp.hbits > 10 && !spare) || !out || !ps.hist || !ps.base || !ps.cur1 ||
            !ps.cur2 || !ps.status || !ps.claim || !ps.scan) {
          give_back();
          A.release(out);
          return CC_ENOMEM;
        }
        if (!rc)
          rc = timed(f, CC_K_MERGE, 7 + (sp.hbits > 10 ? 1 : 0), [&] {
            return cc::launch_part_merge(c->stream, c->dev, R->kw, sp, buf, bound, raw, mid,
                                         spare, raw, ps, out, raw, R->d_counters + f);
          });
        give_back();
        if (rc) {
          A.release(out);
          return rc;
        }
        if (planned) check(R->d_counters + f, raw);
        R->tables[f] = {out, raw, 0, true};
        R->tables[f].sort_n = sp.b;
        R->tables[f].sort_min = sp.hslots ? sp.hslots : sp.b + 1;
        R->tables[f].sort_hbits = sp.hbits;
        R->tables[f].sort_hslots = sp.hslots;
        for (int j = 0; j < sp.b; ++j) R->tables[f].sort_slots[j] = sp.order[j];
        made[f] = true;
        if (!planned) {
          rc = read_u64(c, R->d_counters + f, &R->sizes[f]);
          if (rc) return rc;
        }
        if (f == N - 1) break;
        continue;
      }
      if (fuse == 2) {  // write projected entries densely, sort them, reduce equal keys
        void *buf = A.alloc(raw * rb);
        if (!buf) return CC_ENOMEM;
        rc = write_dense(buf, raw, pos_in(nd.bag, P.nodes[f].vertex));
        if (!rc) release_child(y);
        cc::SortSpec sp = forget_order(f);
        void *srt = nullptr;
        // scan bound of the written buffer: its cursor when appended in chunks
        const u64 *bound = planned ? cursor + x : R->d_counters + x;
        if (!rc) rc = sort_records(f, sp, buf, bound, raw, R->d_counters + x, raw, &srt);
        A.release(buf);
        if (rc) return rc;
        void *out = A.alloc(raw * rb);
        if (!out) {
          A.release(srt);
          return CC_ENOMEM;
        }
        const bool narrow = cc::sort_narrows(R->kw, sp, R->opts.sort_sweep);
        rc = timed(f, CC_K_REDUCE, 3, [&] {
          return cc::launch_reduce(c->stream, c->dev, R->kw, srt, R->d_counters + x, raw, blk, out,
                                   R->d_counters + f, R->opts.sort_sweep ? &sp : nullptr,
                                   narrow);
        });
        A.release(srt);
        if (rc) return rc;
        R->tables[f] = {out, raw, 0, true};
        R->tables[f].sort_n = sp.b;
        for (int j = 0; j < sp.b; ++j) R->tables[f].sort_slots[j] = sp.order[j];
        made[f] = true;
        if (!planned) {
          rc = read_u64(c, R->d_counters + f, &R->sizes[f]);
          if (rc) return rc;
        }
        if (f == N - 1) break;
        continue;
      }
      // the entries of a child sorted or clustered by some slots come out in runs of equal
      // images of those slots: the ungrouped kernels emit each child entry's extensions
      // together, in child order
      int cl_n = 0, cl_min = 0, cl[cc::kMaxBag];
      if (!grouped) {
        const cc::NodeTable &ty = R->tables[y];
        const int *src = ty.sort_n ? ty.sort_slots : ty.cluster_slots;
        cl_n = ty.sort_n ? ty.sort_n : ty.cluster_n;
        cl_min = ty.sort_n ? ty.sort_min : ty.cluster_min;
        for (int j = 0; j < cl_n; ++j) cl[j] = src[j] + (src[j] >= a.p ? 1 : 0);
      }
      void *p = A.alloc(raw * rb);
      if (!p) return CC_ENOMEM;
      rc = write_dense(p, raw, -1);
      if (rc) return rc;
      R->tables[x] = {p, raw, 0, true};
      R->tables[x].cluster_n = cl_n;
      R->tables[x].cluster_min = cl_min;
      for (int j = 0; j < cl_n; ++j) R->tables[x].cluster_slots[j] = cl[j];
      if (planned) R->tables[x].bound = cursor + x;  // holes: scan up to the cursor
      release_child(y);
      continue;  // size already known (exact) or on the device (planned)
    } else if (nd.type == 2) {  // forget
      const int y = nd.child0;
      rc = new_hash(x, entries(y));
      if (rc) return rc;
      cc::ForgetArgs a{R->L, desc(y), (int)P.nodes[y].bag.size(),
                       pos_in(P.nodes[y].bag, nd.vertex), desc(x), R->d_err};
      rc = timed(x, CC_K_FORGET, 1,
                 [&] { return cc::launch_forget(c->stream, c->dev, R->kw, block, a); });
      if (rc) return rc;
      release_child(y);
    } else {  // join
      int y = nd.child0, z = nd.child1;
      if (entries(y) > entries(z)) std::swap(y, z);  // chain the smaller child
      u64 icap = hash_cap(entries(y), lf);
      u64 bound_y = R->tables[y].hashed || planned ? R->tables[y].cap : R->sizes[y];
      void *index = A.alloc(icap * cc::index_slot_bytes(R->kw));
      u64 *next = arena_alloc<u64>(c, std::max<u64>(1, bound_y));
      if (!index || !next) {
        A.release(index);
        A.release(next);
        return CC_ENOMEM;
      }
      CUDA_OK(cudaMemsetAsync(index, 0, icap * cc::index_slot_bytes(R->kw), c->stream));
      u64 *pairs = pairs_dev + x;
      cc::JoinArgs a{};
      a.G = G;
      a.L = R->L;
      a.build = desc(y);
      a.probe = desc(z);
      a.b = (int)nd.bag.size();
      a.index = index;
      a.index_cap = icap;
      a.next = next;
      a.pairs = pairs;
      a.err = R->d_err;
      rc = timed(x, CC_K_JOIN_BUILD, 1,
                 [&] { return cc::launch_join(c->stream, c->dev, R->kw, 0, block, a); });
      u64 np = 0;
      if (!rc && !planned) {
        rc = timed(x, CC_K_JOIN_COUNT, 1,
                   [&] { return cc::launch_join(c->stream, c->dev, R->kw, 1, block, a); });
        if (!rc) rc = read_u64(c, pairs, &np);
        R->pairs[x] = np;
      }
      if (planned) np = room(plan->pairs[x]);
      if (!rc) rc = new_hash(x, np);
      if (!rc) {
        a.out = desc(x);
        rc = timed(x, CC_K_JOIN_WRITE, 1,
                   [&] { return cc::launch_join(c->stream, c->dev, R->kw, 2, block, a); });
      }
      A.release(index);
      A.release(next);
      if (rc) return rc;
      release_child(y);
      release_child(z);
    }
    if (!planned) {
      rc = read_u64(c, R->d_counters + x, &R->sizes[x]);
      if (rc) return rc;
    }
  }
  // root test (Section 3.1): per trial, nonempty root table and the sum of its counts
  cc::RootArgs ra{R->L, desc(N - 1), R->d_exists, R->d_count};
  rc = timed(N - 1, CC_K_ROOT, 1, [&] { return cc::launch_root(c->stream, c->dev, R->kw, ra); });
  return rc;
}

// reads the error word and, for planned runs, the sizes and capacity checks
int finish_run(Ctx *c, Run *R) {
  const int N = (int)R->sizes.size();
  int herr = 0;
  std::vector<u64> words(4 * (size_t)N);
  CUDA_OK(cudaMemcpyAsync(&herr, R->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_OK(cudaMemcpyAsync(words.data(), R->d_counters, words.size() * sizeof(u64),
                          cudaMemcpyDeviceToHost, c->stream));
  CUDA_OK(cudaStreamSynchronize(c->stream));
  for (int x = 0; x < N; ++x) {
    R->sizes[x] = words[x];
    if (words[2 * N + x]) R->pairs[x] = words[2 * N + x];
  }
  for (auto &t : R->timings)
    if (t.kind == CC_K_INTRO_COUNT || t.kind == CC_K_INTRO_WRITE || t.kind == CC_K_INTRO_FUSED ||
        t.kind == CC_K_INTRO_CHAIN)
      t.candidates = words[3 * (size_t)N + t.node];
  for (const auto &chk : R->checks) {
    const u64 v = words[chk.first - R->d_counters];
    if (v > chk.second) herr |= cc::kErrOverflow;
  }
  if (herr & cc::kErrTimeout) return CC_ETIMEOUT;
  if (herr) return CC_ECAPACITY;
  return CC_OK;
}

// ---- reconstruction driver (Section 4): pre-order steps over device state arrays -----------
int enumerate_run(Ctx *c, Run *R, uint64_t limit, int32_t *h_out, uint64_t *n_out,
                  uint64_t *n_total, bool sets, const cc::Coloring *colouring) {
  const Pattern &P = c->patterns.at(R->pattern);
  auto ci = c->colorings.find(R->coloring);
  if (!colouring && ci == c->colorings.end()) return CC_ENOTFOUND;
  const cc::Coloring &col = colouring ? *colouring : ci->second;
  const int N = (int)P.nodes.size();
  const int nF = P.nF;
  // node descriptors
  std::vector<cc::EnumNode> en(N);
  std::vector<int> vstar(N, 0), joins_below(N, 0);
  std::vector<uint32_t> vs(N, 0);
  for (int x = 0; x < N; ++x) {
    const NiceNode &nd = P.nodes[x];
    uint32_t m = 0;
    for (int u : nd.bag) m |= 1u << u;
    if (nd.child0 >= 0) m |= vs[nd.child0];
    if (nd.child1 >= 0) m |= vs[nd.child1];
    vs[x] = m;
    int jb = 0;
    if (nd.child0 >= 0) jb = std::max(jb, joins_below[nd.child0]);
    if (nd.child1 >= 0) jb = std::max(jb, joins_below[nd.child1]);
    joins_below[x] = jb + (nd.type == 3 ? 1 : 0);
    cc::EnumNode &e = en[x];
    e = cc::EnumNode{};
    e.type = nd.type;
    e.child0 = nd.child0;
    e.child1 = nd.child1;
    e.vertex = nd.vertex;
    e.b = (int)nd.bag.size();
    for (int s = 0; s < e.b; ++s) e.bag[s] = nd.bag[s];
    e.vstar = __builtin_popcount(m);
    if (nd.type == 1) {
      const NiceNode &ch = P.nodes[nd.child0];
      e.p = pos_in(nd.bag, nd.vertex);
      for (size_t s = 0; s < ch.bag.size(); ++s)
        if (P.adj[nd.vertex] >> ch.bag[s] & 1u) e.nb_slot[e.nnb++] = (int)s;
      e.degF = R->opts.degree_filter ? P.deg[nd.vertex] : 0;
    } else if (nd.type == 2) {
      for (int w : nd.bag)
        if (P.adj[nd.vertex] >> w & 1u) e.nb_slot[e.nnb++] = w;
    }
    const cc::NodeTable &t = R->tables[x];
    if (nd.type != 1 && !t.slots) return CC_EINVAL;  // tables were not kept
    e.slots = t.slots;
    e.cap = t.cap;
    e.count = R->sizes[x];
    e.hashed = t.hashed;
    e.sorted = !t.hashed && t.sort_n == (int)nd.bag.size() && nd.type != 0;
    if (e.sorted) {
      e.spec.L = R->L;
      e.spec.b = e.b;
      e.spec.nsl = t.sort_n;
      for (int s = 0; s < e.b; ++s) e.spec.order[s] = t.sort_slots[s];
      e.spec.full = 1;
      e.spec.bits = e.b * R->L.nb + R->L.tb + R->L.k;
      e.spec.hbits = t.sort_hbits;
      e.spec.hslots = t.sort_hslots;
    }
    if (nd.type != 0 && nd.type != 1 && !e.hashed && !e.sorted) return CC_EINVAL;
  }
  const int D = std::max(1, joins_below[N - 1]);
  const int RW = 3 + D + nF;
  // pre-order of the nice decomposition from the root
  std::vector<int> pre, stack{N - 1};
  while (!stack.empty()) {
    int x = stack.back();
    stack.pop_back();
    pre.push_back(x);
    if (P.nodes[x].child1 >= 0) stack.push_back(P.nodes[x].child1);
    if (P.nodes[x].child0 >= 0) stack.push_back(P.nodes[x].child0);
  }
  std::vector<void *> owned;
  auto cleanup = [&]() {
    for (void *p : owned) c->arena.release(p);
    owned.clear();
  };
  auto take = [&](size_t bytes) -> void * {
    void *p = c->arena.alloc(bytes);
    if (p) owned.push_back(p);
    return p;
  };
  auto drop = [&](void *p) {
    for (auto it = owned.begin(); it != owned.end(); ++it)
      if (*it == p) {
        owned.erase(it);
        break;
      }
    c->arena.release(p);
  };
  cc::EnumNode *d_nodes = (cc::EnumNode *)take(sizeof(cc::EnumNode) * N);
  u64 *scratch = (u64 *)take(sizeof(u64) * (cc::scan_scratch_words(c->dev) + 8));
  if (!d_nodes || !scratch) {
    cleanup();
    return CC_ENOMEM;
  }
  if (cudaMemcpyAsync(d_nodes, en.data(), sizeof(cc::EnumNode) * N, cudaMemcpyHostToDevice,
                      c->stream) != cudaSuccess) {
    cleanup();
    return CC_ECUDA;
  }
  cc::EnumArgs a{};
  a.G = cc::GraphDev{c->d_row_ptr, c->d_col, col.d_colors, c->n, c->d_deg8,
                     c->patterns.at(R->pattern).d_allow};
  a.L = R->L;
  a.nodes = d_nodes;
  a.nF = nF;
  a.R = RW;
  a.D = D;
  // root states
  u64 n_cur = R->sizes[N - 1];
  int *cur = (int *)take(std::max<u64>(1, n_cur) * RW * sizeof(int));
  if (!cur) {
    cleanup();
    return CC_ENOMEM;
  }
  a.out = cur;
  a.n_in = n_cur;
  u64 *d_n = scratch + cc::scan_scratch_words(c->dev);
  int rc = CC_OK;
  if (cudaMemsetAsync(d_n, 0, sizeof(u64), c->stream) != cudaSuccess) rc = CC_ECUDA;
  const cc::NodeTable &rt = R->tables[N - 1];
  const u64 rbound = rt.hashed ? rt.cap : R->sizes[N - 1];
  if (!rc && cc::launch_enum_init(c->stream, c->dev, R->kw, a, rt.slots, rbound, d_n)) rc = CC_ECUDA;
  c->launches++;
  for (size_t i = 0; i < pre.size() && !rc; ++i) {
    a.x = pre[i];
    a.in = cur;
    a.n_in = n_cur;
    unsigned *cnt = (unsigned *)take(std::max<u64>(1, n_cur) * sizeof(unsigned));
    u64 *off = (u64 *)take((n_cur + 1) * sizeof(u64));
    if (!cnt || !off) {
      rc = CC_ENOMEM;
      break;
    }
    a.cnt = cnt;
    if (cc::launch_enum_step(c->stream, c->dev, R->kw, 0, a) ||
        cc::launch_scan_u32(c->stream, c->dev, cnt, n_cur, off, scratch)) {
      rc = CC_ECUDA;
      break;
    }
    c->launches += 4;
    u64 n_next = 0;
    rc = read_u64(c, off + n_cur, &n_next);
    if (rc) break;
    int *next = (int *)take(std::max<u64>(1, n_next) * RW * sizeof(int));
    if (!next) {
      rc = CC_ENOMEM;
      break;
    }
    a.out = next;
    a.off = off;
    if (cc::launch_enum_step(c->stream, c->dev, R->kw, 1, a)) {
      rc = CC_ECUDA;
      break;
    }
    c->launches++;
    drop(cnt);
    drop(off);
    drop(cur);
    cur = next;
    n_cur = n_next;
  }
  // the union over trials in lexicographic order without repeats
  if (!rc) {
    int *rows = (int *)take(std::max<u64>(1, n_cur) * nF * sizeof(int));
    unsigned *perm = (unsigned *)take(std::max<u64>(1, n_cur) * sizeof(unsigned));
    unsigned *tmp = (unsigned *)take(std::max<u64>(1, n_cur) * sizeof(unsigned));
    u64 *hist = (u64 *)take((256 * 2 * (size_t)c->dev.sms + 512) * sizeof(u64));
    unsigned *flag = (unsigned *)take(std::max<u64>(1, n_cur) * sizeof(unsigned));
    u64 *off = (u64 *)take((n_cur + 1) * sizeof(u64));
    const u64 lim = std::min<u64>(limit, n_cur);
    int *out = (int *)take(std::max<u64>(1, lim) * nF * sizeof(int));
    if (!rows || !perm || !tmp || !hist || !flag || !off || !out) {
      rc = CC_ENOMEM;
    } else {
      unsigned *sorted = nullptr;
      if (cc::launch_rows_extract(c->stream, c->dev, cur, n_cur, RW, D, nF, rows, perm) ||
          (sets && cc::launch_rows_canon(c->stream, c->dev, rows, nF, n_cur)) ||
          cc::launch_rows_sort(c->stream, c->dev, rows, nF, R->L.nb, n_cur, perm, tmp, hist,
                               &sorted) ||
          cc::launch_rows_heads(c->stream, c->dev, rows, nF, sorted, n_cur, flag) ||
          cc::launch_scan_u32(c->stream, c->dev, flag, n_cur, off, scratch) ||
          cc::launch_rows_gather(c->stream, c->dev, rows, nF, sorted, n_cur, flag, off, lim, out))
        rc = CC_ECUDA;
      c->launches += 10;
      u64 distinct = 0;
      if (!rc) rc = read_u64(c, off + n_cur, &distinct);
      if (!rc) {
        const u64 m = std::min<u64>(limit, distinct);
        if (m && cudaMemcpyAsync(h_out, out, m * nF * sizeof(int), cudaMemcpyDeviceToHost,
                                 c->stream) != cudaSuccess)
          rc = CC_ECUDA;
        if (!rc && cudaStreamSynchronize(c->stream) != cudaSuccess) rc = CC_ECUDA;
        *n_out = m;
        *n_total = distinct;
      }
    }
  }
  cleanup();
  return rc;
}

// 64-bit fingerprint of a CSR graph (splitmix64 finaliser over its words); never 0.
long long csr_fingerprint(int32_t n, const int32_t *row_ptr, const int32_t *col) {
  auto mix = [](u64 z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
  };
  u64 h = mix((u64)n + 0x9e3779b97f4a7c15ull);
  for (int32_t i = 0; i <= n; ++i) h = mix(h ^ (u64)(uint32_t)row_ptr[i]);
  const int64_t m2 = row_ptr[n];
  int64_t e = 0;
  for (; e + 1 < m2; e += 2)
    h = mix(h ^ ((u64)(uint32_t)col[e] | (u64)(uint32_t)col[e + 1] << 32));
  if (e < m2) h = mix(h ^ (u64)(uint32_t)col[e]);
  return (long long)(h | 1);
}

// The distance bound of Section 3.2 (mapping expansion): for a vertex u introduced with no
// neighbour in the bag, the slot (in the child bag) of the bag vertex w nearest to u in F (the
// first in bag order among the nearest) and *dist = dist_F(w, u) >= 2; -1 if no bag vertex is in
// u's component (no bound: every host vertex is a candidate).
int near_slot(const Pattern &P, int u, const std::vector<int32_t> &child_bag, int *dist) {
  std::vector<int> d(P.nF, -1), q{u};
  d[u] = 0;
  for (size_t h = 0; h < q.size(); ++h)
    for (int b = 0; b < P.nF; ++b)
      if ((P.adj[q[h]] >> b & 1u) && d[b] < 0) {
        d[b] = d[q[h]] + 1;
        q.push_back(b);
      }
  int best = -1, slot = -1;
  for (size_t s = 0; s < child_bag.size(); ++s) {
    const int dd = d[child_bag[s]];
    if (dd >= 0 && (best < 0 || dd < best)) {
      best = dd;
      slot = (int)s;
    }
  }
  *dist = best;
  return best >= 2 ? slot : -1;
}

// Builds, once per graph and radius r, the CSR of every host vertex's ball of radius r (the
// vertices a breadth-first search from it reaches within r steps, each once, increasing) in the
// context's arena.  CC_ENOMEM if the balls hold more than 2^31 - 1 entries or do not fit.
int ensure_ball(Ctx *c, int r) {
  if (c->balls.count(r)) return CC_OK;
  const int32_t n = c->n;
  std::vector<int32_t> ptr(n + 1, 0), col, stamp(n, -1), depth(n, 0), one;
  for (int32_t s = 0; s < n; ++s) {
    one.clear();
    one.push_back(s);
    stamp[s] = s;
    depth[s] = 0;
    for (size_t h = 0; h < one.size(); ++h) {
      const int32_t x = one[h];
      if (depth[x] == r) continue;
      for (int32_t i = c->h_row_ptr[x]; i < c->h_row_ptr[x + 1]; ++i) {
        const int32_t b = c->h_col[i];
        if (stamp[b] != s) {
          stamp[b] = s;
          depth[b] = depth[x] + 1;
          one.push_back(b);
        }
      }
    }
    std::sort(one.begin(), one.end());
    if (col.size() + one.size() > (size_t)INT32_MAX) return CC_ENOMEM;
    col.insert(col.end(), one.begin(), one.end());
    ptr[s + 1] = (int32_t)col.size();
  }
  int32_t *dp = (int32_t *)c->arena.alloc(((size_t)n + 1) * sizeof(int32_t));
  int32_t *dc = (int32_t *)c->arena.alloc(std::max<size_t>(1, col.size()) * sizeof(int32_t));
  if (!dp || !dc) {
    c->arena.release(dp);
    c->arena.release(dc);
    return CC_ENOMEM;
  }
  if (cudaMemcpyAsync(dp, ptr.data(), ptr.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                      c->stream) != cudaSuccess ||
      (!col.empty() && cudaMemcpyAsync(dc, col.data(), col.size() * sizeof(int32_t),
                                       cudaMemcpyHostToDevice, c->stream) != cudaSuccess) ||
      cudaStreamSynchronize(c->stream) != cudaSuccess) {
    c->arena.release(dp);
    c->arena.release(dc);
    return CC_ECUDA;
  }
  c->balls[r] = {dp, dc};
  return CC_OK;
}

int init_run(Ctx *c, int32_t pid, const cc::Coloring &col, int32_t cid, const cc_run_opts *opts,
             std::unique_ptr<Run> &R, std::vector<long long> &key) {
  auto pi = c->patterns.find(pid);
  if (pi == c->patterns.end()) return CC_ENOTFOUND;
  const Pattern &P = pi->second;
  if (col.k < P.nF) return CC_EINVAL;
  if (P.allow_fp && P.allow_fp != c->graph_fp) return CC_EINVAL;  // masks of another graph
  if (opts && opts->distance_prune) {  // the distance bound needs the graph's balls
    for (const auto &nd : P.nodes)
      if (nd.type == 1) {
        const auto &cb = P.nodes[nd.child0].bag;
        bool nb = false;
        for (int32_t w : cb) nb = nb || (P.adj[nd.vertex] >> w & 1u);
        int dist = 0;
        if (!nb && near_slot(P, nd.vertex, cb, &dist) >= 0) {
          const int rc = ensure_ball(c, dist);
          if (rc) return rc;
        }
      }
  }
  R.reset(new Run());
  cc_default_opts(&R->opts);
  if (opts) R->opts = *opts;
  if (!(R->opts.load_factor > 0.f && R->opts.load_factor <= 0.9f)) R->opts.load_factor = 0.5f;
  if (R->opts.block != 128 && R->opts.block != 256 && R->opts.block != 512) R->opts.block = 256;
  R->pattern = pid;
  R->coloring = cid;
  R->trials = col.trials;
  int bmax = 0;
  for (auto &nd : P.nodes) bmax = std::max<int>(bmax, (int)nd.bag.size());
  int nb = std::max(1, bits_for((u64)std::max(0, c->n - 1)));
  int tb = col.trials > 1 ? bits_for((u64)(col.trials - 1)) : 0;
  R->L.k = col.k;
  R->L.nb = nb;
  R->L.tpos = col.k + bmax * nb;
  R->L.tb = tb;
  int width = R->L.tpos + tb;
  if (bmax > cc::kMaxBag || width > 128) return CC_EKEYWIDTH;
  R->kw = width <= 64 ? 1 : 2;
  const int N = (int)P.nodes.size();
  Arena &A = active_arena(c);
  R->home = &A == &c->arena ? nullptr : &A;
  R->d_counters = arena_alloc<u64>(c, 4 * (size_t)N);
  R->d_exists = arena_alloc<unsigned>(c, col.trials);
  R->d_count = arena_alloc<u64>(c, col.trials);
  R->d_err = arena_alloc<int>(c, 1);
  if (!R->d_counters || !R->d_exists || !R->d_count || !R->d_err) {
    A.release(R->d_counters);
    A.release(R->d_exists);
    A.release(R->d_count);
    A.release(R->d_err);
    R.reset();
    return CC_ENOMEM;
  }
  R->retained = R->opts.retain != 0;
  key = plan_key(c, pid, col.trials, col.k, R->opts);
  return CC_OK;
}

std::vector<long long> plan_key(const Ctx *c, int32_t pid, int32_t trials, int32_t k,
                                const cc_run_opts &o) {
  return {pid, c->graph_fp, trials, k, o.degree_filter, o.fuse, o.group, o.block,
          (long long)(o.load_factor * 1000), o.sort_sweep, o.distance_prune, o.part_bits,
          o.chain};
}

// init_run for colouring id cid of the context, which the run then holds a reference to.
int prepare_run(Ctx *c, int32_t pid, int32_t cid, const cc_run_opts *opts,
                std::unique_ptr<Run> &R, std::vector<long long> &key) {
  auto ci = c->colorings.find(cid);
  if (ci == c->colorings.end()) return CC_ENOTFOUND;
  const int rc = init_run(c, pid, ci->second, cid, opts, R, key);
  if (rc) {
    R.reset();
    return rc;
  }
  ci->second.refs++;  // released by free_run
  return CC_OK;
}

// Frees a run's tables and timings and zeroes its device words, ready for a (re)run.
int reset_run(Ctx *c, Run *R, int N) {
  Arena &H = R->home ? *R->home : c->arena;
  for (auto &t : R->tables)
    if (t.slots) H.release(t.slots);
  R->tables.clear();
  for (auto &t : R->timings) {
    cudaEventDestroy(t.start);
    cudaEventDestroy(t.stop);
  }
  R->timings.clear();
  CUDA_OK(cudaMemsetAsync(R->d_counters, 0, 4 * (size_t)N * sizeof(u64), c->stream));
  CUDA_OK(cudaMemsetAsync(R->d_exists, 0, R->trials * sizeof(unsigned), c->stream));
  CUDA_OK(cudaMemsetAsync(R->d_count, 0, R->trials * sizeof(u64), c->stream));
  return CC_OK;
}

// Folds a finished run's sizes into the plan of its key.
void update_plan(Ctx *c, const std::vector<long long> &key, const Run *R, size_t peak) {
  cc::Plan &plan = c->plans[key];
  const size_t N = R->sizes.size();
  plan.entries.resize(N, 0);
  plan.pairs.resize(N, 0);
  for (size_t x = 0; x < N; ++x) {
    plan.entries[x] = std::max(plan.entries[x], R->sizes[x]);
    plan.pairs[x] = std::max(plan.pairs[x], R->pairs[x]);
  }
  plan.peak_bytes = std::max(plan.peak_bytes, peak);
  plan.runs++;
}

// Runs the nodes on the context's stream: planned when a plan exists (repeated exactly if the
// plan proves too small), exact otherwise; then reads the results and updates the plan.
int run_direct(Ctx *c, Run *R, const cc::Coloring &col, const std::vector<long long> &key,
               bool exact_only) {
  const Pattern &P = c->patterns.at(R->pattern);
  const int N = (int)P.nodes.size();
  int rc = reset_run(c, R, N);
  if (rc) return rc;
  auto pl = c->plans.find(key);
  R->planned = !exact_only && pl != c->plans.end() && pl->second.runs > 0;
  R->graphed = false;
  Arena &A = active_arena(c);
  const size_t base = A.in_use();
  A.reset_high_water();
  if (R->planned) {
    rc = run_nodes(c, R, P, col, &pl->second);
    if (!rc) rc = finish_run(c, R);
    if (rc == CC_ECAPACITY || rc == CC_ENOMEM) {  // outgrew the plan: plan again, exactly
      R->planned = false;
      rc = reset_run(c, R, N);
      A.reset_high_water();
      if (!rc) rc = run_nodes(c, R, P, col, nullptr);
      if (!rc) rc = finish_run(c, R);
    }
  } else {
    rc = run_nodes(c, R, P, col, nullptr);
    if (!rc) rc = finish_run(c, R);
  }
  if (rc) return rc;
  update_plan(c, key, R, A.high_water() - base);
  return CC_OK;
}

void drop_graph(Ctx *c, const std::vector<long long> &gkey) {
  auto it = c->graphs.find(gkey);
  if (it == c->graphs.end()) return;
  cudaStreamSynchronize(c->stream);
  if (it->second->exec) cudaGraphExecDestroy(it->second->exec);
  for (auto &m : it->second->members) c->arena.release(m.block);
  c->graphs.erase(it);
}

void drop_all_graphs(Ctx *c) {
  while (!c->graphs.empty()) {
    std::vector<long long> k = c->graphs.begin()->first;
    drop_graph(c, k);
  }
}

// Graph replay is taken for a run that keeps no tables and times nothing, once it has a plan.
bool graph_eligible(Ctx *c, const Run *R, const std::vector<long long> &key) {
  if (!R->opts.use_graph || R->opts.retain || R->opts.profile) return false;
  auto pl = c->plans.find(key);
  return pl != c->plans.end() && pl->second.runs > 0;
}

// Captures the planned runs of Rs as one CUDA graph: member m runs on branch stream m (on the
// capture stream when there is one member) inside a sub-arena of its own, reading its colours
// from a buffer of the graph and writing the device words of a shadow run.  The sub-arenas stay
// reserved while the graph lives.
int capture_graph(Ctx *c, const std::vector<Run *> &Rs,
                  const std::vector<std::vector<long long>> &keys, std::unique_ptr<cc::GraphSet> &out) {
  const size_t M = Rs.size();
  std::unique_ptr<cc::GraphSet> gs(new cc::GraphSet());
  gs->members.resize(M);
  auto give_back = [&]() {
    for (auto &gm : gs->members) c->arena.release(gm.block);
  };
  while (M > 1 && c->branches.size() < M) {
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return CC_ECUDA;
    c->branches.push_back(s);
  }
  if (!c->capture && cudaStreamCreateWithFlags(&c->capture, cudaStreamNonBlocking) != cudaSuccess) {
    c->capture = nullptr;
    return CC_ECUDA;
  }
  std::vector<cudaEvent_t> ev(M + 1, nullptr);
  bool events_ok = true;
  for (auto &e : ev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      e = nullptr;
      events_ok = false;
    }
  auto drop_events = [&]() {
    for (auto &e : ev)
      if (e) cudaEventDestroy(e);
  };
  if (!events_ok) {
    drop_events();
    return CC_ECUDA;
  }
  // nothing runs while capturing; replays are launched on the context's stream
  cudaStream_t origin = c->stream, main = c->capture;
  if (cudaStreamBeginCapture(main, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    drop_events();
    return CC_ECUDA;
  }
  const u64 launches0 = c->launches;
  int rc = CC_OK;
  if (M > 1) {
    if (cudaEventRecord(ev[M], main) != cudaSuccess) rc = CC_ECUDA;
    for (size_t m = 0; m < M && !rc; ++m)
      if (cudaStreamWaitEvent(c->branches[m], ev[M], 0) != cudaSuccess) rc = CC_ECUDA;
  }
  for (size_t m = 0; m < M && !rc; ++m) {
    // member m takes the largest free range while it is captured and keeps what it touched
    const Run *R = Rs[m];
    const Pattern &P = c->patterns.at(R->pattern);
    const size_t N = P.nodes.size();
    cc::GraphMember &gm = gs->members[m];
    gm.bytes = c->arena.largest_free();
    gm.block = c->arena.alloc(gm.bytes);
    if (!gm.block) {
      rc = CC_ENOMEM;
      break;
    }
    gm.sub.init((char *)gm.block, gm.bytes);
    gm.colours = (uint8_t *)gm.sub.alloc((size_t)R->trials * (size_t)c->n);
    Run *S = new Run();
    gm.shadow.reset(S);
    S->pattern = R->pattern;
    S->opts = R->opts;
    S->L = R->L;
    S->kw = R->kw;
    S->trials = R->trials;
    S->home = &gm.sub;
    S->planned = true;
    S->d_counters = (u64 *)gm.sub.alloc(4 * N * sizeof(u64));
    S->d_exists = (unsigned *)gm.sub.alloc(R->trials * sizeof(unsigned));
    S->d_count = (u64 *)gm.sub.alloc(R->trials * sizeof(u64));
    S->d_err = (int *)gm.sub.alloc(sizeof(int));
    if (!gm.colours || !S->d_counters || !S->d_exists || !S->d_count || !S->d_err) {
      rc = CC_ENOMEM;
      break;
    }
    cc::Coloring view;
    view.trials = S->trials;
    view.k = S->L.k;
    view.d_colors = gm.colours;
    c->stream = M > 1 ? c->branches[m] : main;
    c->active = &gm.sub;
    rc = reset_run(c, S, (int)N);
    if (!rc) rc = run_nodes(c, S, P, view, &c->plans.at(keys[m]));
    c->stream = origin;
    c->active = nullptr;
    gm.bytes = gm.sub.top();
    c->arena.shrink(gm.block, gm.bytes);
  }
  // every forked branch joins the capture stream again, also after a failed step, so that the
  // capture ends cleanly
  if (M > 1)
    for (size_t m = 0; m < M; ++m)
      if (cudaEventRecord(ev[m], c->branches[m]) != cudaSuccess ||
          cudaStreamWaitEvent(main, ev[m], 0) != cudaSuccess)
        rc = rc ? rc : CC_ECUDA;
  cudaGraph_t g = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(main, &g);
  if (!rc && ee != cudaSuccess) rc = CC_ECUDA;
  if (!rc && cudaGraphInstantiate(&gs->exec, g, 0) != cudaSuccess) {
    gs->exec = nullptr;
    rc = CC_ECUDA;
  }
  if (g) cudaGraphDestroy(g);
  drop_events();
  gs->kernels = c->launches - launches0;
  c->launches = launches0;  // nothing ran yet: replays count them
  if (rc) {
    cudaGetLastError();  // clear the error a failed capture leaves behind
    give_back();
    return rc;
  }
  out = std::move(gs);
  return CC_OK;
}

// Replays a captured graph for runs Rs: copies each member's colours into the graph's buffer,
// launches the graph on the context's stream, reads each shadow run's words and hands the
// per-trial results and table sizes to the caller's run.
int replay_graph(Ctx *c, cc::GraphSet &gs, const std::vector<Run *> &Rs) {
  for (size_t m = 0; m < Rs.size(); ++m) {
    const cc::Coloring &col = c->colorings.at(Rs[m]->coloring);
    CUDA_OK(cudaMemcpyAsync(gs.members[m].colours, col.d_colors,
                            (size_t)col.trials * (size_t)c->n, cudaMemcpyDeviceToDevice,
                            c->stream));
  }
  CUDA_OK(cudaGraphLaunch(gs.exec, c->stream));
  c->launches += gs.kernels;
  int worst = CC_OK;
  for (size_t m = 0; m < Rs.size(); ++m) {
    Run *S = gs.members[m].shadow.get();
    Run *R = Rs[m];
    int rc = finish_run(c, S);
    if (rc) {
      worst = worst ? worst : rc;
      continue;
    }
    CUDA_OK(cudaMemcpyAsync(R->d_exists, S->d_exists, R->trials * sizeof(unsigned),
                            cudaMemcpyDeviceToDevice, c->stream));
    CUDA_OK(cudaMemcpyAsync(R->d_count, S->d_count, R->trials * sizeof(u64),
                            cudaMemcpyDeviceToDevice, c->stream));
    R->sizes = S->sizes;
    R->pairs = S->pairs;
    R->planned = true;
    R->graphed = true;
    R->tables.assign(S->sizes.size(), {});
  }
  return worst;
}

int run_sliced(Ctx *c, Run *R, const cc::Coloring &view, int32_t t0,
               const std::vector<long long> &ckey, int s0);

// Trials [t0, t0 + nt) of run R as a run of their own over their rows of the colouring; if
// they do not fit either, each half in turn, and a single trial in slices (run_sliced).
// Per-trial results do not depend on the other trials, so the chunk's exists flags and counts
// are R's, and table sizes add over chunks.
int run_chunk(Ctx *c, Run *R, const cc::Coloring &col, int32_t t0, int32_t nt) {
  cc::Coloring view;
  view.trials = nt;
  view.k = col.k;
  view.d_colors = col.d_colors + (size_t)t0 * (size_t)c->n;
  std::unique_ptr<Run> S;
  std::vector<long long> key;
  int rc = init_run(c, R->pattern, view, -1, &R->opts, S, key);
  if (rc) return rc;
  auto pl = c->plans.find(key);
  if (nt == 1 && pl != c->plans.end() && pl->second.slices > 0) {  // known not to fit whole
    free_run(c, S.get());
    return run_sliced(c, R, view, t0, key, pl->second.slices);
  }
  rc = run_direct(c, S.get(), view, key, false);
  if (!rc) {
    if (cudaMemcpyAsync(R->d_exists + t0, S->d_exists, nt * sizeof(unsigned),
                        cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(R->d_count + t0, S->d_count, nt * sizeof(u64), cudaMemcpyDeviceToDevice,
                        c->stream) != cudaSuccess)
      rc = CC_ECUDA;
    for (size_t x = 0; x < R->sizes.size() && !rc; ++x) {
      R->sizes[x] += S->sizes[x];
      R->pairs[x] = std::max(R->pairs[x], S->pairs[x]);
    }
  }
  free_run(c, S.get());
  if (rc == CC_ENOMEM && nt > 1) {
    const int32_t h = nt / 2;
    rc = run_chunk(c, R, col, t0, h);
    if (!rc) rc = run_chunk(c, R, col, t0 + h, nt - h);
  } else if (rc == CC_ENOMEM) {
    rc = run_sliced(c, R, view, t0, key, 2);
  }
  return rc;
}

// Trial t0 of run R (colouring `view` of that one trial, plan key ckey) split by the image of
// one pattern vertex, after the trial alone ran out of memory.  The colourful embeddings of F
// fall into disjoint classes by the host vertex that pattern vertex r (the vertex of the first
// leaf: every node on the way from that leaf to the root holds r in V*_x, so its tables shrink)
// is mapped to.  Slice i of s restricts r to the host vertices v = i (mod s) through
// allowed-mapping masks (Section 3.2, masking unprofitable mappings), so it counts exactly the
// classes of those vertices: the trial's count is the sum of the slices' counts (mod 2^64) and a
// copy exists iff a slice finds one.  s doubles, from s0 (or from the count remembered for the
// key), until every slice fits, up to 4096 slices.  Table sizes add over slices: exact for the
// nodes whose bag holds r, an upper bound for the others.
int run_sliced(Ctx *c, Run *R, const cc::Coloring &view, int32_t t0,
               const std::vector<long long> &ckey, int s0) {
  constexpr int32_t kSlicePattern = INT32_MIN + 1;  // the slices' masked copy of the pattern
  const int kMaxSlices = R->opts.max_slices > 0 ? R->opts.max_slices : 4096;
  const Pattern &P = c->patterns.at(R->pattern);
  const int r = P.nodes[0].vertex;
  Arena &A = active_arena(c);
  uint32_t *mask = arena_alloc<uint32_t>(c, std::max<size_t>(1, (size_t)c->n));
  if (!mask) return CC_ENOMEM;
  {
    Pattern Ps = P;
    Ps.d_allow = mask;
    Ps.allow_fp = c->graph_fp;
    c->patterns[kSlicePattern] = Ps;
  }
  const size_t N = R->sizes.size();
  int rc = CC_ENOMEM;
  for (int s = std::max(2, s0); s <= kMaxSlices && rc == CC_ENOMEM; s *= 2) {
    u64 count = 0;
    unsigned exists = 0;
    std::vector<u64> sizes(N, 0), pairs(N, 0);
    rc = CC_OK;
    for (int i = 0; i < s && !rc; ++i) {
      if (cc::launch_slice_mask(c->stream, c->dev, P.d_allow, c->n, 1u << r, s, i, mask)) {
        rc = CC_ECUDA;
        break;
      }
      c->launches++;
      std::unique_ptr<Run> S;
      std::vector<long long> key;
      rc = init_run(c, kSlicePattern, view, -1, &R->opts, S, key);
      if (rc) break;
      key = ckey;  // the slice's own plan: the trial's key with (slices, slice) appended
      key.push_back(-2);
      key.push_back(s);
      key.push_back(i);
      rc = run_direct(c, S.get(), view, key, false);
      u64 hc = 0;
      unsigned he = 0;
      if (!rc &&
          (cudaMemcpyAsync(&hc, S->d_count, sizeof(u64), cudaMemcpyDeviceToHost, c->stream) !=
               cudaSuccess ||
           cudaMemcpyAsync(&he, S->d_exists, sizeof(unsigned), cudaMemcpyDeviceToHost,
                           c->stream) != cudaSuccess ||
           cudaStreamSynchronize(c->stream) != cudaSuccess))
        rc = CC_ECUDA;
      if (!rc) {
        count += hc;
        exists |= he ? 1u : 0u;
        for (size_t x = 0; x < N; ++x) {
          sizes[x] += S->sizes[x];
          pairs[x] = std::max(pairs[x], S->pairs[x]);
        }
      }
      free_run(c, S.get());
    }
    if (!rc) {
      if (cudaMemcpyAsync(R->d_count + t0, &count, sizeof(u64), cudaMemcpyHostToDevice,
                          c->stream) != cudaSuccess ||
          cudaMemcpyAsync(R->d_exists + t0, &exists, sizeof(unsigned), cudaMemcpyHostToDevice,
                          c->stream) != cudaSuccess ||
          cudaStreamSynchronize(c->stream) != cudaSuccess)
        rc = CC_ECUDA;
      for (size_t x = 0; x < N && !rc; ++x) {
        R->sizes[x] += sizes[x];
        R->pairs[x] = std::max(R->pairs[x], pairs[x]);
      }
      if (!rc) c->plans[ckey].slices = s;
      R->sliced = std::max(R->sliced, s);
    }
  }
  c->patterns.erase(kSlicePattern);
  A.release(mask);
  return rc;
}

// Runs R's trials in chunks after all of them together ran out of memory (trial streaming),
// down to single trials in slices.
int run_split(Ctx *c, Run *R, const cc::Coloring &col) {
  const int N = (int)c->patterns.at(R->pattern).nodes.size();
  int rc = reset_run(c, R, N);
  if (rc) return rc;
  R->sizes.assign(N, 0);
  R->pairs.assign(N, 0);
  R->planned = R->graphed = false;
  R->streamed = true;
  if (R->trials == 1) {
    rc = run_chunk(c, R, col, 0, 1);
  } else {
    const int32_t h = R->trials / 2;
    rc = run_chunk(c, R, col, 0, h);
    if (!rc) rc = run_chunk(c, R, col, h, R->trials - h);
  }
  if (!rc && cudaStreamSynchronize(c->stream) != cudaSuccess) rc = CC_ECUDA;
  return rc;
}

// Runs R to completion on the context's stream without a graph: planned or exact, after giving
// back the memory of captured graphs if that is what it lacks, and in chunks of trials if all
// trials together do not fit.
int run_one(Ctx *c, Run *R, const std::vector<long long> &key) {
  const cc::Coloring &col = c->colorings.at(R->coloring);
  int rc = run_direct(c, R, col, key, false);
  if (rc == CC_ENOMEM && !c->graphs.empty()) {
    drop_all_graphs(c);
    rc = run_direct(c, R, col, key, false);
  }
  if (rc == CC_ENOMEM && !R->retained) rc = run_split(c, R, col);
  return rc;
}

// Runs Rs (prepared, with plan keys `keys`) from a captured graph, capturing it on first use.
// A member that outgrew the graph's capacities makes the graph stale: it is dropped and every
// member runs again directly (planned, then exactly if need be), which also updates the plans.
int run_graphed(Ctx *c, const std::vector<Run *> &Rs,
                const std::vector<std::vector<long long>> &keys) {
  std::vector<long long> gkey;
  for (size_t m = 0; m < Rs.size(); ++m) {
    gkey.insert(gkey.end(), keys[m].begin(), keys[m].end());
    gkey.push_back(-1);
  }
  auto it = c->graphs.find(gkey);
  if (it == c->graphs.end()) {
    std::unique_ptr<cc::GraphSet> gs;
    int rc = capture_graph(c, Rs, keys, gs);
    if (rc == CC_ENOMEM && !c->graphs.empty()) {  // older graphs hold the memory: drop them
      drop_all_graphs(c);
      rc = capture_graph(c, Rs, keys, gs);
    }
    if (rc == CC_ENOMEM && Rs.size() > 1) {  // too much at once: each half as a graph of its own
      const size_t h = Rs.size() / 2;
      const std::vector<Run *> R0(Rs.begin(), Rs.begin() + h), R1(Rs.begin() + h, Rs.end());
      const std::vector<std::vector<long long>> K0(keys.begin(), keys.begin() + h),
          K1(keys.begin() + h, keys.end());
      rc = run_graphed(c, R0, K0);
      return rc ? rc : run_graphed(c, R1, K1);
    }
    if (rc) {  // no graph: run them one by one
      for (size_t m = 0; m < Rs.size(); ++m) {
        rc = run_one(c, Rs[m], keys[m]);
        if (rc) return rc;
      }
      return CC_OK;
    }
    it = c->graphs.emplace(gkey, std::move(gs)).first;
  }
  int rc = replay_graph(c, *it->second, Rs);
  if (rc == CC_OK) {
    for (size_t m = 0; m < Rs.size(); ++m) update_plan(c, keys[m], Rs[m], 0);
    return CC_OK;
  }
  drop_graph(c, gkey);
  for (size_t m = 0; m < Rs.size(); ++m) {
    rc = run_one(c, Rs[m], keys[m]);
    if (rc) return rc;
  }
  return CC_OK;
}

// Prepares and runs the requests (pids[i], cids[i]) with one set of options: from a captured
// graph when eligible (one branch per request), else one after the other on the context's
// stream.  On failure every run made so far is freed.
int make_runs(Ctx *c, int32_t npat, const int32_t *pids, const int32_t *cids,
              const cc_run_opts *opts, std::vector<std::unique_ptr<Run>> &out) {
  std::vector<std::unique_ptr<Run>> runs(npat);
  std::vector<std::vector<long long>> keys(npat);
  std::vector<Run *> Rs(npat);
  auto fail = [&](int rc) {
    for (auto &R : runs)
      if (R && R->d_counters) free_run(c, R.get());
    return rc;
  };
  for (int32_t i = 0; i < npat; ++i) {
    int rc = prepare_run(c, pids[i], cids[i], opts, runs[i], keys[i]);
    if (rc) {
      runs[i].reset();  // prepare_run has freed what it took
      return fail(rc);
    }
    Rs[i] = runs[i].get();
  }
  // requests with a plan run from captured graphs (at most 64 branches a graph), the others
  // directly, which plans them for the next call
  int rc = CC_OK;
  std::vector<Run *> G;
  std::vector<std::vector<long long>> GK;
  auto flush = [&]() {
    if (!rc && !G.empty()) rc = run_graphed(c, G, GK);
    G.clear();
    GK.clear();
  };
  for (int32_t i = 0; i < npat && !rc; ++i) {
    if (graph_eligible(c, Rs[i], keys[i])) {
      G.push_back(Rs[i]);
      GK.push_back(keys[i]);
      if (G.size() == 64) flush();
    } else {
      rc = run_one(c, Rs[i], keys[i]);
    }
  }
  flush();
  if (rc) return fail(rc);
  out = std::move(runs);
  return CC_OK;
}

int nice_from_td(Pattern &P, const std::vector<std::vector<int>> &bags,
                 const std::vector<int> &parent) {
  int root = -1;
  if (!valid_td(P.adj, P.nF, bags, parent, root)) return CC_EINVAL;
  P.nodes.clear();
  build_nice(P.adj, bags, parent, root, P.nodes);
  P.width = 0;
  for (auto &nd : P.nodes) P.width = std::max<int>(P.width, (int)nd.bag.size() - 1);
  P.td_bags = bags;
  P.td_parent = parent;
  return CC_OK;
}

}  // namespace rt
}  // namespace cc

using namespace cc::rt;

// ------------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------------
extern "C" {

const char *cc_strerror(int code) {
  switch (code) {
    case CC_OK: return "ok";
    case CC_EINVAL: return "invalid argument";
    case CC_ENOMEM: return "device arena exhausted";
    case CC_ECAPACITY: return "table capacity exceeded";
    case CC_ETIMEOUT: return "bounded wait timed out";
    case CC_ECUDA: return "CUDA runtime error";
    case CC_ENOTFOUND: return "unknown id";
    case CC_EKEYWIDTH: return "trial, bag-mapping and colour bits exceed 128";
    case CC_EBUSY: return "the context is serving";
    case CC_ECANCELED: return "served query cancelled before it started";
    default: return "unknown error";
  }
}

void cc_default_opts(cc_run_opts *o) {
  o->degree_filter = 1;
  o->retain = 0;
  o->use_graph = 0;
  o->load_factor = 0.5f;
  o->block = 256;
  o->profile = 0;
  o->group = 1;
  o->fuse = 2;
  o->sort_sweep = 1;
  o->distance_prune = 0;
  o->max_slices = 0;
  o->part_bits = 0;
  o->chain = 1;
}

int cc_create(cc_ctx **out, int device, void *stream, void *d_arena, size_t arena_bytes) {
  if (!out || arena_bytes == 0) return CC_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) return CC_ECUDA;
  if (device < 0 || device >= ndev) return CC_EINVAL;
  CUDA_OK(cudaSetDevice(device));
  Ctx *c = new Ctx();
  c->device = device;
  c->stream = (cudaStream_t)stream;
  if (cudaDeviceGetAttribute(&c->dev.sms, cudaDevAttrMultiProcessorCount, device) !=
      cudaSuccess) {
    delete c;
    return CC_ECUDA;
  }
  c->dev.blocks_per_sm = 8;
  if (cc::prepare_sort_kernels() != 0 || cc::prepare_part_kernels() != 0) {
    delete c;
    return CC_ECUDA;
  }
  char *base = (char *)d_arena;
  if (!base) {
    if (cudaMalloc(&c->owned_arena, arena_bytes) != cudaSuccess) {
      delete c;
      return CC_ENOMEM;
    }
    base = c->owned_arena;
  }
  c->arena.init(base, arena_bytes);
  c->d_err = arena_alloc<int>(c, 1);
  c->d_ones = arena_alloc<u64>(c, 1);
  if (c->d_ones) cudaMemsetAsync(c->d_ones, 0xff, sizeof(u64), c->stream);
  if (!c->d_err || !c->d_ones || ensure_scratch(c, 4096)) {
    if (c->owned_arena) cudaFree(c->owned_arena);
    delete c;
    return CC_ENOMEM;
  }
  *out = (cc_ctx *)c;
  return CC_OK;
}

int cc_serve_stop(cc_ctx *ctx);

int cc_destroy(cc_ctx *ctx) {
  if (!ctx) return CC_EINVAL;
  Ctx *c = (Ctx *)ctx;
  cc_serve_stop(ctx);
  cc::serve_free(c);
  cudaStreamSynchronize(c->stream);
  drop_all_graphs(c);
  for (cudaStream_t s : c->branches) cudaStreamDestroy(s);
  if (c->capture) cudaStreamDestroy(c->capture);
  if (c->owned_arena) cudaFree(c->owned_arena);
  delete c;
  return CC_OK;
}

int cc_check_graph(int32_t n, const int32_t *h_row_ptr, const int32_t *h_col) {
  if (n < 0 || !h_row_ptr) return CC_EINVAL;
  if (h_row_ptr[0] != 0) return CC_EINVAL;
  for (int32_t v = 0; v < n; ++v)
    if (h_row_ptr[v + 1] < h_row_ptr[v]) return CC_EINVAL;
  const int64_t m2 = h_row_ptr[n];
  if (m2 > 0 && !h_col) return CC_EINVAL;
  for (int32_t v = 0; v < n; ++v)
    for (int32_t j = h_row_ptr[v]; j < h_row_ptr[v + 1]; ++j) {
      int32_t w = h_col[j];
      if (w < 0 || w >= n || w == v) return CC_EINVAL;
      if (j > h_row_ptr[v] && h_col[j - 1] >= w) return CC_EINVAL;  // sorted, no duplicates
      if (!std::binary_search(h_col + h_row_ptr[w], h_col + h_row_ptr[w + 1], v))
        return CC_EINVAL;  // symmetric
    }
  return CC_OK;
}

int cc_load_graph(cc_ctx *ctx, int32_t n, const int32_t *h_row_ptr, const int32_t *h_col) {
  Ctx *c = (Ctx *)ctx;
  if (c && cc::serve_active(c)) return CC_EBUSY;
  if (!c) return CC_EINVAL;
  int vr = cc_check_graph(n, h_row_ptr, h_col);
  if (vr) return vr;
  const int64_t m2 = h_row_ptr[n];
  // a new graph invalidates runs, colourings and captured graphs (they hold its addresses)
  drop_all_graphs(c);
  for (auto &r : c->runs) free_run(c, r.second.get());
  c->runs.clear();
  for (auto &col : c->colorings) c->arena.release(col.second.d_colors);
  c->colorings.clear();
  c->arena.release(c->d_row_ptr);
  c->arena.release(c->d_col);
  c->arena.release(c->d_deg8);
  for (auto &b : c->balls) {
    c->arena.release(b.second.first);
    c->arena.release(b.second.second);
  }
  c->balls.clear();
  c->d_row_ptr = arena_alloc<int32_t>(c, (size_t)n + 1);
  c->d_col = arena_alloc<int32_t>(c, std::max<int64_t>(1, m2));
  c->d_deg8 = arena_alloc<uint8_t>(c, std::max<int64_t>(1, n));
  if (!c->d_row_ptr || !c->d_col || !c->d_deg8) {
    c->n = -1;
    return CC_ENOMEM;
  }
  CUDA_OK(cudaMemcpyAsync(c->d_row_ptr, h_row_ptr, ((size_t)n + 1) * sizeof(int32_t),
                          cudaMemcpyHostToDevice, c->stream));
  if (m2 > 0)
    CUDA_OK(cudaMemcpyAsync(c->d_col, h_col, (size_t)m2 * sizeof(int32_t),
                            cudaMemcpyHostToDevice, c->stream));
  if (cc::launch_deg8(c->stream, c->dev, c->d_row_ptr, n, c->d_deg8)) return CC_ECUDA;
  c->launches++;
  const long long fp = csr_fingerprint(n, h_row_ptr, h_col);
  if (fp != c->graph_fp || c->plans.size() > 1024) c->plans.clear();
  c->graph_fp = fp;
  c->h_row_ptr.assign(h_row_ptr, h_row_ptr + n + 1);
  c->h_col.assign(h_col, h_col + m2);
  c->max_deg = 0;
  for (int32_t v = 0; v < n; ++v)
    c->max_deg = std::max<int64_t>(c->max_deg, (int64_t)h_row_ptr[v + 1] - h_row_ptr[v]);
  c->n = n;
  CUDA_OK(cudaStreamSynchronize(c->stream));
  return CC_OK;
}

static int make_pattern(int32_t nF, int32_t mF, const int32_t *h_edges, const cc_td *td,
                        Pattern &P) {
  if (nF < 1 || nF > 32 || mF < 0 || (mF > 0 && !h_edges)) return CC_EINVAL;
  P.nF = nF;
  P.adj.assign(nF, 0u);
  P.deg.assign(nF, 0);
  for (int32_t i = 0; i < mF; ++i) {
    int32_t a = h_edges[2 * i], b = h_edges[2 * i + 1];
    if (a < 0 || b < 0 || a >= nF || b >= nF || a == b) return CC_EINVAL;
    if (P.adj[a] >> b & 1u) continue;
    P.adj[a] |= 1u << b;
    P.adj[b] |= 1u << a;
    P.deg[a]++;
    P.deg[b]++;
  }
  std::vector<std::vector<int>> bags;
  std::vector<int> parent;
  if (td) {
    if (td->num_bags < 1 || !td->h_bag_ptr || !td->h_parent) return CC_EINVAL;
    bags.resize(td->num_bags);
    parent.assign(td->h_parent, td->h_parent + td->num_bags);
    for (int32_t i = 0; i < td->num_bags; ++i) {
      int32_t b0 = td->h_bag_ptr[i], b1 = td->h_bag_ptr[i + 1];
      if (b1 < b0) return CC_EINVAL;
      bags[i].assign(td->h_bag_vtx + b0, td->h_bag_vtx + b1);
    }
  } else {
    std::vector<int> order = nF <= 20 ? exact_order(P.adj, nF) : min_fill_order(P.adj, nF);
    td_from_order(P.adj, nF, order, bags, parent);
  }
  return nice_from_td(P, bags, parent);
}

int cc_nice_decomposition(int32_t nF, int32_t mF, const int32_t *h_edges, const cc_td *td,
                          int32_t max_nodes, int32_t *type, int32_t *child0, int32_t *child1,
                          int32_t *vertex, int32_t *bag_ptr, int32_t *bag_vtx,
                          int32_t *num_nodes, int32_t *width) {
  Pattern P;
  int rc = make_pattern(nF, mF, h_edges, td, P);
  if (rc) return rc;
  if (num_nodes) *num_nodes = (int32_t)P.nodes.size();
  if (width) *width = P.width;
  if ((int32_t)P.nodes.size() > max_nodes) return CC_ECAPACITY;
  int32_t off = 0;
  for (size_t i = 0; i < P.nodes.size(); ++i) {
    if (type) type[i] = P.nodes[i].type;
    if (child0) child0[i] = P.nodes[i].child0;
    if (child1) child1[i] = P.nodes[i].child1;
    if (vertex) vertex[i] = P.nodes[i].vertex;
    if (bag_ptr) bag_ptr[i] = off;
    for (int u : P.nodes[i].bag) {
      if (bag_vtx) bag_vtx[off] = u;
      ++off;
    }
  }
  if (bag_ptr) bag_ptr[P.nodes.size()] = off;
  return CC_OK;
}

int cc_load_pattern(cc_ctx *ctx, int32_t nF, int32_t mF, const int32_t *h_edges,
                    const cc_td *td, int32_t *pattern_id) {
  Ctx *c = (Ctx *)ctx;
  if (!c) return CC_EINVAL;
  std::lock_guard<std::mutex> lock(c->mu);
  if (!pattern_id) return CC_EINVAL;
  Pattern P;
  int rc = make_pattern(nF, mF, h_edges, td, P);
  if (rc) return rc;
  int32_t id = c->next_pattern++;
  c->patterns[id] = std::move(P);
  *pattern_id = id;
  return CC_OK;
}

int cc_load_pattern_masked(cc_ctx *ctx, int32_t nF, int32_t mF, const int32_t *h_edges,
                           const cc_td *td, const uint32_t *h_allow, int32_t *pattern_id) {
  Ctx *c = (Ctx *)ctx;
  if (!c) return CC_EINVAL;
  if (cc::serve_active(c)) return CC_EBUSY;
  if (!pattern_id || !h_allow || c->n < 0) return CC_EINVAL;
  Pattern P;
  int rc = make_pattern(nF, mF, h_edges, td, P);
  if (rc) return rc;
  P.d_allow = arena_alloc<uint32_t>(c, std::max<size_t>(1, (size_t)c->n));
  if (!P.d_allow) return CC_ENOMEM;
  if (c->n > 0 && (cudaMemcpyAsync(P.d_allow, h_allow, (size_t)c->n * sizeof(uint32_t),
                                   cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
                   cudaStreamSynchronize(c->stream) != cudaSuccess)) {
    c->arena.release(P.d_allow);
    return CC_ECUDA;
  }
  P.allow_fp = c->graph_fp;
  std::lock_guard<std::mutex> lock(c->mu);
  const int32_t id = c->next_pattern++;
  c->patterns[id] = std::move(P);
  *pattern_id = id;
  return CC_OK;
}

int cc_pattern_info(cc_ctx *ctx, int32_t pid, int32_t *num_nodes, int32_t *width) {
  Ctx *c = (Ctx *)ctx;
  if (!c) return CC_EINVAL;
  std::lock_guard<std::mutex> lock(c->mu);
  auto it = c->patterns.find(pid);
  if (it == c->patterns.end()) return CC_ENOTFOUND;
  if (num_nodes) *num_nodes = (int32_t)it->second.nodes.size();
  if (width) *width = it->second.width;
  return CC_OK;
}

int cc_pattern_nodes(cc_ctx *ctx, int32_t pid, int32_t *type, int32_t *child0, int32_t *child1,
                     int32_t *vertex, int32_t *bag_ptr, int32_t *bag_vtx) {
  Ctx *c = (Ctx *)ctx;
  if (!c) return CC_EINVAL;
  std::lock_guard<std::mutex> lock(c->mu);
  auto it = c->patterns.find(pid);
  if (it == c->patterns.end()) return CC_ENOTFOUND;
  int32_t off = 0;
  const auto &nodes = it->second.nodes;
  for (size_t i = 0; i < nodes.size(); ++i) {
    if (type) type[i] = nodes[i].type;
    if (child0) child0[i] = nodes[i].child0;
    if (child1) child1[i] = nodes[i].child1;
    if (vertex) vertex[i] = nodes[i].vertex;
    if (bag_ptr) bag_ptr[i] = off;
    for (int u : nodes[i].bag) {
      if (bag_vtx) bag_vtx[off] = u;
      ++off;
    }
  }
  if (bag_ptr) bag_ptr[nodes.size()] = off;
  return CC_OK;
}

int cc_color(cc_ctx *ctx, uint64_t seed, int32_t trials, int32_t k, int32_t *cid) {
  Ctx *c = (Ctx *)ctx;
  if (c && cc::serve_active(c)) return CC_EBUSY;
  if (!c || c->n < 0 || trials < 1 || k < 1 || k > 32 || !cid) return CC_EINVAL;
  cc::Coloring col;
  col.trials = trials;
  col.k = k;
  col.d_colors = arena_alloc<uint8_t>(c, std::max<size_t>(1, (size_t)trials * c->n));
  if (!col.d_colors) return CC_ENOMEM;
  if (check_launch(cc::launch_color(c->stream, c->dev, col.d_colors, c->n, trials, k, seed))) {
    c->arena.release(col.d_colors);
    return CC_ECUDA;
  }
  if ((size_t)trials * c->n > 0) c->launches++;
  int32_t id = c->next_coloring++;
  c->colorings[id] = col;
  *cid = id;
  return CC_OK;
}

int cc_set_colors(cc_ctx *ctx, const uint8_t *h_colors, int32_t trials, int32_t k,
                  int32_t *cid) {
  Ctx *c = (Ctx *)ctx;
  if (c && cc::serve_active(c)) return CC_EBUSY;
  if (!c || c->n < 0 || trials < 1 || k < 1 || k > 32 || !cid) return CC_EINVAL;
  size_t total = (size_t)trials * c->n;
  if (total && !h_colors) return CC_EINVAL;
  for (size_t i = 0; i < total; ++i)
    if (h_colors[i] >= k) return CC_EINVAL;
  cc::Coloring col;
  col.trials = trials;
  col.k = k;
  col.d_colors = arena_alloc<uint8_t>(c, std::max<size_t>(1, total));
  if (!col.d_colors) return CC_ENOMEM;
  if (total)
    CUDA_OK(cudaMemcpyAsync(col.d_colors, h_colors, total, cudaMemcpyHostToDevice, c->stream));
  CUDA_OK(cudaStreamSynchronize(c->stream));
  int32_t id = c->next_coloring++;
  c->colorings[id] = col;
  *cid = id;
  return CC_OK;
}

int cc_get_colors(cc_ctx *ctx, int32_t cid, uint8_t *h_out) {
  Ctx *c = (Ctx *)ctx;
  if (c && cc::serve_active(c)) return CC_EBUSY;
  if (!c || !h_out) return CC_EINVAL;
  auto it = c->colorings.find(cid);
  if (it == c->colorings.end()) return CC_ENOTFOUND;
  size_t total = (size_t)it->second.trials * c->n;
  if (total)
    CUDA_OK(cudaMemcpyAsync(h_out, it->second.d_colors, total, cudaMemcpyDeviceToHost,
                            c->stream));
  CUDA_OK(cudaStreamSynchronize(c->stream));
  return CC_OK;
}

int cc_release_colors(cc_ctx *ctx, int32_t cid) {
  Ctx *c = (Ctx *)ctx;
  if (c && cc::serve_active(c)) return CC_EBUSY;
  if (!c) return CC_EINVAL;
  auto it = c->colorings.find(cid);
  if (it == c->colorings.end()) return CC_ENOTFOUND;
  if (--it->second.refs == 0) {
    c->arena.release(it->second.d_colors);
    c->colorings.erase(it);
  }
  return CC_OK;
}

int cc_run_dp(cc_ctx *ctx, int32_t pid, int32_t cid, const cc_run_opts *opts, int32_t *run_id) {
  return cc_run_batch(ctx, 1, &pid, &cid, opts, run_id);
}

int cc_run_batch(cc_ctx *ctx, int32_t npat, const int32_t *pids, const int32_t *cids,
                 const cc_run_opts *opts, int32_t *run_ids) {
  Ctx *c = (Ctx *)ctx;
  if (c && cc::serve_active(c)) return CC_EBUSY;
  if (!c || c->n < 0 || npat < 0 || (npat && (!pids || !cids || !run_ids))) return CC_EINVAL;
  if (npat == 0) return CC_OK;
  std::vector<std::unique_ptr<Run>> runs;
  int rc = make_runs(c, npat, pids, cids, opts, runs);
  if (rc) return rc;
  for (int32_t i = 0; i < npat; ++i) {
    const int32_t id = c->next_run++;
    c->runs[id] = std::move(runs[i]);
    run_ids[i] = id;
  }
  return CC_OK;
}

static Run *find_run(Ctx *c, int32_t id) {
  auto it = c->runs.find(id);
  return it == c->runs.end() ? nullptr : it->second.get();
}

int cc_release(cc_ctx *ctx, int32_t run_id);

int cc_decide(cc_ctx *ctx, int32_t run_id, uint8_t *h_exists) {
  Ctx *c = (Ctx *)ctx;
  if (c && cc::serve_active(c)) return CC_EBUSY;
  if (c && cc::serve_active(c)) return CC_EBUSY;
  if (!c || !h_exists) return CC_EINVAL;
  Run *R = find_run(c, run_id);
  if (!R) return CC_ENOTFOUND;
  std::vector<unsigned> e(R->trials);
  CUDA_OK(cudaMemcpyAsync(e.data(), R->d_exists, R->trials * sizeof(unsigned),
                          cudaMemcpyDeviceToHost, c->stream));
  CUDA_OK(cudaStreamSynchronize(c->stream));
  for (int32_t t = 0; t < R->trials; ++t) h_exists[t] = e[t] ? 1 : 0;
  return CC_OK;
}

int cc_count(cc_ctx *ctx, int32_t run_id, uint64_t *h_counts) {
  Ctx *c = (Ctx *)ctx;
  if (c && cc::serve_active(c)) return CC_EBUSY;
  if (!c || !h_counts) return CC_EINVAL;
  Run *R = find_run(c, run_id);
  if (!R) return CC_ENOTFOUND;
  CUDA_OK(cudaMemcpyAsync(h_counts, R->d_count, R->trials * sizeof(u64),
                          cudaMemcpyDeviceToHost, c->stream));
  CUDA_OK(cudaStreamSynchronize(c->stream));
  return CC_OK;
}

int cc_table_stats(cc_ctx *ctx, int32_t run_id, uint64_t *h_sizes, uint64_t *h_total) {
  Ctx *c = (Ctx *)ctx;
  if (c && cc::serve_active(c)) return CC_EBUSY;
  if (!c) return CC_EINVAL;
  Run *R = find_run(c, run_id);
  if (!R) return CC_ENOTFOUND;
  u64 tot = 0;
  for (size_t i = 0; i < R->sizes.size(); ++i) {
    if (h_sizes) h_sizes[i] = R->sizes[i];
    tot += R->sizes[i];
  }
  if (h_total) *h_total = tot;
  return CC_OK;
}

int cc_table_dump(cc_ctx *ctx, int32_t run_id, int32_t node, uint64_t capacity, int32_t *h_trial,
                  int32_t *h_phi, uint32_t *h_mask, uint64_t *h_cnt, uint64_t *n_out) {
  Ctx *c = (Ctx *)ctx;
  if (c && cc::serve_active(c)) return CC_EBUSY;
  if (!c || !n_out) return CC_EINVAL;
  Run *R = find_run(c, run_id);
  if (!R) return CC_ENOTFOUND;
  if (node < 0 || node >= (int32_t)R->tables.size()) return CC_EINVAL;
  const cc::NodeTable &t = R->tables[node];
  if (!t.stored || !t.slots) return CC_EINVAL;
  const Pattern &P = c->patterns[R->pattern];
  const int b = (int)P.nodes[node].bag.size();
  const u64 m = R->sizes[node];
  *n_out = m;
  if (m > capacity) return CC_ECAPACITY;
  if (m == 0) return CC_OK;
  const size_t bytes = m * (sizeof(int32_t) * (1 + (size_t)b) + sizeof(uint32_t) + sizeof(u64)) + 64;
  char *buf = (char *)c->arena.alloc(bytes + 512);
  if (!buf) return CC_ENOMEM;
  u64 *d_n = (u64 *)buf;
  int32_t *d_trial = (int32_t *)(buf + 256);
  int32_t *d_phi = d_trial + m;
  uint32_t *d_mask = (uint32_t *)(d_phi + m * b);
  u64 *d_cnt = (u64 *)(((uintptr_t)(d_mask + m) + 7) & ~uintptr_t(7));
  int rc = CC_OK;
  // a planned table appended in chunks has holes: scan it up to its cursor
  TableDesc td{t.slots, t.cap, t.bound ? t.bound : R->d_counters + node, t.hashed};
  if (cudaMemsetAsync(d_n, 0, sizeof(u64), c->stream) != cudaSuccess ||
      cc::launch_unpack(c->stream, c->dev, R->kw, R->L, td, b, m, d_trial, d_phi, d_mask, d_cnt,
                        d_n) != 0) {
    rc = CC_ECUDA;
  } else {
    cudaMemcpyAsync(h_trial, d_trial, m * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
    if (b) cudaMemcpyAsync(h_phi, d_phi, m * b * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(h_mask, d_mask, m * sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(h_cnt, d_cnt, m * sizeof(u64), cudaMemcpyDeviceToHost, c->stream);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) rc = CC_ECUDA;
  }
  c->arena.release(buf);
  return rc;
}

int cc_enumerate(cc_ctx *ctx, int32_t run_id, uint64_t limit, int32_t *h_out, uint64_t *n_out,
                 uint64_t *n_total) {
  Ctx *c = (Ctx *)ctx;
  if (c && cc::serve_active(c)) return CC_EBUSY;
  if (!c || !n_out || !n_total || (limit && !h_out)) return CC_EINVAL;
  Run *R = find_run(c, run_id);
  if (!R) return CC_ENOTFOUND;
  if (!R->retained) return CC_EINVAL;
  return enumerate_run(c, R, limit, h_out, n_out, n_total, false);
}

int cc_enumerate_sets(cc_ctx *ctx, int32_t run_id, uint64_t limit, int32_t *h_out,
                      uint64_t *n_out, uint64_t *n_total) {
  Ctx *c = (Ctx *)ctx;
  if (c && cc::serve_active(c)) return CC_EBUSY;
  if (!c || !n_out || !n_total || (limit && !h_out)) return CC_EINVAL;
  Run *R = find_run(c, run_id);
  if (!R) return CC_ENOTFOUND;
  if (!R->retained) return CC_EINVAL;
  return enumerate_run(c, R, limit, h_out, n_out, n_total, true);
}

int cc_run_timings(cc_ctx *ctx, int32_t run_id, int32_t capacity, int32_t *h_node,
                   int32_t *h_kind, float *h_ms, uint64_t *h_cand, int32_t *n_out) {
  Ctx *c = (Ctx *)ctx;
  if (c && cc::serve_active(c)) return CC_EBUSY;
  if (!c || !n_out) return CC_EINVAL;
  Run *R = find_run(c, run_id);
  if (!R) return CC_ENOTFOUND;
  *n_out = (int32_t)R->timings.size();
  if ((int32_t)R->timings.size() > capacity) return CC_ECAPACITY;
  for (size_t i = 0; i < R->timings.size(); ++i) {
    const auto &t = R->timings[i];
    float ms = 0.f;
    CUDA_OK(cudaEventSynchronize(t.stop));
    CUDA_OK(cudaEventElapsedTime(&ms, t.start, t.stop));
    if (h_node) h_node[i] = t.node;
    if (h_kind) h_kind[i] = t.kind;
    if (h_ms) h_ms[i] = ms;
    if (h_cand) h_cand[i] = t.candidates;
  }
  return CC_OK;
}

int cc_probe_bounded_wait(cc_ctx *ctx, uint32_t polls) {
  Ctx *c = (Ctx *)ctx;
  if (!c || polls == 0) return CC_EINVAL;
  if (cc::serve_active(c)) return CC_EBUSY;
  u64 *flag = arena_alloc<u64>(c, 1);
  int *err = arena_alloc<int>(c, 1);
  int rc = CC_OK, herr = 0;
  if (!flag || !err) {
    rc = CC_ENOMEM;
  } else if (cudaMemsetAsync(flag, 0, sizeof(u64), c->stream) != cudaSuccess ||
             cudaMemsetAsync(err, 0, sizeof(int), c->stream) != cudaSuccess ||
             cc::launch_wait_probe(c->stream, flag, polls, err) != 0 ||
             cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, c->stream) !=
                 cudaSuccess ||
             cudaStreamSynchronize(c->stream) != cudaSuccess) {
    rc = CC_ECUDA;
  } else {
    c->launches++;
    if (herr & cc::kErrTimeout) rc = CC_ETIMEOUT;
  }
  c->arena.release(flag);
  c->arena.release(err);
  return rc;
}

int cc_run_mode(cc_ctx *ctx, int32_t run_id, int32_t *mode) {
  Ctx *c = (Ctx *)ctx;
  if (c && cc::serve_active(c)) return CC_EBUSY;
  if (!c || !mode) return CC_EINVAL;
  Run *R = find_run(c, run_id);
  if (!R) return CC_ENOTFOUND;
  *mode = R->sliced     ? CC_MODE_SLICED
          : R->streamed ? CC_MODE_STREAMED
          : R->graphed ? CC_MODE_GRAPH
          : R->planned ? CC_MODE_PLANNED
                       : CC_MODE_EXACT;
  return CC_OK;
}

int cc_context_stats(cc_ctx *ctx, uint64_t *launches, uint64_t *used, uint64_t *size) {
  Ctx *c = (Ctx *)ctx;
  if (!c) return CC_EINVAL;
  std::lock_guard<std::mutex> lock(c->mu);
  if (launches) *launches = c->launches;
  if (used) *used = c->arena.size() - c->arena.free_bytes();
  if (size) *size = c->arena.size();
  return CC_OK;
}

int cc_release(cc_ctx *ctx, int32_t run_id) {
  Ctx *c = (Ctx *)ctx;
  if (!c) return CC_EINVAL;
  auto it = c->runs.find(run_id);
  if (it == c->runs.end()) return CC_ENOTFOUND;
  free_run(c, it->second.get());
  c->runs.erase(it);
  return CC_OK;
}

}  // extern "C"
