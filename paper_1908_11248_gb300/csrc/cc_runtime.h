// Host runtime state of the colour-coding library, shared by the C ABI (cc_host.cpp) and the
// serving loop (cc_serve.cpp): the device arena, patterns, colourings, runs, plans, captured
// graphs and the context that owns them.
#ifndef CC_RUNTIME_H
#define CC_RUNTIME_H

#include <cstdint>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/cc.h"
#include "cc_internal.h"

namespace cc {

typedef unsigned long long u64;

// ------------------------------------------------------------------------------------------
// device arena: first-fit over one device range, 256-byte aligned blocks
// ------------------------------------------------------------------------------------------
class Arena {
 public:
  void init(char *base, size_t size) {
    base_ = base;
    size_ = size;
    free_.clear();
    used_.clear();
    inuse_ = hw_ = top_ = 0;
    if (size) free_[0] = size;
  }
  void *alloc(size_t bytes) {
    if (bytes == 0) bytes = 1;
    bytes = (bytes + 255) & ~size_t(255);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      size_t off = it->first, sz = it->second;
      free_.erase(it);
      if (sz > bytes) free_[off + bytes] = sz - bytes;
      used_[off] = bytes;
      inuse_ += bytes;
      if (inuse_ > hw_) hw_ = inuse_;
      if (off + bytes > top_) top_ = off + bytes;
      return base_ + off;
    }
    return nullptr;
  }
  void release(void *p) {
    if (!p) return;
    size_t off = (char *)p - base_;
    auto u = used_.find(off);
    if (u == used_.end()) return;
    size_t sz = u->second;
    used_.erase(u);
    inuse_ -= sz;
    auto nx = free_.lower_bound(off);
    if (nx != free_.end() && nx->first == off + sz) {
      sz += nx->second;
      nx = free_.erase(nx);
    }
    if (nx != free_.begin()) {
      auto pv = std::prev(nx);
      if (pv->first + pv->second == off) {
        pv->second += sz;
        return;
      }
    }
    free_[off] = sz;
  }
  // Gives back the tail of block p beyond its first `bytes` bytes.
  void shrink(void *p, size_t bytes) {
    if (!p) return;
    bytes = (bytes + 255) & ~size_t(255);
    if (bytes == 0) bytes = 256;
    const size_t off = (char *)p - base_;
    auto u = used_.find(off);
    if (u == used_.end() || u->second <= bytes) return;
    const size_t tail = off + bytes, tail_sz = u->second - bytes;
    u->second = bytes;
    inuse_ -= tail_sz;
    used_[tail] = tail_sz;  // released at once, so that it merges with its free neighbours
    inuse_ += tail_sz;
    release(base_ + tail);
  }
  // end offset of the highest block handed out since init
  size_t top() const { return top_; }
  size_t free_bytes() const {
    size_t s = 0;
    for (auto &f : free_) s += f.second;
    return s;
  }
  size_t size() const { return size_; }
  size_t in_use() const { return inuse_; }
  size_t high_water() const { return hw_; }
  void reset_high_water() { hw_ = inuse_; }
  size_t largest_free() const {
    size_t s = 0;
    for (auto &f : free_) s = std::max(s, f.second);
    return s;
  }

 private:
  char *base_ = nullptr;
  size_t size_ = 0, inuse_ = 0, hw_ = 0, top_ = 0;
  std::map<size_t, size_t> free_, used_;
};


// ------------------------------------------------------------------------------------------
// context objects
// ------------------------------------------------------------------------------------------

struct NiceNode {
  int32_t type = 0;  // 0 leaf, 1 introduce, 2 forget, 3 join
  int32_t child0 = -1, child1 = -1, vertex = -1, parent = -1;
  std::vector<int32_t> bag;  // increasing
};

struct Pattern {
  int32_t nF = 0;
  std::vector<uint32_t> adj;  // adjacency bitmask per F-vertex
  std::vector<int32_t> deg;
  std::vector<NiceNode> nodes;  // post-order, root last
  int32_t width = 0;
  // the tree decomposition the nice one was built from (given, or computed)
  std::vector<std::vector<int>> td_bags;
  std::vector<int> td_parent;
  // allowed mappings (bit u of d_allow[v]: u may map to v), for the graph with fingerprint
  // allow_fp; null / 0: every mapping allowed
  uint32_t *d_allow = nullptr;
  long long allow_fp = 0;
};

struct Coloring {
  int32_t trials = 0, k = 0;
  uint8_t *d_colors = nullptr;
  int refs = 1;
};

struct NodeTable {
  void *slots = nullptr;
  u64 cap = 0;
  int hashed = 0;
  bool stored = false;
  // a dense table sorted with these bag slots most significant (sort_n == 0: no known order)
  int sort_n = 0;
  int sort_slots[kMaxBag] = {};
  // a bucketed order (sort_hbits > 0, see SortSpec): runs of equal images of the first m order
  // slots are contiguous only for m >= sort_min
  int sort_min = 0, sort_hbits = 0, sort_hslots = 0;
  // a dense table whose entries come in runs of equal images of these slots, except where an
  // append chunk or a kernel's tile ends (written in the order of a child sorted or clustered
  // by them); cluster_n == 0: no known clustering
  int cluster_n = 0, cluster_min = 0;
  int cluster_slots[kMaxBag] = {};
  // scan bound of a dense table written in chunks (holes up to it); null: the entry counter
  unsigned long long *bound = nullptr;
};

// Capacities learned from exact runs of one (pattern, graph, trials, colours, options): the
// largest table sizes and join pair counts seen, per node.
struct Plan {
  std::vector<u64> entries, pairs;
  size_t peak_bytes = 0;  // largest arena use of a run beyond what it started with
  int runs = 0;
  size_t refused = 0;  // a served run of this key ran out of memory in a range this large
  int slices = 0;      // a single trial of this key fitted once split into this many slices
};

struct Timing {
  int32_t node, kind;
  cudaEvent_t start, stop;
  u64 candidates;
};

struct Run {
  int32_t pattern = -1, coloring = -1;
  std::vector<Timing> timings;
  cc_run_opts opts{};
  KeyLayout L{};
  int kw = 1;
  int32_t trials = 0;
  std::vector<NodeTable> tables;
  // per node, four words each: entries, chunk cursor, join pairs, candidates examined
  u64 *d_counters = nullptr;
  unsigned *d_exists = nullptr;
  u64 *d_count = nullptr;
  std::vector<u64> sizes, pairs;
  std::vector<std::pair<const u64 *, u64>> checks;  // planned runs: device word <= capacity
  bool retained = false;
  bool planned = false;
  bool graphed = false;
  bool streamed = false;  // its trials ran in chunks (all at once did not fit)
  int sliced = 0;         // most slices one of its trials was split into (0: none)
  u64 *d_blk = nullptr;  // per-run scratch: block counts and bases, pair counters
  int *d_err = nullptr;  // per-run device error word
  Arena *home = nullptr;  // the arena its memory came from (null: the context's)
};

// A captured CUDA graph of planned runs (one member per run; members are parallel branches).
// Each member owns a sub-arena reserved from the context arena for the graph's lifetime, the
// colouring buffer the graph reads, and a shadow run whose device words the graph writes.
struct GraphMember {
  void *block = nullptr;
  size_t bytes = 0;
  Arena sub;
  uint8_t *colours = nullptr;
  std::unique_ptr<Run> shadow;
};

struct GraphSet {
  cudaGraphExec_t exec = nullptr;
  std::vector<GraphMember> members;
  u64 kernels = 0;  // kernel launches per replay
};

struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  DevInfo dev;
  Arena arena;
  Arena *active = nullptr;  // where run allocations go: the arena, or a captured graph's own
  char *owned_arena = nullptr;
  // graph
  int32_t n = -1;
  int32_t *d_row_ptr = nullptr, *d_col = nullptr;
  uint8_t *d_deg8 = nullptr;  // min(degree, 255) per vertex
  int64_t max_deg = 0;        // largest vertex degree of the loaded graph
  std::vector<int32_t> h_row_ptr, h_col;
  // per radius r, per vertex the vertices within distance r (CSR row pointers and columns,
  // built on first use by the distance bound)
  std::map<int, std::pair<int32_t *, int32_t *>> balls;
  int *d_err = nullptr;
  u64 *d_ones = nullptr;     // a device word holding ~0 (an unbounded scan limit)
  // content fingerprint of the loaded graph: plans stay valid while the graph's content is the
  // same, so reloading an identical graph keeps them
  long long graph_fp = 0;
  std::map<std::vector<long long>, Plan> plans;
  std::map<std::vector<long long>, std::unique_ptr<GraphSet>> graphs;
  std::vector<cudaStream_t> branches;  // streams of captured batch branches
  cudaStream_t capture = nullptr;      // where graphs are captured (the context's stream may be
                                       // the legacy default stream, which cannot be captured)
  u64 *d_scratch = nullptr;  // small per-call scratch (block counts, pair counter)
  size_t scratch_words = 0;
  std::map<int32_t, Pattern> patterns;
  std::map<int32_t, Coloring> colorings;
  std::map<int32_t, std::unique_ptr<Run>> runs;
  int32_t next_pattern = 1, next_coloring = 1, next_run = 1;
  u64 launches = 0;
  // serving: while a server runs it alone issues device work; mu orders its use of the pattern
  // table against cc_load_pattern and the other pattern calls
  struct Server *server = nullptr;
  std::mutex mu;
};

// Frees the serving state of a context; true while a server runs on it (cc_serve.cpp).
void serve_free(Ctx *c);
bool serve_active(const Ctx *c);

// ------------------------------------------------------------------------------------------
// run machinery (cc_host.cpp), used by the C ABI and by the serving loop
// ------------------------------------------------------------------------------------------
namespace rt {

// where run allocations go: the context's active sub-arena, else its arena
Arena &active_arena(Ctx *c);

template <typename T>
T *arena_alloc(Ctx *c, size_t count) {
  return (T *)active_arena(c).alloc(count * sizeof(T));
}

// Sets up run R of pattern pid under colouring col (id cid, or -1 for a colouring the caller
// owns): options, key layout, device words (from the active arena) and the plan key.
int init_run(Ctx *c, int32_t pid, const Coloring &col, int32_t cid, const cc_run_opts *opts,
             std::unique_ptr<Run> &R, std::vector<long long> &key);
// The key under which runs share a plan: pattern, graph content, trials, colours and the
// options that shape the tables (normalised as init_run leaves them).
std::vector<long long> plan_key(const Ctx *c, int32_t pid, int32_t trials, int32_t k,
                                const cc_run_opts &o);
// Frees a run's tables, device words and timings; drops its colouring reference.
void free_run(Ctx *c, Run *r);
// Frees a run's tables and timings and zeroes its device words, ready for a (re)run.
int reset_run(Ctx *c, Run *R, int N);
// Issues every node of the run on the context's stream (planned when plan is non-null).
int run_nodes(Ctx *c, Run *R, const Pattern &P, const Coloring &col, const Plan *plan);
// Reads the run's error word, sizes and capacity checks (waits for the context's stream).
int finish_run(Ctx *c, Run *R);
// Folds a finished run's sizes (and its arena peak) into the plan of its key.
void update_plan(Ctx *c, const std::vector<long long> &key, const Run *R, size_t peak);
// Runs R to completion on the context's stream: planned if a plan exists and exact_only is
// false (exactly again if it proves too small), else exactly; updates the plan.
int run_direct(Ctx *c, Run *R, const Coloring &col, const std::vector<long long> &key,
               bool exact_only);
// Runs R (tables not kept) after it ran out of memory: its trials in halves, and a single trial
// split by the image of one pattern vertex into slices that fit (results exact; table sizes add
// over chunks and slices).
int run_split(Ctx *c, Run *R, const Coloring &col);
// Destroys every captured graph and gives back its memory.
void drop_all_graphs(Ctx *c);
// Checks the tree decomposition (bags, parent) of P's graph (P.nF, P.adj set) and builds P's
// nice decomposition from it.  CC_EINVAL if it is not a tree decomposition of F.
int nice_from_td(Pattern &P, const std::vector<std::vector<int>> &bags,
                 const std::vector<int> &parent);
// The `limit` lexicographically smallest distinct embeddings over a retained run's trials
// (Section 4), into h_out[n_out][n_F]; *n_total the number of distinct ones.  With `sets`, each
// embedding is replaced by its vertex set in increasing order before the distinct ones are kept.
// `colouring`: the run's colouring when it is not one of the context's (a served query's own).
int enumerate_run(Ctx *c, Run *R, uint64_t limit, int32_t *h_out, uint64_t *n_out,
                  uint64_t *n_total, bool sets, const Coloring *colouring = nullptr);
// Runs (pattern, colouring) requests with one set of options (cc_run_batch without ids).
int make_runs(Ctx *c, int32_t npat, const int32_t *pids, const int32_t *cids,
              const cc_run_opts *opts, std::vector<std::unique_ptr<Run>> &out);

}  // namespace rt
}  // namespace cc

#endif  // CC_RUNTIME_H

