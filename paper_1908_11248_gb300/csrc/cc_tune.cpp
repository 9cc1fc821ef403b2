// Autotuner of the colour-coding library (cc_autotune in include/cc.h).
//
// The running time depends on the decomposition supplied, not on the treewidth of F (section
// on obtaining a nice tree decomposition); among decompositions of equal width the table sizes
// still depend on the order of introduces, forgets and joins, and the device time on how each
// node rule is carried out.  The tuner times the planned run of one (pattern, colouring) under candidate node schedules
// (the pattern's decomposition rooted at different bags, which changes the order in which the
// nice decomposition introduces, forgets and joins) and candidate execution options (forget
// scheme, threads per block, hash load factor, sort schedule, grouped and chained introduces), by coordinate
// descent from the starting options, and returns the fastest.  Every candidate's per-trial
// counts must equal the first's: the root results do not depend on any of these choices.
#include <algorithm>
#include <chrono>
#include <cstdint>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/cc.h"
#include "cc_internal.h"
#include "cc_runtime.h"

namespace cc {
namespace {

// The decomposition (bags, parent) re-rooted at bag r: parents follow the tree's edges away
// from r.
std::vector<int> reroot(const std::vector<int> &parent, int r) {
  const int nb = (int)parent.size();
  std::vector<std::vector<int>> nbr(nb);
  for (int i = 0; i < nb; ++i)
    if (parent[i] >= 0) {
      nbr[i].push_back(parent[i]);
      nbr[parent[i]].push_back(i);
    }
  std::vector<int> out(nb, -2), todo{r};
  out[r] = -1;
  for (size_t h = 0; h < todo.size(); ++h)
    for (int j : nbr[todo[h]])
      if (out[j] == -2) {
        out[j] = todo[h];
        todo.push_back(j);
      }
  return out;
}

bool same_nice(const Pattern &a, const Pattern &b) {
  if (a.nodes.size() != b.nodes.size()) return false;
  for (size_t i = 0; i < a.nodes.size(); ++i) {
    const NiceNode &x = a.nodes[i], &y = b.nodes[i];
    if (x.type != y.type || x.vertex != y.vertex || x.child0 != y.child0 ||
        x.child1 != y.child1 || x.bag != y.bag)
      return false;
  }
  return true;
}

}  // namespace
}  // namespace cc

using cc::Ctx;
using cc::Pattern;
using cc::Run;

extern "C" {

int cc_autotune(cc_ctx *ctx, int32_t pattern_id, int32_t coloring_id, const cc_run_opts *base,
                int32_t max_schedules, int32_t repeats, cc_run_opts *best_opts,
                int32_t *best_pattern_id, float *best_ms, int32_t *configs_tried) {
  Ctx *c = (Ctx *)ctx;
  if (!c || !best_opts || !best_pattern_id || max_schedules < 1 || repeats < 1) return CC_EINVAL;
  if (cc::serve_active(c)) return CC_EBUSY;
  if (c->n < 0) return CC_EINVAL;
  auto ci = c->colorings.find(coloring_id);
  if (ci == c->colorings.end()) return CC_ENOTFOUND;
  const int32_t T = ci->second.trials;

  // candidate schedules: the pattern as loaded, then its decomposition rooted at other bags
  std::vector<int32_t> schedules;
  {
    std::lock_guard<std::mutex> lock(c->mu);
    auto pi = c->patterns.find(pattern_id);
    if (pi == c->patterns.end()) return CC_ENOTFOUND;
    schedules.push_back(pattern_id);
    const Pattern base_p = pi->second;
    const int nb = (int)base_p.td_bags.size();
    for (int r = 0; r < nb && (int)schedules.size() < max_schedules; ++r) {
      Pattern Q;
      Q.nF = base_p.nF;
      Q.adj = base_p.adj;
      Q.deg = base_p.deg;
      Q.d_allow = base_p.d_allow;
      Q.allow_fp = base_p.allow_fp;
      if (cc::rt::nice_from_td(Q, base_p.td_bags, cc::reroot(base_p.td_parent, r))) continue;
      bool dup = false;
      for (int32_t s : schedules) dup = dup || cc::same_nice(c->patterns.at(s), Q);
      if (dup) continue;
      const int32_t id = c->next_pattern++;
      c->patterns[id] = std::move(Q);
      schedules.push_back(id);
    }
  }

  std::vector<uint64_t> want;
  std::vector<unsigned> want_e;
  int tried = 0;
  // the best wall time of `repeats` runs, after one run that makes the plan
  auto measure = [&](int32_t pid, const cc_run_opts &o, float &ms) -> int {
    double best = 1e30;
    for (int rep = 0; rep <= repeats; ++rep) {
      std::vector<std::unique_ptr<Run>> runs;
      const auto t0 = std::chrono::steady_clock::now();
      int rc = cc::rt::make_runs(c, 1, &pid, &coloring_id, &o, runs);
      const double dt =
          std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      if (rc) return rc;
      Run *R = runs[0].get();
      std::vector<uint64_t> cnt(T);
      std::vector<unsigned> ex(T);
      int e = 0;
      if (cudaMemcpyAsync(cnt.data(), R->d_count, T * sizeof(uint64_t), cudaMemcpyDeviceToHost,
                          c->stream) != cudaSuccess ||
          cudaMemcpyAsync(ex.data(), R->d_exists, T * sizeof(unsigned), cudaMemcpyDeviceToHost,
                          c->stream) != cudaSuccess ||
          cudaStreamSynchronize(c->stream) != cudaSuccess)
        e = CC_ECUDA;
      cc::rt::free_run(c, R);
      if (e) return e;
      if (want.empty()) {
        want = cnt;
        want_e = ex;
      } else if (cnt != want || ex != want_e) {
        return CC_ECUDA;  // a candidate disagrees at the root: an internal error
      }
      if (rep > 0) best = std::min(best, dt);
    }
    ms = (float)best;
    ++tried;
    return CC_OK;
  };

  cc_run_opts cur;
  cc_default_opts(&cur);
  if (base) cur = *base;
  cur.retain = 0;
  cur.profile = 0;
  cur.use_graph = 0;
  int32_t cur_pid = schedules[0];
  float cur_ms = 0.f;
  int rc = measure(cur_pid, cur, cur_ms);
  if (rc) return rc;
  for (size_t s = 1; s < schedules.size(); ++s) {
    float ms;
    rc = measure(schedules[s], cur, ms);
    if (rc) return rc;
    if (ms < cur_ms) {
      cur_ms = ms;
      cur_pid = schedules[s];
    }
  }
  // one option at a time, each over its values, keeping the best
  auto sweep = [&](auto set, std::initializer_list<float> values) -> int {
    for (float v : values) {
      cc_run_opts o = cur;
      set(o, v);
      if (std::memcmp(&o, &cur, sizeof o) == 0) continue;
      float ms;
      int r = measure(cur_pid, o, ms);
      if (r) return r;
      if (ms < cur_ms) {
        cur_ms = ms;
        cur = o;
      }
    }
    return CC_OK;
  };
  if (!rc) rc = sweep([](cc_run_opts &o, float v) { o.fuse = (int)v; }, {2, 1, 0});
  if (!rc) rc = sweep([](cc_run_opts &o, float v) { o.block = (int)v; }, {256, 128, 512});
  if (!rc) rc = sweep([](cc_run_opts &o, float v) { o.load_factor = v; }, {0.5f, 0.35f, 0.7f});
  if (!rc) rc = sweep([](cc_run_opts &o, float v) { o.sort_sweep = (int)v; }, {1, 0});
  if (!rc) rc = sweep([](cc_run_opts &o, float v) { o.group = (int)v; }, {1, 0});
  if (!rc) rc = sweep([](cc_run_opts &o, float v) { o.chain = (int)v; }, {1, 0});
  if (rc) return rc;
  *best_opts = cur;
  *best_pattern_id = cur_pid;
  if (best_ms) *best_ms = cur_ms;
  if (configs_tried) *configs_tried = tried;
  return CC_OK;
}

}  // extern "C"
