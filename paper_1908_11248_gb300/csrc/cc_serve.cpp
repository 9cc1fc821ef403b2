// Serving loop of the colour-coding library (cc_serve_* in include/cc.h).
//
// Many pattern queries over one resident graph (the setting of Section 5, where every query of
// a data set runs against the same host graph).  One server thread owns the context's device
// work while it runs.  Queries wait in a queue; the thread admits them while an execution slot
// (a CUDA stream) is free and the table memory their plan says they need fits in the budget, so
// queries that arrive while others run join them on the GPU (continuous batching).  Each query
// runs inside its own sub-range of the arena, reserved when it is admitted and trimmed to what
// its kernels touch, so that concurrent queries never share memory.
//
// A query whose (pattern, graph, trials, colours, options) key has no plan yet runs exactly,
// on its slot's stream while the other slots keep running; afterwards its plan gives later
// queries of the same key their capacities and their memory estimate.  A planned query whose
// tables outgrow the plan runs again exactly.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <stdexcept>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/cc.h"
#include "cc_internal.h"
#include "cc_runtime.h"

namespace cc {

using Clock = std::chrono::steady_clock;

struct ServeQuery {
  int64_t ticket = 0;
  int32_t pattern = 0, trials = 0, k = 0;
  uint64_t seed = 0;
  uint64_t limit = 0;  // > 0: also reconstruct the first `limit` embeddings (Section 4)
  bool exact = false;  // run exactly (the plan proved too small)
  Clock::time_point submitted;
};

struct ServeResult {
  bool done = false;
  int32_t status = CC_OK;
  std::vector<u64> counts;
  std::vector<uint8_t> exists;
  std::vector<int32_t> rows;  // n_rows * n_F embeddings, lexicographic
  u64 n_rows = 0;
  int64_t latency_ns = 0;
};

// An execution slot: a stream, the query running on it and the arena range it holds.
struct ServeSlot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  bool busy = false;
  ServeQuery q;
  void *block = nullptr;
  size_t bytes = 0;
  Arena sub;
  Coloring view;
  std::unique_ptr<Run> run;
  std::vector<long long> key;
};

struct Server {
  std::mutex mu;  // queue, results, flags and counters
  std::condition_variable cv;
  std::deque<ServeQuery> queue;
  std::map<int64_t, ServeResult> results;
  int64_t next_ticket = 1;
  int64_t cancel_upto = 0;  // queued queries with tickets up to this one end cancelled
  bool running = false, stopping = false;
  std::thread worker;
  size_t budget = 0;    // arena bytes the queries may hold at once
  size_t reserved = 0;  // arena bytes held by running queries
  std::vector<ServeSlot> slots;
  cc_run_opts opts{};
  // counters
  u64 submitted = 0, completed = 0, exact_runs = 0, reruns = 0, sliced = 0;
  int32_t inflight_max = 0;
  size_t reserved_max = 0;
};

namespace {

void wake(Server *S) { S->cv.notify_all(); }

void publish(Server *S, const ServeQuery &q, int32_t status, std::vector<u64> counts,
             std::vector<uint8_t> exists, std::vector<int32_t> rows = {}, u64 n_rows = 0) {
  std::lock_guard<std::mutex> g(S->mu);
  ServeResult &r = S->results[q.ticket];
  r.done = true;
  r.status = status;
  r.counts = std::move(counts);
  r.exists = std::move(exists);
  r.rows = std::move(rows);
  r.n_rows = n_rows;
  r.latency_ns =
      std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now() - q.submitted).count();
  S->completed++;
}

// Reads the per-trial results of a finished run from its slot's stream.
int read_results(Ctx *c, ServeSlot &sl, std::vector<u64> &counts, std::vector<uint8_t> &exists) {
  const int32_t T = sl.run->trials;
  std::vector<unsigned> e(T);
  counts.assign(T, 0);
  if (cudaMemcpyAsync(counts.data(), sl.run->d_count, T * sizeof(u64), cudaMemcpyDeviceToHost,
                      sl.stream) != cudaSuccess ||
      cudaMemcpyAsync(e.data(), sl.run->d_exists, T * sizeof(unsigned), cudaMemcpyDeviceToHost,
                      sl.stream) != cudaSuccess ||
      cudaStreamSynchronize(sl.stream) != cudaSuccess)
    return CC_ECUDA;
  exists.assign(T, 0);
  for (int32_t t = 0; t < T; ++t) exists[t] = e[t] ? 1 : 0;
  (void)c;
  return CC_OK;
}

// Gives the slot's arena range back and frees it for the next query.
void vacate(Server *S, Ctx *c, ServeSlot &sl) {
  sl.run.reset();  // its memory lies in the range released below
  c->arena.release(sl.block);
  {
    std::lock_guard<std::mutex> g(S->mu);
    S->reserved -= sl.bytes;
  }
  sl.block = nullptr;
  sl.bytes = 0;
  sl.busy = false;
}

// Reserves for slot sl the largest free arena range that the budget still allows.
bool reserve(Server *S, Ctx *c, ServeSlot &sl) {
  size_t avail;
  {
    std::lock_guard<std::mutex> g(S->mu);
    avail = S->budget > S->reserved ? S->budget - S->reserved : 0;
  }
  avail = std::min(avail, c->arena.largest_free()) & ~size_t(255);
  if (avail < ((size_t)1 << 20)) return false;
  sl.block = c->arena.alloc(avail);
  if (!sl.block) return false;
  sl.bytes = avail;
  sl.sub.init((char *)sl.block, avail);
  std::lock_guard<std::mutex> g(S->mu);
  S->reserved += avail;
  return true;
}

// Trims slot sl's range to the part its query's kernels touch.
void trim(Server *S, Ctx *c, ServeSlot &sl) {
  const size_t keep = std::max<size_t>(256, (sl.sub.top() + 255) & ~size_t(255));
  if (keep >= sl.bytes) return;
  c->arena.shrink(sl.block, keep);
  std::lock_guard<std::mutex> g(S->mu);
  S->reserved -= sl.bytes - keep;
  sl.bytes = keep;
}

enum Outcome { kIssued, kDone, kRetry };

// Starts query q on free slot sl.  Planned queries are only issued (kIssued: the slot's event
// marks their end); exact ones run to completion here (kDone).  kRetry: there is not enough
// memory while other queries run; the caller queues q again.
Outcome issue(Server *S, Ctx *c, ServeSlot &sl, const ServeQuery &q, bool alone) {
  std::lock_guard<std::mutex> g(c->mu);
  auto pi = c->patterns.find(q.pattern);
  if (pi == c->patterns.end()) {
    publish(S, q, CC_ENOTFOUND, {}, {});
    return kDone;
  }
  {  // a query of this key already ran out of the whole budget: refuse it without running
    auto pl = c->plans.find(rt::plan_key(c, q.pattern, q.trials, q.k, S->opts));
    if (pl != c->plans.end() && pl->second.refused >= S->budget) {
      publish(S, q, CC_ENOMEM, {}, {});
      return kDone;
    }
  }
  if (!reserve(S, c, sl)) {
    if (!alone) return kRetry;
    publish(S, q, CC_ENOMEM, {}, {});
    return kDone;
  }
  const Pattern &P = pi->second;
  cudaStream_t origin = c->stream;
  c->stream = sl.stream;
  c->active = &sl.sub;
  sl.q = q;
  int rc = CC_OK;
  Outcome out = kDone;
  bool published = false;
  try {  // a host allocation failure ends this query only, with CC_ENOMEM
  uint8_t *colours = (uint8_t *)sl.sub.alloc(std::max<size_t>(1, (size_t)q.trials * c->n));
  if (!colours) rc = CC_ENOMEM;
  else if (launch_color(sl.stream, c->dev, colours, c->n, q.trials, q.k, q.seed) != 0) rc = CC_ECUDA;
  else if ((size_t)q.trials * c->n > 0) c->launches++;
  sl.view = Coloring{};
  sl.view.trials = q.trials;
  sl.view.k = q.k;
  sl.view.d_colors = colours;
  cc_run_opts qo = S->opts;
  qo.retain = q.limit > 0 ? 1 : 0;  // a reconstruction needs every node's table
  if (!rc) rc = rt::init_run(c, q.pattern, sl.view, -1, &qo, sl.run, sl.key);
  if (!rc) {
    bool exact = true;
    auto pl = c->plans.find(sl.key);
    const bool split = pl != c->plans.end() && pl->second.slices > 0 && q.limit == 0;
    if (!q.exact && !split && q.limit == 0 && pl != c->plans.end() && pl->second.runs > 0) {
      exact = false;
      rc = rt::reset_run(c, sl.run.get(), (int)P.nodes.size());
      if (!rc) rc = rt::run_nodes(c, sl.run.get(), P, sl.view, &pl->second);
      if (!rc && cudaEventRecord(sl.done, sl.stream) != cudaSuccess) rc = CC_ECUDA;
      if (rc == CC_ENOMEM)  // the planned capacities need more than this range
        pl->second.peak_bytes = std::max(pl->second.peak_bytes, sl.bytes + 256);
      if (!rc) {
        sl.run->planned = true;
        sl.busy = true;
        out = kIssued;
      } else if (rc == CC_ENOMEM && alone) {
        // the whole budget is too small for the planned capacities: run exactly instead
        cudaStreamSynchronize(sl.stream);
        exact = true;
        rc = CC_OK;
      }
    }
    if (!rc && exact) {
      // run here, to completion: exactly (first query of its key, or one that outgrew its
      // plan), in slices when a single trial of its key needs more than the budget, or
      // planned with its tables kept when it asks for embeddings
      {
        std::lock_guard<std::mutex> g2(S->mu);
        if (q.limit == 0 || q.exact || pl == c->plans.end() || pl->second.runs == 0)
          S->exact_runs++;
      }
      const bool planned_enum = q.limit > 0 && !q.exact && pl != c->plans.end() &&
                                pl->second.runs > 0;
      if (split && alone) {
        rc = rt::run_split(c, sl.run.get(), sl.view);
      } else if (split) {
        rc = CC_ENOMEM;  // wait until it runs alone
      } else {
        rc = rt::run_direct(c, sl.run.get(), sl.view, sl.key, !planned_enum);
        if (rc == CC_ENOMEM && alone && q.limit == 0) {
          {
            std::lock_guard<std::mutex> g2(S->mu);
            S->sliced++;
          }
          rc = rt::run_split(c, sl.run.get(), sl.view);
        }
      }
      if (rc == CC_ENOMEM && alone) {
        size_t &r = c->plans[sl.key].refused;
        r = std::max(r, sl.bytes);
      }
      std::vector<u64> counts;
      std::vector<uint8_t> exists;
      std::vector<int32_t> rows;
      uint64_t n_rows = 0, n_total = 0;
      if (!rc) rc = read_results(c, sl, counts, exists);
      if (!rc && q.limit > 0) {
        const int32_t nF = c->patterns.at(q.pattern).nF;
        rows.assign((size_t)q.limit * nF, 0);
        rc = rt::enumerate_run(c, sl.run.get(), q.limit, rows.data(), &n_rows, &n_total, false,
                               &sl.view);
        rows.resize((size_t)n_rows * nF);
      }
      if (!rc) {
        publish(S, q, CC_OK, std::move(counts), std::move(exists), std::move(rows), n_rows);
        published = true;
      }
    }
  }
  } catch (const std::exception &) {
    cudaStreamSynchronize(sl.stream);
    out = kDone;
    rc = CC_ENOMEM;
    if (published) rc = CC_OK;
  }
  c->stream = origin;
  c->active = nullptr;
  if (out == kIssued) {
    trim(S, c, sl);
    std::lock_guard<std::mutex> g2(S->mu);
    S->reserved_max = std::max(S->reserved_max, S->reserved);
    return kIssued;
  }
  cudaStreamSynchronize(sl.stream);  // nothing of it may still run when its range is reused
  vacate(S, c, sl);
  if (published) return kDone;
  if (rc == CC_ENOMEM && !alone) return kRetry;
  publish(S, q, rc ? rc : CC_ECUDA, {}, {});
  return kDone;
}

// Finishes the query of busy slot sl once its event has completed (e: the event's status).
void complete(Server *S, Ctx *c, ServeSlot &sl, cudaError_t e) {
  std::lock_guard<std::mutex> g(c->mu);
  cudaStream_t origin = c->stream;
  c->stream = sl.stream;
  int rc = e == cudaSuccess ? rt::finish_run(c, sl.run.get()) : CC_ECUDA;
  std::vector<u64> counts;
  std::vector<uint8_t> exists;
  if (!rc) rc = read_results(c, sl, counts, exists);
  if (!rc) rt::update_plan(c, sl.key, sl.run.get(), sl.bytes);
  c->stream = origin;
  ServeQuery q = sl.q;
  vacate(S, c, sl);
  if (rc == CC_ECAPACITY) {  // the plan was too small for this colouring: run it exactly
    q.exact = true;
    std::lock_guard<std::mutex> g2(S->mu);
    S->reruns++;
    S->queue.push_front(q);
    return;
  }
  publish(S, q, rc, std::move(counts), std::move(exists));
}

// Memory a query is expected to hold: its plan's peak, or 0 when it has no plan yet (it then
// runs exactly, in whatever range is free).
size_t estimate(Server *S, Ctx *c, const ServeQuery &q) {
  if (q.exact) return 0;
  std::lock_guard<std::mutex> g(c->mu);
  auto pl = c->plans.find(rt::plan_key(c, q.pattern, q.trials, q.k, S->opts));
  return pl == c->plans.end() ? 0 : pl->second.peak_bytes;
}

void serve_loop(Server *S, Ctx *c) {
  cudaSetDevice(c->device);
  for (;;) {
    int inflight = 0;
    for (ServeSlot &sl : S->slots) {
      if (!sl.busy) continue;
      const cudaError_t e = cudaEventQuery(sl.done);
      if (e == cudaErrorNotReady) {
        ++inflight;
        continue;
      }
      complete(S, c, sl, e);
    }
    // admission: while a slot is free and the next query's memory fits
    for (ServeSlot &sl : S->slots) {
      if (sl.busy) continue;
      ServeQuery q;
      {
        std::lock_guard<std::mutex> g(S->mu);
        if (S->queue.empty()) break;
        q = S->queue.front();
      }
      bool cancelled;
      {
        std::lock_guard<std::mutex> g(S->mu);
        cancelled = q.ticket <= S->cancel_upto;
        if (cancelled) S->queue.pop_front();
      }
      if (cancelled) {  // put back by a retry after cc_serve_cancel dropped the queue
        publish(S, q, CC_ECANCELED, {}, {});
        continue;
      }
      const size_t need = estimate(S, c, q);
      {
        std::lock_guard<std::mutex> g(S->mu);
        if (inflight > 0 && S->reserved + need > S->budget) break;
        S->queue.pop_front();
      }
      const Outcome o = issue(S, c, sl, q, inflight == 0);
      if (o == kRetry) {
        std::lock_guard<std::mutex> g(S->mu);
        S->queue.push_front(q);
        break;
      }
      if (o == kIssued) {
        ++inflight;
        std::lock_guard<std::mutex> g(S->mu);
        S->inflight_max = std::max<int32_t>(S->inflight_max, inflight);
      }
    }
    std::unique_lock<std::mutex> lk(S->mu);
    if (inflight == 0 && S->queue.empty()) {
      if (S->stopping) break;
      S->cv.wait(lk, [&] { return !S->queue.empty() || S->stopping; });
    } else if (inflight > 0) {
      // poll the running queries; a submission wakes the loop at once
      S->cv.wait_for(lk, std::chrono::microseconds(20));
    }
  }
}

}  // namespace

void serve_free(Ctx *c) {
  if (!c->server) return;
  cc_serve_stop((cc_ctx *)c);
  delete c->server;
  c->server = nullptr;
}

bool serve_active(const Ctx *c) { return c->server && c->server->running; }

}  // namespace cc

using cc::Ctx;
using cc::Server;

extern "C" {

int cc_serve_start(cc_ctx *ctx, size_t mem_budget, int32_t max_inflight) {
  Ctx *c = (Ctx *)ctx;
  if (!c || c->n < 0 || max_inflight < 0 || max_inflight > 64) return CC_EINVAL;
  if (cc::serve_active(c)) return CC_EBUSY;
  if (!c->server) c->server = new Server();
  Server *S = c->server;
  const int nslots = max_inflight ? max_inflight : 8;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return CC_ECUDA;
  const size_t free_bytes = c->arena.free_bytes();
  S->budget = mem_budget ? std::min(mem_budget, free_bytes) : free_bytes / 2;
  S->reserved = 0;
  S->submitted = S->completed = S->exact_runs = S->reruns = S->sliced = 0;
  S->inflight_max = 0;
  S->reserved_max = 0;
  cc_default_opts(&S->opts);
  S->slots = std::vector<cc::ServeSlot>(nslots);
  for (auto &sl : S->slots)
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
      for (auto &t : S->slots) {
        if (t.stream) cudaStreamDestroy(t.stream);
        if (t.done) cudaEventDestroy(t.done);
      }
      S->slots.clear();
      return CC_ECUDA;
    }
  S->stopping = false;
  S->running = true;
  S->worker = std::thread(cc::serve_loop, S, c);
  return CC_OK;
}

int cc_serve_submit(cc_ctx *ctx, int32_t pattern_id, uint64_t seed, int32_t trials, int32_t k,
                    uint64_t limit, int64_t *ticket) {
  Ctx *c = (Ctx *)ctx;
  if (!c || !ticket || trials < 1 || k < 1 || k > 32) return CC_EINVAL;
  Server *S = c->server;
  if (!S) return CC_EINVAL;
  {
    std::lock_guard<std::mutex> g(S->mu);
    if (!S->running || S->stopping) return CC_EINVAL;
    cc::ServeQuery q;
    q.ticket = S->next_ticket++;
    q.pattern = pattern_id;
    q.trials = trials;
    q.k = k;
    q.seed = seed;
    q.limit = limit;
    q.submitted = cc::Clock::now();
    S->results[q.ticket] = cc::ServeResult{};
    S->queue.push_back(q);
    S->submitted++;
    *ticket = q.ticket;
  }
  cc::wake(S);
  return CC_OK;
}

int cc_serve_poll(cc_ctx *ctx, int64_t ticket, int32_t *done, int32_t *status,
                  uint64_t *h_counts, uint8_t *h_exists, int32_t *h_rows, uint64_t *n_rows,
                  int64_t *latency_ns) {
  Ctx *c = (Ctx *)ctx;
  if (!c || !done) return CC_EINVAL;
  Server *S = c->server;
  if (!S) return CC_ENOTFOUND;
  std::lock_guard<std::mutex> g(S->mu);
  auto it = S->results.find(ticket);
  if (it == S->results.end()) return CC_ENOTFOUND;
  const cc::ServeResult &r = it->second;
  *done = r.done ? 1 : 0;
  if (!r.done) return CC_OK;
  if (status) *status = r.status;
  if (latency_ns) *latency_ns = r.latency_ns;
  if (h_counts)
    for (size_t t = 0; t < r.counts.size(); ++t) h_counts[t] = r.counts[t];
  if (h_exists)
    for (size_t t = 0; t < r.exists.size(); ++t) h_exists[t] = r.exists[t];
  if (n_rows) *n_rows = r.n_rows;
  if (h_rows)
    for (size_t i = 0; i < r.rows.size(); ++i) h_rows[i] = r.rows[i];
  S->results.erase(it);
  return CC_OK;
}

int cc_serve_stats(cc_ctx *ctx, uint64_t *submitted, uint64_t *completed,
                   int32_t *inflight_max, uint64_t *reserved_max, uint64_t *exact_runs,
                   uint64_t *reruns, uint64_t *sliced) {
  Ctx *c = (Ctx *)ctx;
  if (!c) return CC_EINVAL;
  Server *S = c->server;
  if (!S) return CC_ENOTFOUND;
  std::lock_guard<std::mutex> g(S->mu);
  if (submitted) *submitted = S->submitted;
  if (completed) *completed = S->completed;
  if (inflight_max) *inflight_max = S->inflight_max;
  if (reserved_max) *reserved_max = S->reserved_max;
  if (exact_runs) *exact_runs = S->exact_runs;
  if (reruns) *reruns = S->reruns;
  if (sliced) *sliced = S->sliced;
  return CC_OK;
}

int cc_serve_cancel(cc_ctx *ctx, uint64_t *n_cancelled) {
  Ctx *c = (Ctx *)ctx;
  if (!c) return CC_EINVAL;
  Server *S = c->server;
  if (!S) return CC_EINVAL;
  std::deque<cc::ServeQuery> dropped;
  {
    std::lock_guard<std::mutex> g(S->mu);
    if (!S->running) return CC_EINVAL;
    S->cancel_upto = S->next_ticket - 1;
    dropped.swap(S->queue);
  }
  for (const auto &q : dropped) cc::publish(S, q, CC_ECANCELED, {}, {});
  if (n_cancelled) *n_cancelled = dropped.size();
  cc::wake(S);
  return CC_OK;
}

int cc_serve_stop(cc_ctx *ctx) {
  Ctx *c = (Ctx *)ctx;
  if (!c) return CC_EINVAL;
  Server *S = c->server;
  if (!S || !S->running) return CC_OK;
  {
    std::lock_guard<std::mutex> g(S->mu);
    S->stopping = true;
  }
  cc::wake(S);
  if (S->worker.joinable()) S->worker.join();
  for (auto &sl : S->slots) {
    cudaStreamDestroy(sl.stream);
    cudaEventDestroy(sl.done);
  }
  S->slots.clear();
  S->running = false;
  return CC_OK;
}

}  // extern "C"
