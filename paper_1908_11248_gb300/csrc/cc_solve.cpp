// Repetition driver of the colour-coding library (cc_solve in include/cc.h).
//
// One colouring finds a given copy of F only if the copy is colourful, which for k = n_F colours
// happens with probability n_F!/n_F^n_F, close to (and above) e^-n_F (Section 2.1).  Repeating
// with independent colourings until e^n_F ln(1/eps) of them have run makes the chance of missing
// a present copy at most eps (the count of repetitions read as in that section, its printed
// formula being garbled); for enumeration the embeddings found under the different colourings are
// merged, each once (Section 4 reconstructs per colouring).  Colourings run in batches of trials
// (all trials of a batch in the same launches), trial t of the whole solve being coloured by
// Philox counter (v, t, 0, 0) under the solve's seed, so a solve equals a single run over all its
// trials.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <memory>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/cc.h"
#include "cc_internal.h"
#include "cc_runtime.h"

namespace cc {
namespace {

// merges sorted distinct rows b into sorted distinct rows a (row length w), keeping the first
// `limit` rows of the union
void merge_rows(std::vector<int32_t> &a, const std::vector<int32_t> &b, int w, uint64_t limit) {
  std::vector<int32_t> out;
  out.reserve(std::min<size_t>((a.size() + b.size()), (size_t)limit * w));
  size_t i = 0, j = 0;
  auto less = [&](const int32_t *x, const int32_t *y) {
    return std::lexicographical_compare(x, x + w, y, y + w);
  };
  while ((i < a.size() || j < b.size()) && out.size() < (size_t)limit * w) {
    const int32_t *x = i < a.size() ? &a[i] : nullptr, *y = j < b.size() ? &b[j] : nullptr;
    if (x && (!y || less(x, y))) {
      out.insert(out.end(), x, x + w);
      i += w;
    } else if (y && (!x || less(y, x))) {
      out.insert(out.end(), y, y + w);
      j += w;
    } else {  // equal rows: once
      out.insert(out.end(), x, x + w);
      i += w;
      j += w;
    }
  }
  a.swap(out);
}

}  // namespace
}  // namespace cc

using cc::Ctx;
using cc::Run;

extern "C" {

int32_t cc_solve_trials(int32_t n_F, double epsilon) {
  if (n_F < 1 || !(epsilon > 0.0 && epsilon < 1.0)) return -1;
  const double ell = std::ceil(std::exp((double)n_F) * std::log(1.0 / epsilon));
  return ell > 2147483647.0 ? 2147483647 : (int32_t)ell;
}

int cc_solve(cc_ctx *ctx, int32_t pattern_id, uint64_t seed, int32_t k, double epsilon,
             int32_t batch, int32_t max_trials, uint64_t limit, int32_t *h_out, uint64_t *n_out,
             uint8_t *found, int32_t *trials_run, double *estimate) {
  Ctx *c = (Ctx *)ctx;
  if (!c || !n_out || !found || !trials_run || batch < 1 || max_trials < 1 || (limit && !h_out))
    return CC_EINVAL;
  if (cc::serve_active(c)) return CC_EBUSY;
  if (c->n < 0 || k < 1 || k > 32) return CC_EINVAL;
  int32_t nF = 0;
  {
    std::lock_guard<std::mutex> lock(c->mu);
    auto pi = c->patterns.find(pattern_id);
    if (pi == c->patterns.end()) return CC_ENOTFOUND;
    nF = pi->second.nF;
  }
  if (k < nF) return CC_EINVAL;
  const int32_t ell = cc_solve_trials(nF, epsilon);
  if (ell < 0) return CC_EINVAL;
  const int32_t total = std::min(ell, max_trials);
  cc_run_opts opts;
  cc_default_opts(&opts);
  opts.retain = limit ? 1 : 0;
  std::vector<int32_t> rows, part;
  double sum = 0.0;
  bool any = false;
  int32_t done = 0;
  int rc = CC_OK;
  while (done < total && !rc) {
    const int32_t B = std::min(batch, total - done);
    // colouring of trials done .. done+B-1, held as a context colouring while the batch runs
    cc::Coloring col;
    col.trials = B;
    col.k = k;
    col.d_colors = cc::rt::arena_alloc<uint8_t>(c, std::max<size_t>(1, (size_t)B * c->n));
    if (!col.d_colors) return CC_ENOMEM;
    if (cc::launch_color(c->stream, c->dev, col.d_colors, c->n, B, k, seed, done) != 0) {
      c->arena.release(col.d_colors);
      return CC_ECUDA;
    }
    if ((size_t)B * c->n > 0) c->launches++;
    const int32_t cid = c->next_coloring++;
    c->colorings[cid] = col;
    std::vector<std::unique_ptr<Run>> runs;
    rc = cc::rt::make_runs(c, 1, &pattern_id, &cid, &opts, runs);
    if (!rc) {
      Run *R = runs[0].get();
      std::vector<uint64_t> cnt(B);
      std::vector<unsigned> ex(B);
      if (cudaMemcpyAsync(cnt.data(), R->d_count, B * sizeof(uint64_t), cudaMemcpyDeviceToHost,
                          c->stream) != cudaSuccess ||
          cudaMemcpyAsync(ex.data(), R->d_exists, B * sizeof(unsigned), cudaMemcpyDeviceToHost,
                          c->stream) != cudaSuccess ||
          cudaStreamSynchronize(c->stream) != cudaSuccess)
        rc = CC_ECUDA;
      for (int32_t t = 0; t < B && !rc; ++t) {
        sum += (double)cnt[t];
        any = any || ex[t] != 0;
      }
      if (!rc && limit) {
        part.assign((size_t)limit * nF, 0);
        uint64_t m = 0, tot = 0;
        rc = cc::rt::enumerate_run(c, R, limit, part.data(), &m, &tot, false);
        if (!rc) {
          part.resize((size_t)m * nF);
          cc::merge_rows(rows, part, nF, limit);
        }
      }
      cc::rt::free_run(c, R);
    }
    // the run held its own reference; this drops the solve's
    auto it = c->colorings.find(cid);
    if (it != c->colorings.end() && --it->second.refs == 0) {
      c->arena.release(it->second.d_colors);
      c->colorings.erase(it);
    }
    if (rc) return rc;
    done += B;
    if (!limit && any) break;  // decision: a colourful copy was found
  }
  *found = any ? 1 : 0;
  *trials_run = done;
  *n_out = rows.size() / (size_t)nF;
  if (limit && !rows.empty()) std::memcpy(h_out, rows.data(), rows.size() * sizeof(int32_t));
  if (estimate) {
    // a fixed injective map is colourful with probability (k)_{n_F} / k^{n_F}
    double p = 1.0;
    for (int32_t i = 0; i < nF; ++i) p *= (double)(k - i) / (double)k;
    *estimate = done ? sum / done / p : 0.0;
  }
  return CC_OK;
}

}  // extern "C"
