// cc_count_noalloc: a colour-coding count that allocates no device memory.
//
// Some callers cannot call cudaMalloc (or anything that does): processes whose device memory is
// owned by another allocator that must not be bypassed (a framework's caching pool, a fixed
// partition of the GPU handed to a plug-in), and library code loaded into such processes that
// has no allocator of its own to ask.  For them this entry point runs the whole count (graph
// upload, colouring, dynamic programme, root test) inside one fixed-size device array that is
// part of the library image itself, so the only memory it touches is that array and the
// caller's host buffers.
//
// It copies the host inputs in and the results out, and waits for the caller's stream between
// steps, so it returns only when its work is done.  Called on a stream that is being captured
// into a CUDA graph it does nothing and returns CC_EINVAL.
//
// The array is a file-scope __device__ variable: every GPU that loads this library holds
// CC_NOALLOC_BYTES of it until the process exits.  In host code its name is only a stand-in, so
// its device address is looked up once per device (cudaGetSymbolAddress, with that device
// current) on the first call made on that device.  All calls on a device share the array and it
// keeps the previous call's contents; everything the count needs zeroed is cleared by the call
// itself.  Two calls whose work overlaps on the same GPU (different streams or threads) race on
// the array and must be serialised by the caller.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/cc.h"

static __device__ __align__(256) unsigned char cc_noalloc_scratch[CC_NOALLOC_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch[kMaxDevices] = {};  // device address of the array, per device
}  // namespace

extern "C" int cc_count_noalloc(int device, void *cuda_stream, int32_t n,
                                const int32_t *h_row_ptr, const int32_t *h_col, int32_t n_F,
                                int32_t m_F, const int32_t *h_edges, const cc_td *td,
                                uint64_t seed, int32_t trials, int32_t k, uint64_t *h_counts,
                                uint8_t *h_exists) {
  if (device < 0 || device >= kMaxDevices || n < 0 || !h_row_ptr || trials < 1 || !h_counts ||
      !h_exists)
    return CC_EINVAL;
  // a stream being captured must see no copy or wait from this call
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing((cudaStream_t)cuda_stream, &cap) != cudaSuccess) return CC_ECUDA;
  if (cap != cudaStreamCaptureStatusNone) return CC_EINVAL;
  // what a context holds before any table: the CSR (int32 row pointers and columns), one degree
  // byte and one colour byte per vertex and trial, and its small words and scratch (under 1 MiB)
  const unsigned long long m2 = (unsigned long long)h_row_ptr[n];
  const unsigned long long fixed = 4ull * ((unsigned long long)n + 1 + m2) +
                                   (unsigned long long)n * (1ull + (unsigned long long)trials) +
                                   (1ull << 20);
  if (fixed > CC_NOALLOC_BYTES) return CC_ENOMEM;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) return CC_ECUDA;
  if (cudaSetDevice(device) != cudaSuccess) return CC_EINVAL;
  void *base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch[device]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, cc_noalloc_scratch) != cudaSuccess) {
        cudaSetDevice(prev);
        return CC_ECUDA;
      }
      g_scratch[device] = p;
    }
    base = g_scratch[device];
  }
  cc_ctx *ctx = nullptr;
  int rc = cc_create(&ctx, device, cuda_stream, base, CC_NOALLOC_BYTES);
  if (rc == CC_OK) {
    int32_t pid = 0, cid = 0, run = 0;
    cc_run_opts opts;
    cc_default_opts(&opts);
    rc = cc_load_graph(ctx, n, h_row_ptr, h_col);
    if (rc == CC_OK) rc = cc_load_pattern(ctx, n_F, m_F, h_edges, td, &pid);
    if (rc == CC_OK) rc = cc_color(ctx, seed, trials, k, &cid);
    if (rc == CC_OK) rc = cc_run_dp(ctx, pid, cid, &opts, &run);
    if (rc == CC_OK) rc = cc_count(ctx, run, h_counts);
    if (rc == CC_OK) rc = cc_decide(ctx, run, h_exists);
    cc_destroy(ctx);
  }
  cudaSetDevice(prev);
  return rc;
}
