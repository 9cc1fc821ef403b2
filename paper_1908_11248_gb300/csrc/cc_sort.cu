// Sorting and reduce-by-key of table records.
//
// The forget rule (Section 3.1) merges entries whose mappings become equal once the forgotten
// vertex is dropped.  Here the introduce below a forget writes its entries already projected
// (slot of the forgotten vertex removed), this file sorts them so that equal keys become
// adjacent, and reduce-by-key sums the counts of each run into one entry.  The sort order is
// chosen for the consumer: the G-vertices of the slots that the next introduce's vertex is
// adjacent to come first, so that runs of equal bag-neighbour images are contiguous and share
// their candidate lists (cc_kernels.cu, grouped introduce).
//
// Radix sort: least-significant digit first, 8 bits per pass, G blocks each owning one
// contiguous range of the input.  A pass is a per-block digit histogram, one exclusive scan
// over (digit, block) in digit-major order, and a scatter.  The scatter reads a tile of
// records, ranks equal digits in input order (warp match plus per-warp counts), stages the tile
// in shared memory grouped by digit and writes each digit's run with consecutive threads, so
// global writes are coalesced.  Every pass is stable, hence so is the sort.
#include <cstdint>

#include "cc_device.cuh"
#include "cc_internal.h"

namespace cc {
namespace {

using namespace dev;

template <typename K, typename SK, int BLOCK>
__global__ void __launch_bounds__(BLOCK) sort_hist_kernel(SortSpec sp, const void *src,
                                                          const u64 *n_ptr, u64 n_cap, int shift,
                                                          u64 *hist) {
  const u64 n = min(*n_ptr, n_cap);
  __shared__ unsigned s_h[256];
  const Slot<K> *in = reinterpret_cast<const Slot<K> *>(src);
  for (int d = threadIdx.x; d < 256; d += BLOCK) s_h[d] = 0;
  __syncthreads();
  const u64 G = gridDim.x, chunk = (n + G - 1) / G;
  const u64 lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  for (u64 i = lo + threadIdx.x; i < hi; i += BLOCK) {
    K key;
    u64 c;
    load_slot(in, i, key, c);
    if (key == 0) continue;
    atomicAdd(&s_h[(unsigned)(sort_key<SK>(key, sp) >> shift) & 255u], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += BLOCK) hist[(u64)d * G + blockIdx.x] = s_h[d];
}

// Offsets of the (digit, block) histogram, digit-major.  Block d scans row d (the counts of
// digit d over the G blocks) in place and writes the row total; then one block turns the 256
// row totals into digit bases at hist[256 * G + d].  A scatter's offset for (d, b) is
// hist[d * G + b] + hist[256 * G + d].
__global__ void __launch_bounds__(256) row_scan_kernel(u64 *hist, int G) {
  __shared__ u64 s_w[8];
  __shared__ u64 s_carry;
  u64 *row = hist + (u64)blockIdx.x * G;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int base = 0; base < G; base += 256) {
    const int i = base + threadIdx.x;
    const u64 v = i < G ? row[i] : 0;
    u64 x = v;
    for (int o = 1; o < 32; o <<= 1) {
      u64 y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_w[w] = x;
    __syncthreads();
    u64 before = s_carry;
    for (int q = 0; q < w; ++q) before += s_w[q];
    if (i < G) row[i] = before + x - v;
    __syncthreads();
    if (threadIdx.x == 255) s_carry = before + x;
    __syncthreads();
  }
  if (threadIdx.x == 0) hist[(u64)256 * G + 256 + blockIdx.x] = s_carry;
}

__global__ void __launch_bounds__(256) digit_base_kernel(u64 *hist, int G) {
  __shared__ u64 s_w[8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const u64 v = hist[(u64)256 * G + 256 + threadIdx.x];
  u64 x = v;
  for (int o = 1; o < 32; o <<= 1) {
    u64 y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[w] = x;
  __syncthreads();
  u64 before = 0;
  for (int q = 0; q < w; ++q) before += s_w[q];
  hist[(u64)256 * G + threadIdx.x] = before + x - v;
}

template <typename K, typename SK, int BLOCK, int ITEMS>
__global__ void __launch_bounds__(BLOCK) sort_scatter_kernel(SortSpec sp, const void *src,
                                                             const u64 *n_ptr, u64 n_cap,
                                                             int shift, const u64 *off,
                                                             void *dst, u64 dst_cap) {
  const u64 n = min(*n_ptr, n_cap);
  static_assert(BLOCK == 256, "one thread per digit");
  constexpr int W = BLOCK / 32, TILE = BLOCK * ITEMS;
  __shared__ Slot<K> s_stage[TILE];
  __shared__ unsigned char s_sdig[TILE];
  __shared__ unsigned s_wc[W][256];
  __shared__ unsigned s_thist[256], s_tstart[256], s_trun[256], s_wsum[W];
  __shared__ u64 s_brun[256];
  const Slot<K> *in = reinterpret_cast<const Slot<K> *>(src);
  Slot<K> *out = reinterpret_cast<Slot<K> *>(dst);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  s_brun[tid] = 0;
  for (int x = 0; x < W; ++x) s_wc[x][tid] = 0;
  const u64 G = gridDim.x, chunk = (n + G - 1) / G;
  const u64 lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  for (u64 tb = lo; tb < hi; tb += TILE) {
    K key[ITEMS];
    u64 cnt[ITEMS];
    int dig[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const u64 i = tb + (u64)j * BLOCK + tid;
      key[j] = 0;
      cnt[j] = 0;
      if (i < hi) load_slot(in, i, key[j], cnt[j]);
      dig[j] = key[j] != 0 ? (int)((unsigned)(sort_key<SK>(key[j], sp) >> shift) & 255u) : -1;
    }
    s_thist[tid] = 0;
    s_trun[tid] = 0;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < ITEMS; ++j)
      if (dig[j] >= 0) atomicAdd(&s_thist[dig[j]], 1u);
    __syncthreads();
    {  // exclusive scan of the tile histogram, thread d owns digit d
      unsigned v = s_thist[tid], x = v;
      for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) s_wsum[w] = x;
      __syncthreads();
      unsigned before = 0;
      for (int q = 0; q < w; ++q) before += s_wsum[q];
      s_tstart[tid] = before + x - v;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const int d = dig[j];
      const unsigned peers = __match_any_sync(0xffffffffu, d >= 0 ? d : 256 + lane);
      const int rank = __popc(peers & ((1u << lane) - 1u));
      if (d >= 0 && lane == __ffs(peers) - 1) s_wc[w][d] = __popc(peers);
      __syncthreads();
      {
        unsigned acc = s_trun[tid];
        for (int x = 0; x < W; ++x) {
          unsigned c = s_wc[x][tid];
          s_wc[x][tid] = acc;
          acc += c;
        }
        s_trun[tid] = acc;
      }
      __syncthreads();
      if (d >= 0) {
        const unsigned local = s_tstart[d] + s_wc[w][d] + rank;
        s_stage[local].key = key[j];
        s_stage[local].cnt = cnt[j];
        s_sdig[local] = (unsigned char)d;
      }
      __syncthreads();
      for (int x = 0; x < W; ++x) s_wc[x][tid] = 0;
      __syncthreads();
    }
    const unsigned tcount = s_tstart[255] + s_thist[255];
    for (unsigned i = tid; i < tcount; i += BLOCK) {
      const int d = s_sdig[i];
      const u64 pos = off[(u64)d * G + blockIdx.x] + off[256 * G + d] + s_brun[d] + (i - s_tstart[d]);
      if (pos < dst_cap) store_slot(out, pos, s_stage[i].key, s_stage[i].cnt);
    }
    __syncthreads();
    s_brun[tid] += s_thist[tid];
    __syncthreads();
  }
}

// ---- one-sweep passes ------------------------------------------------------------------
// All digit histograms come from one read of the input (per pass, 256 global counts turned into
// digit bases).  Each pass is then one kernel: blocks claim tiles in increasing order, publish
// their tile's digit counts, and find the counts of all earlier tiles by looking back through
// the published words (decoupled look-back): an "aggregate" word carries one tile's count, an
// "inclusive" word the sum over it and all tiles before it.  A word is (epoch << 48) |
// (inclusive << 47) | count; words of another epoch are not yet published.  Waiting for an
// earlier tile is bounded: after kSpinLimit polls the pass records a timeout and goes on.
constexpr u64 kCountMask = (1ull << 47) - 1ull;
constexpr unsigned kSpinLimit = 1u << 22;

template <typename K, typename SK, int BLOCK>
__global__ void __launch_bounds__(BLOCK) sweep_hist_kernel(SortSpec sp, const void *src,
                                                           const u64 *n_ptr, u64 n_cap,
                                                           int passes, u64 *ghist) {
  __shared__ unsigned h[16][256];
  const Slot<K> *in = reinterpret_cast<const Slot<K> *>(src);
  for (int i = threadIdx.x; i < 16 * 256; i += BLOCK) h[i / 256][i % 256] = 0;
  __syncthreads();
  const u64 n = min(*n_ptr, n_cap);
  for (u64 i = blockIdx.x * (u64)BLOCK + threadIdx.x; i < n; i += (u64)gridDim.x * BLOCK) {
    K key;
    u64 c;
    load_slot(in, i, key, c);
    if (key == 0) continue;
    const SK k = sort_key<SK>(key, sp);
    for (int p = 0; p < passes; ++p) atomicAdd(&h[p][(unsigned)(k >> (8 * p)) & 255u], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * 256; i += BLOCK)
    if (h[i / 256][i % 256]) atomicAdd(&ghist[i], (u64)h[i / 256][i % 256]);
}

// per pass (one block each): exclusive scan of its 256 digit counts, in place
__global__ void __launch_bounds__(256) sweep_bases_kernel(u64 *ghist) {
  __shared__ u64 s_w[8];
  u64 *row = ghist + (u64)blockIdx.x * 256;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const u64 v = row[threadIdx.x];
  u64 x = v;
  for (int o = 1; o < 32; o <<= 1) {
    u64 y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[w] = x;
  __syncthreads();
  u64 before = 0;
  for (int q = 0; q < w; ++q) before += s_w[q];
  row[threadIdx.x] = before + x - v;
}

// One pass.  Warp w of the block owns elements [w*32*ITEMS, (w+1)*32*ITEMS) of the tile, read
// in ITEMS coalesced rounds.  The tile's digit counts (shared-memory atomics) are published
// first, since every later tile's look-back waits for them; stable ranks then come from the
// warp's own sequential rounds (match on the digit, one leader per digit) on top of
// per-(warp, digit) bases, so a tile needs six block barriers.  With STORE_S the records leave carrying their sort key in place of the packed
// key (a full sort key is a bijection of the key): later passes read digits off it directly,
// and reduce-by-key turns it back.
template <typename K, typename SK, int BLOCK, int ITEMS, bool FROM_KEY, bool STORE_S>
__global__ void __launch_bounds__(BLOCK, 4) sweep_pass_kernel(SortSpec sp, const void *src,
                                                           const u64 *n_ptr, u64 n_cap, int shift,
                                                           u64 epoch, const u64 *bases,
                                                           u64 *status, unsigned *tile_ctr,
                                                           void *dst, u64 dst_cap, int *err) {
  static_assert(BLOCK == 256, "one thread per digit");
  constexpr int W = BLOCK / 32, TILE = BLOCK * ITEMS, PER_WARP = 32 * ITEMS;
  __shared__ Slot<K> s_stage[TILE];
  __shared__ unsigned char s_sdig[TILE];
  __shared__ unsigned s_wc[W][256];
  __shared__ unsigned s_tstart[256], s_wsum[W];
  __shared__ u64 s_excl[256];
  __shared__ unsigned s_tile, s_tcount, s_hist[256];
  const Slot<K> *in = reinterpret_cast<const Slot<K> *>(src);
  Slot<K> *out = reinterpret_cast<Slot<K> *>(dst);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const u64 n = min(*n_ptr, n_cap);
  const u64 tiles = (n + TILE - 1) / TILE;
  const u64 base_d = bases[tid];
  for (int x = 0; x < W; ++x) s_wc[x][tid] = 0;
  s_hist[tid] = 0;
  while (true) {
    if (tid == 0) s_tile = atomicAdd(tile_ctr, 1u);
    __syncthreads();  // (1) also orders the previous tile's write-out before reuse
    const u64 tile = s_tile;
    if (tile >= tiles) break;
    const u64 wb = tile * TILE + (u64)w * PER_WARP;
    K key[ITEMS];
    u64 cnt[ITEMS];
    int dig[ITEMS];
    unsigned peers[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {  // all loads first, so that they are in flight together
      const u64 i = wb + (u64)j * 32 + lane;
      key[j] = 0;
      cnt[j] = 0;
      if (i < n) load_slot(in, i, key[j], cnt[j]);
    }
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {  // digits, and the tile's digit counts
      if (key[j] != 0 && FROM_KEY && STORE_S) key[j] = (K)sort_key<SK>(key[j], sp);
      SK sk = (FROM_KEY && !STORE_S) ? sort_key<SK>(key[j], sp) : (SK)key[j];
      dig[j] = key[j] != 0 ? (int)((unsigned)(sk >> shift) & 255u) : -1;
      if (dig[j] >= 0) atomicAdd(&s_hist[dig[j]], 1u);
    }
    __syncthreads();  // (2)
    // publish this tile's count of digit tid before ranking: every later tile's look-back
    // waits for it
    const unsigned tcount_d = s_hist[tid];  // records of digit tid in this tile
    s_hist[tid] = 0;
    u64 *word = status + tile * 256 + tid;
    atomicExch(word, (epoch << 48) | (tile == 0 ? (1ull << 47) : 0ull) | tcount_d);
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {  // stable ranks: per-(warp, digit) counts in input order
      peers[j] = __match_any_sync(0xffffffffu, dig[j] >= 0 ? dig[j] : 256 + lane);
      if (dig[j] >= 0 && lane == __ffs(peers[j]) - 1) s_wc[w][dig[j]] += __popc(peers[j]);
      __syncwarp();
    }
    {  // look back for the tiles before this one
      u64 excl = 0;
      if (tile > 0) {
        long long j = (long long)tile - 1;
        unsigned spins = 0;
        while (j >= 0) {
          const u64 v = __ldcv(status + (u64)j * 256 + tid);
          if ((v >> 48) != epoch) {
            if (++spins > kSpinLimit) {
              atomicOr(err, kErrTimeout);
              break;
            }
            continue;
          }
          excl += v & kCountMask;
          if (v >> 47 & 1ull) break;
          --j;
        }
        atomicExch(word, (epoch << 48) | (1ull << 47) | (excl + tcount_d));
      }
      s_excl[tid] = base_d + excl;
    }
    __syncthreads();  // the per-warp counts are complete
    {  // tile-local start of digit tid, then each warp's base within it
      unsigned x = tcount_d;
      for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) s_wsum[w] = x;
      __syncthreads();  // (3)
      unsigned start = x - tcount_d;
      for (int q = 0; q < w; ++q) start += s_wsum[q];
      s_tstart[tid] = start;
      if (tid == 255) s_tcount = start + tcount_d;  // records in the tile
      for (int q = 0; q < W; ++q) {
        const unsigned c = s_wc[q][tid];
        s_wc[q][tid] = start;
        start += c;
      }
    }
    __syncthreads();  // (4)
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const int d = dig[j];
      if (d >= 0) {
        const unsigned local = s_wc[w][d] + __popc(peers[j] & lt);
        s_stage[local].key = key[j];
        s_stage[local].cnt = cnt[j];
        s_sdig[local] = (unsigned char)d;
      }
      __syncwarp();
      if (d >= 0 && lane == __ffs(peers[j]) - 1) s_wc[w][d] += __popc(peers[j]);
      __syncwarp();
    }
    __syncthreads();  // (5)
    const unsigned tcount = s_tcount;
    for (unsigned i = tid; i < tcount; i += BLOCK) {
      const int d = s_sdig[i];
      const u64 pos = s_excl[d] + (i - s_tstart[d]);
      if (pos < dst_cap) store_slot(out, pos, s_stage[i].key, s_stage[i].cnt);
    }
    for (int x = 0; x < W; ++x) s_wc[x][tid] = 0;
  }
}

// ---- one pass over 4096-record tiles: 512 threads, the first 256 owning one digit each ------
// The same steps as sweep_pass_kernel with twice the tile per block, so that each tile's
// fixed costs (claim, barriers, look-back over 256 digit words, publication) are spread over
// twice the records; the staging buffer lives in dynamic shared memory.
// KI: record type read; K: record type written (narrower when the records leave carrying a
// sort key of at most 64 bits in place of a 128-bit packed key).
template <typename K, typename SK, int ITEMS, bool FROM_KEY, bool STORE_S, typename KI = K>
__global__ void __launch_bounds__(512, 2) sweep_pass_wide_kernel(SortSpec sp, const void *src,
                                                                const u64 *n_ptr, u64 n_cap,
                                                                int shift, u64 epoch,
                                                                const u64 *bases, u64 *status,
                                                                unsigned *tile_ctr, void *dst,
                                                                u64 dst_cap, int *err) {
  constexpr int BLOCK = 512, W = BLOCK / 32, TILE = BLOCK * ITEMS, PER_WARP = 32 * ITEMS;
  extern __shared__ __align__(16) unsigned char s_wdyn[];
  Slot<K> *const s_stage = reinterpret_cast<Slot<K> *>(s_wdyn);
  unsigned char *const s_sdig = s_wdyn + (size_t)TILE * sizeof(Slot<K>);
  __shared__ unsigned s_wc[W][256];
  __shared__ unsigned s_tstart[256], s_wsum[8];
  __shared__ u64 s_excl[256];
  __shared__ unsigned s_tile, s_tcount, s_hist[256];
  const Slot<KI> *in = reinterpret_cast<const Slot<KI> *>(src);
  Slot<K> *out = reinterpret_cast<Slot<K> *>(dst);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const bool owner = tid < 256;  // warps 0..7: thread tid owns digit tid
  const unsigned lt = (1u << lane) - 1u;
  const u64 n = min(*n_ptr, n_cap);
  const u64 tiles = (n + TILE - 1) / TILE;
  const u64 base_d = owner ? bases[tid] : 0ull;
  if (owner) {
    for (int x = 0; x < W; ++x) s_wc[x][tid] = 0;
    s_hist[tid] = 0;
  }
  while (true) {
    if (tid == 0) s_tile = atomicAdd(tile_ctr, 1u);
    __syncthreads();  // also orders the previous tile's write-out before reuse
    const u64 tile = s_tile;
    if (tile >= tiles) break;
    const u64 wb = tile * TILE + (u64)w * PER_WARP;
    K key[ITEMS];
    u64 cnt[ITEMS];
    int dig[ITEMS];
    unsigned peers[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const u64 i = wb + (u64)j * 32 + lane;
      KI kin = 0;
      cnt[j] = 0;
      if (i < n) load_slot(in, i, kin, cnt[j]);
      // a full sort key never is 0 for a valid record: it holds the nonempty colour set
      key[j] = (FROM_KEY && STORE_S) ? (kin != 0 ? (K)sort_key<SK>(kin, sp) : (K)0) : (K)kin;
    }
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      SK sk = (FROM_KEY && !STORE_S) ? sort_key<SK>(key[j], sp) : (SK)key[j];
      dig[j] = key[j] != 0 ? (int)((unsigned)(sk >> shift) & 255u) : -1;
      if (dig[j] >= 0) atomicAdd(&s_hist[dig[j]], 1u);
    }
    __syncthreads();
    unsigned tcount_d = 0;
    u64 *word = status + tile * 256 + tid;
    if (owner) {  // publish this tile's count of digit tid
      tcount_d = s_hist[tid];
      s_hist[tid] = 0;
      atomicExch(word, (epoch << 48) | (tile == 0 ? (1ull << 47) : 0ull) | tcount_d);
    }
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      peers[j] = __match_any_sync(0xffffffffu, dig[j] >= 0 ? dig[j] : 256 + lane);
      if (dig[j] >= 0 && lane == __ffs(peers[j]) - 1) s_wc[w][dig[j]] += __popc(peers[j]);
      __syncwarp();
    }
    if (owner) {  // look back for the tiles before this one
      u64 excl = 0;
      if (tile > 0) {
        long long j = (long long)tile - 1;
        unsigned spins = 0;
        while (j >= 0) {
          const u64 v = __ldcv(status + (u64)j * 256 + tid);
          if ((v >> 48) != epoch) {
            if (++spins > kSpinLimit) {
              atomicOr(err, kErrTimeout);
              break;
            }
            continue;
          }
          excl += v & kCountMask;
          if (v >> 47 & 1ull) break;
          --j;
        }
        atomicExch(word, (epoch << 48) | (1ull << 47) | (excl + tcount_d));
      }
      s_excl[tid] = base_d + excl;
    }
    __syncthreads();  // the per-warp counts are complete
    unsigned x = tcount_d;
    if (owner) {
      for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) s_wsum[w] = x;
    }
    __syncthreads();
    if (owner) {  // tile-local start of digit tid, then each warp's base within it
      unsigned start = x - tcount_d;
      for (int q = 0; q < w; ++q) start += s_wsum[q];
      s_tstart[tid] = start;
      if (tid == 255) s_tcount = start + tcount_d;
      for (int q = 0; q < W; ++q) {
        const unsigned c = s_wc[q][tid];
        s_wc[q][tid] = start;
        start += c;
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const int d = dig[j];
      if (d >= 0) {
        const unsigned local = s_wc[w][d] + __popc(peers[j] & lt);
        s_stage[local].key = key[j];
        s_stage[local].cnt = cnt[j];
        s_sdig[local] = (unsigned char)d;
      }
      __syncwarp();
      if (d >= 0 && lane == __ffs(peers[j]) - 1) s_wc[w][d] += __popc(peers[j]);
      __syncwarp();
    }
    __syncthreads();
    const unsigned tcount = s_tcount;
    for (unsigned i = tid; i < tcount; i += BLOCK) {
      const int d = s_sdig[i];
      const u64 pos = s_excl[d] + (i - s_tstart[d]);
      if (pos < dst_cap) store_slot(out, pos, s_stage[i].key, s_stage[i].cnt);
    }
    if (owner)
      for (int q = 0; q < W; ++q) s_wc[q][tid] = 0;
  }
}

// ---- one pass with the next tile's records streamed in by the tensor memory accelerator ----
// The same ranking and look-back as sweep_pass_kernel, but a block claims its next tile as soon
// as it starts the current one and has the bulk-copy engine (cp.async.bulk) bring that tile's
// records into a second shared buffer meanwhile, so reads stay in flight while the block ranks,
// waits on its predecessors and writes out.  The current tile's buffer then serves as the
// staging area of its own scatter.  Waits on the copy barrier are bounded like the look-back.
__device__ __forceinline__ unsigned smem_addr(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(u64 *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

// thread 0: arm the barrier for `bytes` and copy them from global src to shared dst
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, u64 *bar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// true once the barrier's phase `parity` has completed; false after kSpinLimit polls
__device__ __forceinline__ bool mbar_wait(u64 *bar, unsigned parity) {
  for (unsigned spins = 0; spins < kSpinLimit; ++spins) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

template <typename K, typename SK, int ITEMS, bool FROM_KEY, bool STORE_S>
__global__ void __launch_bounds__(256, 3) sweep_pass_tma_kernel(SortSpec sp, const void *src,
                                                               const u64 *n_ptr, u64 n_cap,
                                                               int shift, u64 epoch,
                                                               const u64 *bases, u64 *status,
                                                               unsigned *tile_ctr, void *dst,
                                                               u64 dst_cap, int *err) {
  constexpr int BLOCK = 256, W = BLOCK / 32, TILE = BLOCK * ITEMS, PER_WARP = 32 * ITEMS;
  extern __shared__ __align__(128) unsigned char s_dyn[];  // two tiles of records
  Slot<K> *const s_buf0 = reinterpret_cast<Slot<K> *>(s_dyn);
  __shared__ __align__(8) u64 s_bar[2];
  __shared__ unsigned char s_sdig[TILE];
  __shared__ unsigned s_wc[W][256];
  __shared__ unsigned s_tstart[256], s_wsum[W];
  __shared__ u64 s_excl[256];
  __shared__ u64 s_tile[2];
  __shared__ unsigned s_tcount;
  const Slot<K> *in = reinterpret_cast<const Slot<K> *>(src);
  Slot<K> *out = reinterpret_cast<Slot<K> *>(dst);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const u64 n = min(*n_ptr, n_cap);
  const u64 tiles = (n + TILE - 1) / TILE;
  const u64 base_d = bases[tid];
  auto tile_bytes = [&](u64 t) {
    return (unsigned)(min((u64)TILE, n - t * TILE) * sizeof(Slot<K>));
  };
  for (int x = 0; x < W; ++x) s_wc[x][tid] = 0;
  if (tid == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const u64 t = atomicAdd(tile_ctr, 1u);
    s_tile[0] = t;
    if (t < tiles) bulk_load(s_buf0, in + t * TILE, tile_bytes(t), &s_bar[0]);
  }
  __syncthreads();
  unsigned phase = 0u;    // bit b: parity of buffer b's next copy
  unsigned pending = s_tile[0] < tiles ? 1u : 0u;  // bit b: a copy into b not yet waited for
  int cur = 0;
  while (true) {
    const u64 tile = s_tile[cur];
    if (tile >= tiles) break;
    if (tid == 0) {  // claim the next tile and start bringing it in
      const u64 t = atomicAdd(tile_ctr, 1u);
      s_tile[cur ^ 1] = t;
      if (t < tiles)
        bulk_load(s_buf0 + (cur ^ 1) * TILE, in + t * TILE, tile_bytes(t), &s_bar[cur ^ 1]);
    }
    const bool got = mbar_wait(&s_bar[cur], phase >> cur & 1u);
    if (got) {
      phase ^= 1u << cur;
      pending &= ~(1u << cur);
    }
    if (__syncthreads_or(!got)) {  // the copy never landed: give up on the pass
      if (tid == 0) atomicOr(err, kErrTimeout);
      break;
    }
    if (s_tile[cur ^ 1] < tiles) pending |= 1u << (cur ^ 1);
    Slot<K> *buf = s_buf0 + cur * TILE;
    const int wb = w * PER_WARP;
    K key[ITEMS];
    u64 cnt[ITEMS];
    int dig[ITEMS];
    unsigned peers[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const int i = wb + j * 32 + lane;
      key[j] = 0;
      cnt[j] = 0;
      if (tile * TILE + (u64)i < n) {
        key[j] = buf[i].key;
        cnt[j] = buf[i].cnt;
      }
    }
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      if (key[j] != 0 && FROM_KEY && STORE_S) key[j] = (K)sort_key<SK>(key[j], sp);
      SK sk = (FROM_KEY && !STORE_S) ? sort_key<SK>(key[j], sp) : (SK)key[j];
      dig[j] = key[j] != 0 ? (int)((unsigned)(sk >> shift) & 255u) : -1;
      peers[j] = __match_any_sync(0xffffffffu, dig[j] >= 0 ? dig[j] : 256 + lane);
      if (dig[j] >= 0 && lane == __ffs(peers[j]) - 1) s_wc[w][dig[j]] += __popc(peers[j]);
      __syncwarp();
    }
    __syncthreads();  // every record of buf is in registers; the counts are complete
    unsigned tcount_d = 0;
    for (int x = 0; x < W; ++x) tcount_d += s_wc[x][tid];
    {
      u64 *word = status + tile * 256 + tid;
      atomicExch(word, (epoch << 48) | (tile == 0 ? (1ull << 47) : 0ull) | tcount_d);
      u64 excl = 0;
      if (tile > 0) {
        long long j = (long long)tile - 1;
        unsigned spins = 0;
        while (j >= 0) {
          const u64 v = __ldcv(status + (u64)j * 256 + tid);
          if ((v >> 48) != epoch) {
            if (++spins > kSpinLimit) {
              atomicOr(err, kErrTimeout);
              break;
            }
            continue;
          }
          excl += v & kCountMask;
          if (v >> 47 & 1ull) break;
          --j;
        }
        atomicExch(word, (epoch << 48) | (1ull << 47) | (excl + tcount_d));
      }
      s_excl[tid] = base_d + excl;
    }
    {
      unsigned x = tcount_d;
      for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) s_wsum[w] = x;
      __syncthreads();
      unsigned start = x - tcount_d;
      for (int q = 0; q < w; ++q) start += s_wsum[q];
      s_tstart[tid] = start;
      if (tid == 255) s_tcount = start + tcount_d;
      for (int q = 0; q < W; ++q) {
        const unsigned c = s_wc[q][tid];
        s_wc[q][tid] = start;
        start += c;
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {  // stage the tile in digit order in its own buffer
      const int d = dig[j];
      if (d >= 0) {
        const unsigned local = s_wc[w][d] + __popc(peers[j] & lt);
        buf[local].key = key[j];
        buf[local].cnt = cnt[j];
        s_sdig[local] = (unsigned char)d;
      }
      __syncwarp();
      if (d >= 0 && lane == __ffs(peers[j]) - 1) s_wc[w][d] += __popc(peers[j]);
      __syncwarp();
    }
    __syncthreads();
    const unsigned tcount = s_tcount;
    for (unsigned i = tid; i < tcount; i += BLOCK) {
      const int d = s_sdig[i];
      const u64 pos = s_excl[d] + (i - s_tstart[d]);
      if (pos < dst_cap) store_slot(out, pos, buf[i].key, buf[i].cnt);
    }
    for (int x = 0; x < W; ++x) s_wc[x][tid] = 0;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();  // the staging is written out before the buffer receives a new tile
    cur ^= 1;
  }
  // leave no copy landing in shared memory after the block has gone
  for (int b = 0; b < 2; ++b)
    if ((pending >> b & 1u) && !mbar_wait(&s_bar[b], phase >> b & 1u) && tid == 0)
      atomicOr(err, kErrTimeout);
}

// ---- reduce by key: equal keys are adjacent; one record per run with the summed count ------
template <typename K, int BLOCK>
__global__ void __launch_bounds__(BLOCK) reduce_count_kernel(const void *src, const u64 *n_ptr,
                                                             u64 n_cap, u64 *blk) {
  const u64 n = min(*n_ptr, n_cap);
  __shared__ u64 s_red[BLOCK / 32];
  const Slot<K> *in = reinterpret_cast<const Slot<K> *>(src);
  const u64 G = gridDim.x, chunk = (n + G - 1) / G;
  const u64 lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  u64 heads = 0;
  for (u64 i = lo + threadIdx.x; i < hi; i += BLOCK) {
    K key, prev = 0;
    u64 c;
    load_slot(in, i, key, c);
    if (i > 0) load_slot(in, i - 1, prev, c);
    heads += key != prev;
  }
  u64 s = block_sum<BLOCK>(heads, s_red);
  if (threadIdx.x == 0) blk[blockIdx.x] = s;
}

// exclusive scan of the per-block counts (one block of 1024 threads); bases at blk[G..2G),
// total at blk[2G]
__global__ void __launch_bounds__(1024) blk_scan_kernel(u64 *blk, int G) {
  block_scan_array(blk, blk + G, (u64)G, blk + 2 * G);
}

// KI: record type read (64-bit sort keys when a 128-bit table's records were narrowed)
template <typename K, int BLOCK, bool FROM_S, typename KI = K>
__global__ void __launch_bounds__(BLOCK) reduce_write_kernel(const void *src, const u64 *n_ptr,
                                                             u64 n_cap, const u64 *blk, void *dst,
                                                             u64 *count, SortSpec sp) {
  const u64 n = min(*n_ptr, n_cap);
  __shared__ int s_wc[BLOCK / 32];
  const Slot<KI> *in = reinterpret_cast<const Slot<KI> *>(src);
  Slot<K> *out = reinterpret_cast<Slot<K> *>(dst);
  const u64 G = gridDim.x, chunk = (n + G - 1) / G;
  const u64 lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  u64 cursor = blk[G + blockIdx.x];
  for (u64 base = lo; base < hi; base += BLOCK) {
    const u64 i = base + threadIdx.x;
    bool head = false;
    KI key = 0;
    u64 sum = 0;
    if (i < hi) {
      KI prev = 0;
      u64 c;
      load_slot(in, i, key, sum);
      if (i > 0) load_slot(in, i - 1, prev, c);
      head = key != prev;
      if (head)  // the run may continue past this block's range
        for (u64 j = i + 1; j < n; ++j) {
          KI kj;
          load_slot(in, j, kj, c);
          if (kj != key) break;
          sum += c;
        }
    }
    int tot;
    const int rank = block_flag_rank<BLOCK>(head, s_wc, tot);
    if (head) store_slot(out, cursor + rank, FROM_S ? unsort_key((K)key, sp) : (K)key, sum);
    cursor += (u64)tot;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *count = blk[2 * G];
}

int grid256(const DevInfo &d) { return d.sms * d.blocks_per_sm; }

template <typename K, typename SK, int ITEMS>
int sort_impl(cudaStream_t s, const DevInfo &d, const SortSpec &sp, const void *src,
              const u64 *n_src, u64 src_cap, const u64 *n, u64 buf_cap, void *buf_a, void *buf_b,
              u64 *hist, int *which, const SweepScratch *sw) {
  const int G = grid256(d);
  const void *in = src;
  const u64 *n_in = n_src;
  u64 in_cap = src_cap;
  void *bufs[2] = {buf_a, buf_b};
  int cur = 0;
  const int passes = (sp.bits + 7) / 8;
  if (sw) {  // one-sweep: histograms once, then one kernel per pass
    cudaMemsetAsync(sw->ghist, 0, sizeof(u64) * 256 * passes, s);
    cudaMemsetAsync(sw->tile_ctr, 0, sizeof(unsigned) * passes, s);
    cudaMemsetAsync(sw->status, 0, sizeof(u64) * 256 * sw->max_tiles, s);
    sweep_hist_kernel<K, SK, 256><<<G, 256, 0, s>>>(sp, src, n_src, src_cap, passes, sw->ghist);
    sweep_bases_kernel<<<passes, 256, 0, s>>>(sw->ghist);
    constexpr int TI = ITEMS * 3 / 4;  // items per thread of the bulk-copy pass
    constexpr size_t TSMEM = 2 * 256 * TI * sizeof(Slot<K>);
    const int GT = d.sms * 3;
    // 64-bit records: 512-thread passes over 4096-record tiles
    constexpr bool WIDE = sizeof(K) == 8;
    constexpr size_t WSMEM = (size_t)512 * ITEMS * (sizeof(Slot<K>) + 1);
    const int GW = d.sms * 2;
    if constexpr (sizeof(K) == 16 && sizeof(SK) == 8) {
      if (sp.full && !sw->tma) {  // 16-byte (sort key, count) records from the first pass on
        constexpr size_t NSMEM = (size_t)512 * 8 * (sizeof(Slot<u64>) + 1);
        for (int p = 0; p < passes; ++p) {
          if (p == 0)
            sweep_pass_wide_kernel<u64, u64, 8, true, true, K><<<GW, 512, NSMEM, s>>>(
                sp, in, n_in, in_cap, 0, 1ull, sw->ghist, sw->status, sw->tile_ctr, bufs[cur],
                buf_cap, sw->err);
          else
            sweep_pass_wide_kernel<u64, u64, 8, false, true><<<GW, 512, NSMEM, s>>>(
                sp, in, n_in, in_cap, 8 * p, (u64)(p + 1), sw->ghist + 256 * p, sw->status,
                sw->tile_ctr + p, bufs[cur], buf_cap, sw->err);
          in = bufs[cur];
          n_in = n;
          in_cap = buf_cap;
          cur ^= 1;
        }
        *which = cur ^ 1;
        return (int)cudaGetLastError();
      }
    }
    for (int p = 0; p < passes; ++p) {
#define CC_PASS(FK, SS)                                                                   \
  if (sw->tma)                                                                            \
    sweep_pass_tma_kernel<K, SK, TI, FK, SS><<<GT, 256, TSMEM, s>>>(                       \
        sp, in, n_in, in_cap, 8 * p, (u64)(p + 1), sw->ghist + 256 * p, sw->status,       \
        sw->tile_ctr + p, bufs[cur], buf_cap, sw->err);                                   \
  else if (WIDE)                                                                          \
    sweep_pass_wide_kernel<K, SK, ITEMS, FK, SS><<<GW, 512, WSMEM, s>>>(                    \
        sp, in, n_in, in_cap, 8 * p, (u64)(p + 1), sw->ghist + 256 * p, sw->status,       \
        sw->tile_ctr + p, bufs[cur], buf_cap, sw->err);                                   \
  else                                                                                    \
    sweep_pass_kernel<K, SK, 256, ITEMS, FK, SS><<<G, 256, 0, s>>>(                        \
        sp, in, n_in, in_cap, 8 * p, (u64)(p + 1), sw->ghist + 256 * p, sw->status,       \
        sw->tile_ctr + p, bufs[cur], buf_cap, sw->err)
      if (!sp.full) {  // partial order: recompute the tuple each pass
        CC_PASS(true, false);
      } else if (p == 0) {  // full order: records carry their sort key after the first pass
        CC_PASS(true, true);
      } else {
        CC_PASS(false, true);
      }
#undef CC_PASS
      in = bufs[cur];
      n_in = n;
      in_cap = buf_cap;
      cur ^= 1;
    }
    *which = cur ^ 1;
    return (int)cudaGetLastError();
  }
  for (int shift = 0; shift < sp.bits; shift += 8) {
    sort_hist_kernel<K, SK, 256><<<G, 256, 0, s>>>(sp, in, n_in, in_cap, shift, hist);
    row_scan_kernel<<<256, 256, 0, s>>>(hist, G);
    digit_base_kernel<<<1, 256, 0, s>>>(hist, G);
    sort_scatter_kernel<K, SK, 256, ITEMS><<<G, 256, 0, s>>>(sp, in, n_in, in_cap, shift, hist,
                                                             bufs[cur], buf_cap);
    in = bufs[cur];
    n_in = n;
    in_cap = buf_cap;
    cur ^= 1;
  }
  *which = cur ^ 1;
  return (int)cudaGetLastError();
}

}  // namespace

int sort_grid(const DevInfo &d) { return grid256(d); }

int sort_passes(const SortSpec &sp) { return (sp.bits + 7) / 8; }

int sweep_tile(int kw) { return kw == 1 ? 256 * 6 : 256 * 3; }  // the smaller (bulk-copy) tile

namespace {
template <typename K, typename SK, int TI>
int allow_tma_smem() {
  constexpr int bytes = (int)(2 * 256 * TI * sizeof(Slot<K>));
  int r = 0;
  r |= (int)cudaFuncSetAttribute(sweep_pass_tma_kernel<K, SK, TI, true, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  r |= (int)cudaFuncSetAttribute(sweep_pass_tma_kernel<K, SK, TI, true, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  r |= (int)cudaFuncSetAttribute(sweep_pass_tma_kernel<K, SK, TI, false, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return r;
}
}  // namespace

template <typename SK>
int allow_wide_smem() {
  constexpr int bytes = 512 * 8 * (int)(sizeof(Slot<u64>) + 1);
  int r = 0;
  r |= (int)cudaFuncSetAttribute(sweep_pass_wide_kernel<u64, SK, 8, true, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  r |= (int)cudaFuncSetAttribute(sweep_pass_wide_kernel<u64, SK, 8, true, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  r |= (int)cudaFuncSetAttribute(sweep_pass_wide_kernel<u64, SK, 8, false, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  r |= (int)cudaFuncSetAttribute(sweep_pass_wide_kernel<u64, u64, 8, true, true, u128>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return r;
}

int prepare_sort_kernels() {
  int r = allow_tma_smem<u64, u64, 6>() | allow_tma_smem<u64, u128, 6>();
  r |= allow_wide_smem<u64>() | allow_wide_smem<u128>();
  r |= allow_tma_smem<u128, u64, 3>() | allow_tma_smem<u128, u128, 3>();
  return r;
}

int launch_sort_records(cudaStream_t s, const DevInfo &d, int kw, const SortSpec &sp,
                        const void *src, const unsigned long long *n_src,
                        unsigned long long src_cap, const unsigned long long *n,
                        unsigned long long buf_cap, void *buf_a, void *buf_b,
                        unsigned long long *hist, int *which, const SweepScratch *sw) {
  *which = -1;
  if (sp.bits == 0) return 0;
  if (kw == 1) {
    return sp.bits <= 64
               ? sort_impl<u64, u64, 8>(s, d, sp, src, n_src, src_cap, n, buf_cap, buf_a, buf_b,
                                        hist, which, sw)
               : sort_impl<u64, u128, 8>(s, d, sp, src, n_src, src_cap, n, buf_cap, buf_a, buf_b,
                                         hist, which, sw);
  }
  return sp.bits <= 64
             ? sort_impl<u128, u64, 4>(s, d, sp, src, n_src, src_cap, n, buf_cap, buf_a, buf_b,
                                       hist, which, sw)
             : sort_impl<u128, u128, 4>(s, d, sp, src, n_src, src_cap, n, buf_cap, buf_a, buf_b,
                                        hist, which, sw);
}

bool sort_narrows(int kw, const SortSpec &sp, int sort_sweep) {
  return kw == 2 && sp.full && sp.bits <= 64 && sort_sweep == 1;
}

int launch_reduce(cudaStream_t s, const DevInfo &d, int kw, const void *src,
                  const unsigned long long *n, unsigned long long n_cap, unsigned long long *blk,
                  void *dst, unsigned long long *count, const SortSpec *from_s, bool narrow) {
  const int G = grid256(d);
  const SortSpec sp = from_s ? *from_s : SortSpec{};
  if (kw == 1 || narrow) reduce_count_kernel<u64, 256><<<G, 256, 0, s>>>(src, n, n_cap, blk);
  else reduce_count_kernel<u128, 256><<<G, 256, 0, s>>>(src, n, n_cap, blk);
  blk_scan_kernel<<<1, 1024, 0, s>>>(blk, G);
  if (narrow && from_s) {  // 64-bit sort keys in, 128-bit packed keys out
    reduce_write_kernel<u128, 256, true, u64><<<G, 256, 0, s>>>(src, n, n_cap, blk, dst, count,
                                                                sp);
  } else if (kw == 1) {
    if (from_s)
      reduce_write_kernel<u64, 256, true><<<G, 256, 0, s>>>(src, n, n_cap, blk, dst, count, sp);
    else
      reduce_write_kernel<u64, 256, false><<<G, 256, 0, s>>>(src, n, n_cap, blk, dst, count, sp);
  } else {
    if (from_s)
      reduce_write_kernel<u128, 256, true><<<G, 256, 0, s>>>(src, n, n_cap, blk, dst, count, sp);
    else
      reduce_write_kernel<u128, 256, false><<<G, 256, 0, s>>>(src, n, n_cap, blk, dst, count, sp);
  }
  return (int)cudaGetLastError();
}

}  // namespace cc
