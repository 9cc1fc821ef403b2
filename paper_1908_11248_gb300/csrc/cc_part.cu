// Bucketed merge of a forget's records (Section 3.1, forget rule: entries whose mappings agree
// once the forgotten vertex is dropped are merged, their counts summed).
//
// The records an introduce wrote already projected (the forgotten slot removed) are merged by
// key and ordered for the next node in four steps:
//   1. a histogram of buckets: the top hb bits of a hash of the images of the next introduce's
//      bag-neighbour slots (of the whole key when it has none), one global add per record;
//   2. an exclusive scan of the histogram: where every bucket starts;
//   3. a split of the records into buckets, most significant bucket bits first, one or two
//      splits of at most 10 bits: each tile counts its records per digit in shared memory,
//      reserves room for each digit with one global add and writes each digit's records together;
//   4. per bucket, in bucket order, a sort of the bucket by the full key order (8-bit LSD passes,
//      in shared memory, or in global scratch for a bucket larger than shared memory), a merge of
//      equal keys (counts summed mod 2^64), and a write at the bucket's place in the output, found
//      by a decoupled look-back over the earlier buckets' merged counts (bounded waits).
// The result is a dense table sorted by (bucket, full sort key): equal keys merged, the records
// of equal bag-neighbour images in one run, and every key findable by binary search.
#include <cstdint>

#include "cc_device.cuh"
#include "cc_internal.h"

namespace cc {
namespace {

using namespace dev;

// polls of a look-back wait before it gives up (with back-off of up to 4 us a poll: seconds)
constexpr unsigned kPartSpinLimit = 1u << 22;
constexpr u64 kAvail = 1ull << 62, kIncl = 1ull << 63, kCnt = (1ull << 62) - 1ull;

// ---- 1. histogram of buckets -------------------------------------------------------------
template <typename K>
__global__ void __launch_bounds__(256) part_hist_kernel(SortSpec sp, const void *src,
                                                        const u64 *n_src, u64 src_cap,
                                                        unsigned *hist) {
  const Slot<K> *in = reinterpret_cast<const Slot<K> *>(src);
  const u64 n = min(*n_src, src_cap);
  for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < n;
       i += (u64)gridDim.x * blockDim.x) {
    K key;
    u64 c;
    load_slot(in, i, key, c);
    if (key != 0) atomicAdd(&hist[sort_bucket(key, sp)], 1u);
  }
}

// ---- 2. bucket starts (a multi-block exclusive scan of the histogram, total at base[F]) and the
// split cursors: cur2[b] = base[b]; cur1[d] = base[d << h2] ------------------------------------
__global__ void __launch_bounds__(256) part_cursor_kernel(const u64 *base, u64 F, int h2,
                                                          u64 *cur1, u64 *cur2) {
  for (u64 b = blockIdx.x * (u64)blockDim.x + threadIdx.x; b < F;
       b += (u64)gridDim.x * blockDim.x) {
    cur2[b] = base[b];
    if ((b & ((1ull << h2) - 1ull)) == 0) cur1[b >> h2] = base[b];
  }
}

// ---- 3. split into buckets ------------------------------------------------------------------
// LEVEL 1: tiles of the whole source (holes skipped), digit = bucket >> h2, room from cur[digit].
// LEVEL 2: tiles inside each first-level group (2^h2 consecutive buckets, placed by level 1),
// digit = bucket & (2^h2 - 1), room from cur[bucket].
template <typename K, int BLOCK, int ITEMS, int LEVEL>
__global__ void __launch_bounds__(BLOCK) part_split_kernel(SortSpec sp, const void *src,
                                                           const u64 *n_src, u64 src_cap,
                                                           int h1, int h2, const u64 *base,
                                                           u64 F, u64 *cur, void *dst,
                                                           u64 dst_cap) {
  constexpr int TILE = BLOCK * ITEMS;
  extern __shared__ __align__(16) unsigned char s_dyn[];
  Slot<K> *s_stage = reinterpret_cast<Slot<K> *>(s_dyn);
  unsigned short *s_sdig = reinterpret_cast<unsigned short *>(s_dyn + TILE * sizeof(Slot<K>));
  __shared__ unsigned s_cnt[1024], s_off[1024];
  __shared__ u64 s_gbase[1024];
  __shared__ unsigned s_wsum[BLOCK / 32];
  __shared__ u64 s_tstart[1025];
  __shared__ unsigned s_total;
  const Slot<K> *in = reinterpret_cast<const Slot<K> *>(src);
  Slot<K> *out = reinterpret_cast<Slot<K> *>(dst);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int dbits = LEVEL == 1 ? h1 : h2;
  const int D = 1 << dbits;
  const int G1 = 1 << h1;
  // tiles: LEVEL 1 over [0, n); LEVEL 2 per group g over [base[g << h2], base[(g+1) << h2])
  u64 ntiles;
  const u64 n = LEVEL == 1 ? min(*n_src, src_cap) : 0;
  if (LEVEL == 1) {
    ntiles = (n + TILE - 1) / TILE;
  } else {
    if (tid == 0) {
      u64 t = 0;
      for (int g = 0; g < G1; ++g) {
        s_tstart[g] = t;
        t += (base[(u64)(g + 1) << h2] - base[(u64)g << h2] + TILE - 1) / TILE;
      }
      s_tstart[G1] = t;
    }
    __syncthreads();
    ntiles = s_tstart[G1];
  }
  for (u64 tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    u64 lo, hi;
    int g = 0;
    if (LEVEL == 1) {
      lo = tile * TILE;
      hi = min(n, lo + TILE);
    } else {
      int a = 0, b = G1 - 1;  // the group whose tiles hold this one
      while (a < b) {
        const int m = (a + b + 1) >> 1;
        if (s_tstart[m] <= tile) a = m;
        else b = m - 1;
      }
      g = a;
      const u64 glo = base[(u64)g << h2], ghi = base[(u64)(g + 1) << h2];
      lo = glo + (tile - s_tstart[g]) * TILE;
      hi = min(ghi, lo + TILE);
    }
    for (int d = tid; d < D; d += BLOCK) s_cnt[d] = 0;
    __syncthreads();
    K key[ITEMS];
    u64 cnt[ITEMS];
    int dig[ITEMS];
    unsigned rk[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const u64 i = lo + (u64)j * BLOCK + tid;
      key[j] = 0;
      cnt[j] = 0;
      if (i < hi) load_slot(in, i, key[j], cnt[j]);
    }
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      dig[j] = -1;
      if (key[j] != 0) {
        const uint32_t bk = sort_bucket(key[j], sp);
        dig[j] = LEVEL == 1 ? (int)(bk >> h2) : (int)(bk & ((1u << h2) - 1u));
        rk[j] = atomicAdd(&s_cnt[dig[j]], 1u);
      }
    }
    __syncthreads();
    // exclusive scan of the tile's digit counts; one global reservation per nonempty digit
    {
      constexpr int PER = 1024 / BLOCK;
      unsigned v[PER], x = 0;
#pragma unroll
      for (int k = 0; k < PER; ++k) {
        const int d = tid * PER + k;
        v[k] = d < D ? s_cnt[d] : 0u;
        x += v[k];
      }
      unsigned incl = x;
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      if (lane == 31) s_wsum[w] = incl;
      __syncthreads();
      unsigned before = incl - x;
      for (int q = 0; q < w; ++q) before += s_wsum[q];
      if (tid == BLOCK - 1) s_total = before + x;
#pragma unroll
      for (int k = 0; k < PER; ++k) {
        const int d = tid * PER + k;
        if (d < D) {
          s_off[d] = before;
          if (v[k]) {
            const u64 gi = LEVEL == 1 ? (u64)d : ((u64)g << h2) | (u64)d;
            s_gbase[d] = atomicAdd(&cur[gi], (u64)v[k]);
          }
        }
        before += v[k];
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < ITEMS; ++j)
      if (dig[j] >= 0) {
        const unsigned p = s_off[dig[j]] + rk[j];
        s_stage[p].key = key[j];
        s_stage[p].cnt = cnt[j];
        s_sdig[p] = (unsigned short)dig[j];
      }
    __syncthreads();
    const unsigned tcount = s_total;
    for (unsigned i = tid; i < tcount; i += BLOCK) {
      const int d = s_sdig[i];
      const u64 pos = s_gbase[d] + (i - s_off[d]);
      if (pos < dst_cap) store_slot(out, pos, s_stage[i].key, s_stage[i].cnt);
    }
    __syncthreads();
  }
}

// ---- 4. per-bucket sort, merge and placement -----------------------------------------------
// Sort keys and counts as separate arrays (generic pointers: shared memory, or global scratch
// for a bucket larger than shared memory).
template <typename SK>
struct Lanes {
  SK *k;
  u64 *c;
};

// One stable LSD pass by 8 bits at `shift` of the S records of src into dst, by the block: a
// digit histogram over all records, its exclusive scan, then chunk by chunk (CHUNK records, in
// order) per-warp stable ranks from warp matches on the digit.
template <typename SK, int BLOCK, int ITEMS>
__device__ __forceinline__ void lsd_pass(Lanes<SK> src, Lanes<SK> dst, unsigned S, int shift,
                                         unsigned (*s_wc)[256], unsigned *s_dpos,
                                         unsigned *s_wsum) {
  constexpr int W = BLOCK / 32, CHUNK = BLOCK * ITEMS, PER_WARP = 32 * ITEMS;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const unsigned lt = (1u << lane) - 1u;
  // digit totals and their exclusive scan (thread d < 256 owns digit d)
  if (tid < 256) s_wc[0][tid] = 0;
  __syncthreads();
  for (unsigned i = tid; i < S; i += BLOCK)
    atomicAdd(&s_wc[0][(unsigned)(src.k[i] >> shift) & 255u], 1u);
  __syncthreads();
  unsigned v = 0, incl = 0;
  if (tid < 256) {  // whole warps
    v = s_wc[0][tid];
    incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) s_wsum[w] = incl;
  }
  __syncthreads();
  if (tid < 256) {
    unsigned before = 0;
    for (int q = 0; q < w; ++q) before += s_wsum[q];
    s_dpos[tid] = before + incl - v;
  }
  __syncthreads();
  for (unsigned c0 = 0; c0 < S; c0 += CHUNK) {
    for (int x = 0; x < W; ++x) s_wc[x][tid & 255] = 0;
    __syncthreads();
    int dig[ITEMS];
    unsigned peers[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const unsigned i = c0 + w * PER_WARP + j * 32 + lane;
      dig[j] = i < S ? (int)((unsigned)(src.k[i] >> shift) & 255u) : -1;
      peers[j] = __match_any_sync(0xffffffffu, dig[j] >= 0 ? dig[j] : 256 + lane);
      if (dig[j] >= 0 && lane == __ffs(peers[j]) - 1) s_wc[w][dig[j]] += __popc(peers[j]);
      __syncwarp();
    }
    __syncthreads();
    if (tid < 256) {  // per-warp starts of digit tid in this chunk; advance the digit's start
      unsigned start = s_dpos[tid];
      for (int x = 0; x < W; ++x) {
        const unsigned cc = s_wc[x][tid];
        s_wc[x][tid] = start;
        start += cc;
      }
      s_dpos[tid] = start;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const int d = dig[j];
      const unsigned i = c0 + w * PER_WARP + j * 32 + lane;
      if (d >= 0) {
        const unsigned pos = s_wc[w][d] + __popc(peers[j] & lt);
        dst.k[pos] = src.k[i];
        dst.c[pos] = src.c[i];
      }
      __syncwarp();
      if (d >= 0 && lane == __ffs(peers[j]) - 1) s_wc[w][d] += __popc(peers[j]);
      __syncwarp();
    }
    __syncthreads();
  }
}

template <typename K, typename SK, int BLOCK, int ITEMS>
__global__ void __launch_bounds__(BLOCK) part_local_kernel(
    SortSpec sp, const void *xsrc, void *yspace, const unsigned *hist, const u64 *base, u64 F,
    u64 *status, unsigned *claim, void *dst, u64 dst_cap, u64 *dst_count, int *err) {
  constexpr int CAP = BLOCK * ITEMS, W = BLOCK / 32;
  extern __shared__ __align__(16) unsigned char s_dyn[];
  SK *s_k0 = reinterpret_cast<SK *>(s_dyn);
  SK *s_k1 = s_k0 + CAP;
  u64 *s_c0 = reinterpret_cast<u64 *>(s_k1 + CAP);
  u64 *s_c1 = s_c0 + CAP;
  __shared__ unsigned s_wc[W][256];
  __shared__ unsigned s_dpos[256], s_wsum[BLOCK / 32];
  __shared__ int s_wflag[BLOCK / 32];
  __shared__ u64 s_b, s_excl;
  __shared__ unsigned s_m;
  const Slot<K> *in = reinterpret_cast<const Slot<K> *>(xsrc);
  Slot<K> *out = reinterpret_cast<Slot<K> *>(dst);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int passes = (sp.bits + 7) / 8;
  for (;;) {
    if (tid == 0) s_b = atomicAdd(claim, 1u);
    __syncthreads();
    const u64 b = s_b;
    if (b >= F) break;
    const u64 st = base[b];
    const unsigned S = hist[b];
    Lanes<SK> A, B;
    if (S <= (unsigned)CAP) {
      A = Lanes<SK>{s_k0, s_c0};
      B = Lanes<SK>{s_k1, s_c1};
    } else {  // larger than shared memory: sort keys and counts in the bucket's own ranges of the
              // two record spaces (each S records of at least sizeof(SK) + 8 bytes)
      unsigned char *yb = reinterpret_cast<unsigned char *>(yspace) + st * sizeof(Slot<K>);
      unsigned char *xb = const_cast<unsigned char *>(
                              reinterpret_cast<const unsigned char *>(xsrc)) +
                          st * sizeof(Slot<K>);
      A = Lanes<SK>{reinterpret_cast<SK *>(yb), reinterpret_cast<u64 *>(yb + (u64)S * sizeof(SK))};
      B = Lanes<SK>{reinterpret_cast<SK *>(xb), reinterpret_cast<u64 *>(xb + (u64)S * sizeof(SK))};
    }
    for (unsigned i = tid; i < S; i += BLOCK) {
      K key;
      u64 c;
      load_slot(in, st + i, key, c);
      A.k[i] = sort_key<SK>(key, sp);
      A.c[i] = c;
    }
    __syncthreads();
    for (int p = 0; p < passes; ++p) {
      lsd_pass<SK, BLOCK, ITEMS>(A, B, S, 8 * p, s_wc, s_dpos, s_wsum);
      const Lanes<SK> t = A;
      A = B;
      B = t;
    }
    // merge runs of equal keys into B (compacted, counts summed); m = merged records
    unsigned m = 0;
    for (unsigned c0 = 0; c0 < S; c0 += BLOCK) {
      const unsigned i = c0 + tid;
      bool head = false;
      SK k = 0;
      u64 sum = 0;
      if (i < S) {
        k = A.k[i];
        head = i == 0 || A.k[i - 1] != k;
        if (head) {
          sum = A.c[i];
          for (unsigned j = i + 1; j < S && A.k[j] == k; ++j) sum += A.c[j];
        }
      }
      const unsigned bal = __ballot_sync(0xffffffffu, head);
      if (lane == 0) s_wflag[w] = __popc(bal);
      __syncthreads();
      unsigned before = 0, tot = 0;
      for (int q = 0; q < BLOCK / 32; ++q) {
        before += q < w ? (unsigned)s_wflag[q] : 0u;
        tot += (unsigned)s_wflag[q];
      }
      if (head) {
        const unsigned r = m + before + __popc(bal & ((1u << lane) - 1u));
        B.k[r] = k;
        B.c[r] = sum;
      }
      m += tot;
      __syncthreads();
    }
    // place the bucket: publish its merged count, then look back for the earlier buckets'
    if (tid == 0) {
      u64 excl = 0;
      if (b == 0) {
        atomicExch(&status[0], kAvail | kIncl | (u64)m);
      } else {
        atomicExch(&status[b], kAvail | (u64)m);
        long long j = (long long)b - 1;
        unsigned spins = 0;
        unsigned nap = 32;
        while (j >= 0) {
          const u64 v = __ldcv(status + j);
          if (!(v & kAvail)) {
            // an earlier bucket is still being sorted (a large one can take milliseconds):
            // back off, and give up after kPartSpinLimit polls
            if (++spins > kPartSpinLimit) {
              atomicOr(err, kErrTimeout);
              break;
            }
            __nanosleep(nap);
            if (nap < 4096) nap <<= 1;
            continue;
          }
          excl += v & kCnt;
          if (v & kIncl) break;
          --j;
        }
        atomicExch(&status[b], kAvail | kIncl | (excl + m));
      }
      s_excl = excl;
      s_m = m;
      if (b == F - 1) *dst_count = excl + m;
    }
    __syncthreads();
    const u64 o0 = s_excl;
    for (unsigned i = tid; i < s_m; i += BLOCK)
      if (o0 + i < dst_cap) store_slot(out, o0 + i, unsort_key((K)B.k[i], sp), B.c[i]);
    __syncthreads();
  }
}

int grid_of(const DevInfo &d) { return d.sms * d.blocks_per_sm; }

template <typename K, int BLOCK, int ITEMS, int LEVEL>
int allow_split_smem() {
  const int bytes = BLOCK * ITEMS * (int)(sizeof(Slot<K>) + sizeof(unsigned short));
  return (int)cudaFuncSetAttribute(part_split_kernel<K, BLOCK, ITEMS, LEVEL>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <typename K, typename SK, int BLOCK, int ITEMS>
int allow_local_smem() {
  const int bytes = 2 * BLOCK * ITEMS * (int)(sizeof(SK) + sizeof(u64));
  return (int)cudaFuncSetAttribute(part_local_kernel<K, SK, BLOCK, ITEMS>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// tile shapes: splits over 256 threads; local sorts over 256 threads, CAP records of shared memory
template <typename K>
struct PartShape;
template <>
struct PartShape<u64> {
  static constexpr int kSplitItems = 16;
};
template <>
struct PartShape<u128> {
  static constexpr int kSplitItems = 8;
};
template <typename SK>
struct LocalShape;
template <>
struct LocalShape<u64> {
  static constexpr int kItems = 8;  // 2048 records: 64 KB of sort keys and counts
};
template <>
struct LocalShape<u128> {
  static constexpr int kItems = 6;  // 1536 records: 72 KB
};

template <typename K, typename SK>
int part_impl(cudaStream_t s, const DevInfo &d, const SortSpec &sp, const void *src,
              const u64 *n_src, u64 src_cap, void *mid, void *spare, u64 space_cap,
              const PartScratch &ps, void *dst, u64 dst_cap, u64 *dst_count) {
  const int hb = sp.hbits, h2 = hb > 10 ? hb / 2 : 0, h1 = hb - h2;
  const u64 F = 1ull << hb;
  constexpr int SI = PartShape<K>::kSplitItems, LI = LocalShape<SK>::kItems;
  const int G = grid_of(d);
  int r = 0;
  r |= (int)cudaMemsetAsync(ps.hist, 0, F * sizeof(unsigned), s);
  r |= (int)cudaMemsetAsync(ps.status, 0, F * sizeof(u64), s);
  r |= (int)cudaMemsetAsync(ps.claim, 0, sizeof(unsigned), s);
  part_hist_kernel<K><<<G, 256, 0, s>>>(sp, src, n_src, src_cap, ps.hist);
  r |= launch_scan_u32(s, d, ps.hist, F, ps.base, ps.scan);
  part_cursor_kernel<<<d.sms * 4, 256, 0, s>>>(ps.base, F, h2, ps.cur1, ps.cur2);
  const size_t split_smem = 256 * SI * (sizeof(Slot<K>) + sizeof(unsigned short));
  // one split: src -> mid, buckets sorted from mid with src as the spare space; two splits:
  // src -> mid -> spare, buckets sorted from spare with mid as the spare space
  part_split_kernel<K, 256, SI, 1><<<G, 256, split_smem, s>>>(
      sp, src, n_src, src_cap, h1, h2, ps.base, F, h2 ? ps.cur1 : ps.cur2, mid, space_cap);
  void *x = mid, *y = const_cast<void *>(src);
  if (h2) {
    part_split_kernel<K, 256, SI, 2><<<G, 256, split_smem, s>>>(
        sp, mid, ps.base + F, space_cap, h1, h2, ps.base, F, ps.cur2, spare, space_cap);
    x = spare;
    y = mid;
  }
  SortSpec local = sp;
  local.hbits = 0;  // inside a bucket: the plain full order
  const size_t local_smem = 2 * 256 * LI * (sizeof(SK) + sizeof(u64));
  part_local_kernel<K, SK, 256, LI><<<G, 256, local_smem, s>>>(
      local, x, y, ps.hist, ps.base, F, ps.status, ps.claim, dst, dst_cap, dst_count, ps.err);
  r |= (int)cudaGetLastError();
  return r;
}

}  // namespace

int prepare_part_kernels() {
  int r = 0;
  r |= allow_split_smem<u64, 256, PartShape<u64>::kSplitItems, 1>();
  r |= allow_split_smem<u64, 256, PartShape<u64>::kSplitItems, 2>();
  r |= allow_split_smem<u128, 256, PartShape<u128>::kSplitItems, 1>();
  r |= allow_split_smem<u128, 256, PartShape<u128>::kSplitItems, 2>();
  r |= allow_local_smem<u64, u64, 256, LocalShape<u64>::kItems>();
  r |= allow_local_smem<u64, u128, 256, LocalShape<u128>::kItems>();
  r |= allow_local_smem<u128, u64, 256, LocalShape<u64>::kItems>();
  r |= allow_local_smem<u128, u128, 256, LocalShape<u128>::kItems>();
  return r;
}

int part_bucket_bits(unsigned long long records, int kw) {
  // about half a shared-memory bucket per bucket on average
  const unsigned long long cap = kw == 1 ? 1024 : 768;
  int hb = 1;
  while (hb < 20 && (records >> hb) > cap) ++hb;
  return hb;
}

int launch_part_merge(cudaStream_t s, const DevInfo &d, int kw, const SortSpec &sp,
                      const void *src, const unsigned long long *n_src,
                      unsigned long long src_cap, void *mid, void *spare,
                      unsigned long long space_cap, const PartScratch &ps, void *dst,
                      unsigned long long dst_cap, unsigned long long *dst_count) {
  if (kw == 1)
    return sp.bits <= 64 ? part_impl<u64, u64>(s, d, sp, src, n_src, src_cap, mid, spare,
                                               space_cap, ps, dst, dst_cap, dst_count)
                         : part_impl<u64, u128>(s, d, sp, src, n_src, src_cap, mid, spare,
                                                space_cap, ps, dst, dst_cap, dst_count);
  return sp.bits <= 64 ? part_impl<u128, u64>(s, d, sp, src, n_src, src_cap, mid, spare,
                                              space_cap, ps, dst, dst_cap, dst_count)
                       : part_impl<u128, u128>(s, d, sp, src, n_src, src_cap, mid, spare,
                                               space_cap, ps, dst, dst_cap, dst_count);
}

}  // namespace cc
