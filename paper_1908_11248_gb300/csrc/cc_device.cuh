// Device helpers shared by the kernel translation units: table records, packed-key field
// access, record loads and stores, the open-addressing hash table, block-wide scans and the
// sorted-adjacency membership test.  Everything here is inline device code.
#pragma once

#include <climits>
#include <cstdint>

#include "cc_internal.h"

namespace cc {
namespace dev {

typedef unsigned long long u64;
typedef unsigned __int128 u128;

template <typename K>
struct alignas(sizeof(K) == 8 ? 16 : 32) Slot {
  K key;
  u64 cnt;
};

// ---- key helpers ------------------------------------------------------------------------
template <typename K>
__device__ __forceinline__ K low_mask(int s) {
  return s >= (int)(8 * sizeof(K)) ? ~(K)0 : (((K)1 << s) - (K)1);
}

template <typename K>
__device__ __forceinline__ int key_slot(K key, const KeyLayout &L, int i) {
  return (int)((key >> (L.k + i * L.nb)) & (K)((1ull << L.nb) - 1ull));
}

template <typename K>
__device__ __forceinline__ uint32_t key_mask(K key, const KeyLayout &L) {
  return (uint32_t)(key & (K)((1ull << L.k) - 1ull));
}

template <typename K>
__device__ __forceinline__ int key_trial(K key, const KeyLayout &L) {
  return L.tb ? (int)(key >> L.tpos) : 0;
}

template <typename K>
__device__ __forceinline__ K key_trial_bits(K key, const KeyLayout &L) {
  return L.tb ? (key >> L.tpos) << L.tpos : (K)0;
}

// insert vertex v as slot p of a bag that had b slots
template <typename K>
__device__ __forceinline__ K key_insert(K key, const KeyLayout &L, int p, int v) {
  K body = key & low_mask<K>(L.tpos);
  int lo = L.k + p * L.nb;
  K lower = body & low_mask<K>(lo);
  K upper = body >> lo;
  return lower | ((K)(unsigned)v << lo) | (upper << (lo + L.nb)) | key_trial_bits(key, L);
}

// drop slot q
template <typename K>
__device__ __forceinline__ K key_remove(K key, const KeyLayout &L, int q) {
  K body = key & low_mask<K>(L.tpos);
  int lo = L.k + q * L.nb;
  K lower = body & low_mask<K>(lo);
  K upper = body >> (lo + L.nb);
  return lower | (upper << lo) | key_trial_bits(key, L);
}

// MurmurHash3 64-bit finaliser (Appleby), a published bit mixer
static __device__ __forceinline__ u64 fmix64(u64 x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ull;
  x ^= x >> 33;
  return x;
}
static __device__ __forceinline__ u64 key_hash(u64 k) { return fmix64(k); }
static __device__ __forceinline__ u64 key_hash(u128 k) { return fmix64((u64)k ^ fmix64((u64)(k >> 64))); }

// ---- record load/store (16-byte vector accesses) ---------------------------------------
static __device__ __forceinline__ void load_slot(const Slot<u64> *s, u64 i, u64 &key, u64 &cnt) {
  ulonglong2 r = reinterpret_cast<const ulonglong2 *>(s)[i];
  key = r.x;
  cnt = r.y;
}
static __device__ __forceinline__ void load_slot(const Slot<u128> *s, u64 i, u128 &key, u64 &cnt) {
  const ulonglong2 *p = reinterpret_cast<const ulonglong2 *>(s) + 2 * i;
  ulonglong2 a = p[0];
  key = ((u128)a.y << 64) | a.x;
  cnt = p[1].x;
}
static __device__ __forceinline__ void store_slot(Slot<u64> *s, u64 i, u64 key, u64 cnt) {
  reinterpret_cast<ulonglong2 *>(s)[i] = make_ulonglong2(key, cnt);
}
static __device__ __forceinline__ void store_slot(Slot<u128> *s, u64 i, u128 key, u64 cnt) {
  ulonglong2 *p = reinterpret_cast<ulonglong2 *>(s) + 2 * i;
  p[0] = make_ulonglong2((u64)key, (u64)(key >> 64));
  p[1] = make_ulonglong2(cnt, 0ull);
}

template <typename K>
__device__ __forceinline__ u64 table_bound(const TableDesc &t) {
  if (t.hashed) return t.cap;
  u64 c = *t.count;
  return c < t.cap ? c : t.cap;
}

// ---- hash table (open addressing, linear probing, key claimed by compare-and-swap) -------
// The home slot of a key is its 64-bit hash scaled to [0, cap) by a multiply-high (Lemire's
// range reduction), so capacities need not be powers of two.
static __device__ __forceinline__ u64 home_slot(u64 h, u64 cap) { return __umul64hi(h, cap); }
static __device__ __forceinline__ u64 next_slot(u64 h, u64 cap) { return h + 1 == cap ? 0 : h + 1; }

// Longest probe sequence of an insert or a lookup.  An insert that finds no room within it
// reports a full table (the caller flags an overflow), so every key that was inserted lies within
// this many slots of its home and a lookup may stop there too.  A table at the largest load
// factor (0.9) exceeds it by chance with negligible probability; a table that is really full
// costs each thread at most this many probes instead of a sweep of the whole table.
constexpr u64 kProbeLimit = 1ull << 15;
static __device__ __forceinline__ u64 probe_limit(u64 cap) {
  return cap < kProbeLimit ? cap : kProbeLimit;
}

// Adds count c to key's record.  Returns 1 if the key was new, 0 if it was present, -1 if the
// table is full (no room within the probe limit).  A new key and its count are installed by one 128-bit compare-and-swap of the
// whole (key, count) record; later additions are 64-bit atomic adds on the count.
static __device__ __forceinline__ int hash_add(Slot<u64> *slots, u64 cap, u64 key, u64 c) {
  u64 h = home_slot(key_hash(key), cap);
  for (u64 probe = 0, lim = probe_limit(cap); probe < lim; ++probe) {
    u64 cur = *reinterpret_cast<volatile u64 *>(&slots[h].key);  // 8-byte reads are atomic
    if (cur == key) {
      atomicAdd(&slots[h].cnt, c);
      return 0;
    }
    if (cur == 0) {
      u128 old = atomicCAS(reinterpret_cast<u128 *>(&slots[h]), (u128)0,
                           (u128)key | ((u128)c << 64));
      if (old == 0) return 1;
      if ((u64)old == key) {
        atomicAdd(&slots[h].cnt, c);
        return 0;
      }
    }
    h = next_slot(h, cap);
  }
  return -1;
}

static __device__ __forceinline__ int hash_add(Slot<u128> *slots, u64 cap, u128 key, u64 c) {
  u64 h = home_slot(key_hash(key), cap);
  for (u64 probe = 0, lim = probe_limit(cap); probe < lim; ++probe) {
    // a 16-byte plain read is not guaranteed to be single-copy atomic: always compare-and-swap
    u128 old = atomicCAS(&slots[h].key, (u128)0, key);
    if (old == 0) {
      atomicAdd(&slots[h].cnt, c);
      return 1;
    }
    if (old == key) {
      atomicAdd(&slots[h].cnt, c);
      return 0;
    }
    h = next_slot(h, cap);
  }
  return -1;
}

// find-or-insert; returns the slot index or -1 if the table is full (within the probe limit)
template <typename K>
__device__ __forceinline__ long long hash_claim(Slot<K> *slots, u64 cap, K key) {
  u64 h = home_slot(key_hash(key), cap);
  for (u64 probe = 0, lim = probe_limit(cap); probe < lim; ++probe) {
    K old = atomicCAS(&slots[h].key, (K)0, key);
    if (old == 0 || old == key) return (long long)h;
    h = next_slot(h, cap);
  }
  return -1;
}

// lookup in a table no thread is writing; -1 if absent
template <typename K>
__device__ __forceinline__ long long hash_find(const Slot<K> *slots, u64 cap, K key) {
  u64 h = home_slot(key_hash(key), cap);
  for (u64 probe = 0, lim = probe_limit(cap); probe < lim; ++probe) {
    K cur;
    u64 c;
    load_slot(slots, h, cur, c);
    if (cur == key) return (long long)h;
    if (cur == 0) return -1;
    h = next_slot(h, cap);
  }
  return -1;
}

// An earlier step of the run raised an error word (a planned room ran out, a wait gave up): the
// run is repeated or reported anyway, so the node kernels after it skip their work.  The block
// form is uniform over the block (one barrier), the warp form over the warp (lane 0's read).
__device__ __forceinline__ bool block_run_failed(const int *err) {
  return __syncthreads_or(*reinterpret_cast<const volatile int *>(err) != 0) != 0;
}
__device__ __forceinline__ bool warp_run_failed(const int *err) {
  int e = 0;
  if ((threadIdx.x & 31) == 0) e = *reinterpret_cast<const volatile int *>(err);
  return __shfl_sync(0xffffffffu, e, 0) != 0;
}

// ---- block reductions -------------------------------------------------------------------
template <int BLOCK>
__device__ __forceinline__ u64 block_sum(u64 v, u64 *s_red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) s_red[w] = v;
  __syncthreads();
  u64 t = 0;
  if (threadIdx.x == 0)
    for (int i = 0; i < BLOCK / 32; ++i) t += s_red[i];
  return t;  // valid in thread 0
}

// exclusive prefix of per-thread 64-bit values; s_off[BLOCK] receives the total
template <int BLOCK>
__device__ __forceinline__ void block_exclusive_scan(long long v, long long *s_off,
                                                     long long *s_warp) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  long long x = v;
  for (int o = 1; o < 32; o <<= 1) {
    long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[w] = x;
  __syncthreads();
  if (w == 0) {
    long long s = lane < BLOCK / 32 ? s_warp[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < BLOCK / 32) s_warp[lane] = s;  // inclusive warp totals
  }
  __syncthreads();
  long long before = (w ? s_warp[w - 1] : 0) + x - v;
  s_off[threadIdx.x] = before;
  if (threadIdx.x == BLOCK - 1) s_off[BLOCK] = before + v;
  __syncthreads();
}

// Exclusive scan of m 64-bit values in[0, m) into out[0, m) (in == out allowed) by ONE block of
// blockDim.x threads (a multiple of 32, at most 1024): chunks of blockDim.x values, each scanned
// with warp shuffles and one pass over the warp totals, carry the running sum forward; *total
// receives the sum of all m values.  Every thread of the block must call it.
__device__ __forceinline__ void block_scan_array(const u64 *in, u64 *out, u64 m, u64 *total) {
  __shared__ u64 s_w[32];
  __shared__ u64 s_carry;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (u64 base = 0; base < m; base += blockDim.x) {
    const u64 i = base + threadIdx.x;
    const u64 v = i < m ? in[i] : 0;
    u64 x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const u64 y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_w[w] = x;
    __syncthreads();
    if (w == 0) {  // inclusive scan of the warp totals
      u64 s = lane < nw ? s_w[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const u64 y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      if (lane < nw) s_w[lane] = s;
    }
    __syncthreads();
    const u64 carry = s_carry;
    if (i < m) out[i] = carry + (w ? s_w[w - 1] : 0) + x - v;
    __syncthreads();  // every thread has read s_carry and s_w
    if (threadIdx.x == 0) s_carry = carry + s_w[nw - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = s_carry;
}

// exclusive rank of a flag within the block (deterministic order), and the block's count
template <int BLOCK>
__device__ __forceinline__ int block_flag_rank(bool f, int *s_wc, int &total) {
  unsigned bal = __ballot_sync(0xffffffffu, f);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();  // previous readers of s_wc are done
  if (lane == 0) s_wc[w] = __popc(bal);
  __syncthreads();
  int before = 0;
  total = 0;
  for (int i = 0; i < BLOCK / 32; ++i) {
    int c = s_wc[i];
    before += i < w ? c : 0;
    total += c;
  }
  return before + __popc(bal & ((1u << lane) - 1u));
}

static __device__ __forceinline__ bool adjacent(const GraphDev &G, int a, int v) {
  int lo = G.row_ptr[a], hi = G.row_ptr[a + 1];
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    int c = __ldg(G.col + mid);
    if (c < v) lo = mid + 1;
    else if (c > v) hi = mid;
    else return true;
  }
  return false;
}


// Bucket of a key in a bucketed order: the top sp.hbits bits of a hash of the images of the
// first sp.hslots slots of sp.order (of the whole key when hslots is 0).
template <typename K>
__device__ __forceinline__ uint32_t sort_bucket(K key, const SortSpec &sp) {
  u64 h;
  if (sp.hslots > 0) {
    h = 0x9E3779B97F4A7C15ull;
#pragma unroll
    for (int j = 0; j < kMaxBag; ++j)
      if (j < sp.hslots) h = fmix64(h + (u64)(unsigned)key_slot(key, sp.L, sp.order[j]));
  } else {
    h = key_hash(key);
  }
  return (uint32_t)(h >> (64 - sp.hbits));
}

// The value records are sorted by (SortSpec): in a bucketed order the bucket first, then the
// G-vertices of slots order[0..), then, for a full order, the trial and the colour set.
template <typename SK, typename K>
__device__ __forceinline__ SK sort_key(K key, const SortSpec &sp) {
  SK s = 0;
  const int ns = sp.full ? sp.b : sp.nsl;
#pragma unroll
  for (int j = 0; j < kMaxBag; ++j)
    if (j < ns) s = (s << sp.L.nb) | (SK)(unsigned)key_slot(key, sp.L, sp.order[j]);
  if (sp.full) {
    if (sp.L.tb) s = (s << sp.L.tb) | (SK)(unsigned)key_trial(key, sp.L);
    s = (s << sp.L.k) | (SK)key_mask(key, sp.L);
  }
  if (sp.hbits) s |= (SK)sort_bucket(key, sp) << sp.bits;
  return s;
}

// Inverse of a full sort key (sp.full == 1): the packed key it was made from.
template <typename K>
__device__ __forceinline__ K unsort_key(K s, const SortSpec &sp) {
  const KeyLayout &L = sp.L;
  K key = s & (K)((1ull << L.k) - 1ull);
  s >>= L.k;
  if (L.tb) {
    key |= (s & (K)((1ull << L.tb) - 1ull)) << L.tpos;
    s >>= L.tb;
  }
  const K vmask = (K)((1ull << L.nb) - 1ull);
#pragma unroll
  for (int j = kMaxBag - 1; j >= 0; --j)
    if (j < sp.b) {
      key |= (s & vmask) << (L.k + sp.order[j] * L.nb);
      s >>= L.nb;
    }
  return key;
}

}  // namespace dev
}  // namespace cc
