// Device kernels of the colour-coding dynamic programme (arXiv 1908.11248, Sections 2.1, 3.1).
//
// Tables are arrays of (packed key, uint64 count) records.  A key packs the trial index, the bag
// mapping phi (one G-vertex id per bag slot, slots in increasing F-vertex order, Section 3.2)
// and the colour set C (bit i = colour i, Section 3.2) into 64 or 128 bits, so that a whole key
// can be compared, hashed and claimed with one compare-and-swap.  All trials of a colouring live
// in the same tables, so one launch per node serves every trial.
//
// Node rules (Section 3.1, "Dynamic Programming Description"), extended from the Boolean table to
// counts of colourful embeddings mod 2^64:
//   leaf      (u)       : (phi = (v), C = {zeta(v)}) with count 1 for every host vertex v
//   introduce (u)       : (phi' + u->v, C' + zeta(v)) for every child entry and candidate v with
//                         zeta(v) not in C' and every edge of F[V_x] at u present in G
//   forget    (u)       : (phi' restricted to V_x, C), counts of equal results summed
//   join      (y, z)    : (phi, C' | C''), count c' * c'', whenever C' & C'' is exactly the colour
//                         set of phi's image; equal results summed
//   root                : a colourful copy exists iff the root table is nonempty; the count is
//                         the sum of the root counts
#include <algorithm>
#include <climits>
#include <cstdint>

#include "cc_device.cuh"
#include "cc_internal.h"

namespace cc {
namespace {

using namespace dev;

// ---- Philox4x32-10 (Salmon et al., SC'11) and the colouring of Section 2.1 -----------------
__global__ void color_kernel(uint8_t *out, int32_t n, int32_t trials, int32_t k, uint32_t key0,
                             uint32_t key1, uint32_t t0) {
  u64 total = (u64)n * (u64)trials;
  for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < total;
       i += (u64)gridDim.x * blockDim.x) {
    uint32_t t = (uint32_t)(i / (u64)n), v = (uint32_t)(i % (u64)n);
    uint32_t x0 = v, x1 = t0 + t, x2 = 0u, x3 = 0u;
    uint32_t k0 = key0, k1 = key1;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
      uint32_t lo0 = 0xD2511F53u * x0, hi0 = __umulhi(0xD2511F53u, x0);
      uint32_t lo1 = 0xCD9E8D57u * x2, hi1 = __umulhi(0xCD9E8D57u, x2);
      uint32_t n0 = hi1 ^ x1 ^ k0, n2 = hi0 ^ x3 ^ k1;
      x0 = n0;
      x1 = lo1;
      x2 = n2;
      x3 = lo0;
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    out[i] = (uint8_t)(((u64)x0 * (u64)(uint32_t)k) >> 32);
  }
}

// ---- leaf: one record per (trial, host vertex); filtered vertices leave an empty slot -------
template <typename K, int BLOCK>
__global__ void __launch_bounds__(BLOCK) leaf_kernel(LeafArgs a) {
  __shared__ u64 s_red[BLOCK / 32];
  Slot<K> *out = reinterpret_cast<Slot<K> *>(a.out.slots);
  const u64 n = (u64)a.G.n, total = n * (u64)a.trials;
  u64 made = 0;
  for (u64 i = blockIdx.x * (u64)BLOCK + threadIdx.x; i < total; i += (u64)gridDim.x * BLOCK) {
    int t = (int)(i / n), v = (int)(i % n);
    K key = 0;
    if ((a.degF == 0 || a.G.row_ptr[v + 1] - a.G.row_ptr[v] >= a.degF) &&
        (!a.G.allow || (a.G.allow[v] & a.ubit))) {
      int c = a.G.colors[i];
      key = ((K)1 << c) | ((K)(unsigned)v << a.L.k);
      if (a.L.tb) key |= (K)(unsigned)t << a.L.tpos;
      ++made;
    }
    store_slot(out, i, key, key ? 1ull : 0ull);
  }
  u64 s = block_sum<BLOCK>(made, s_red);
  if (threadIdx.x == 0 && s) atomicAdd(a.out.count, s);
}

// ---- introduce ---------------------------------------------------------------------------
// Each block takes BLOCK child entries at a time, lays their candidate lists (the adjacency of
// the bag neighbour whose image has the smallest degree, or all of V(G) when u has no bag
// neighbour) end to end with a block prefix sum, and walks the concatenation with all threads,
// so a hub's list is shared by the whole block.
//   MODE 0: count the valid extensions per block (blk_count[blockIdx.x])
//   MODE 1: write them densely at blk_base[blockIdx.x] + block-local rank (deterministic order)
//   MODE 2: project out slot q (the parent forget) and add into the hashed output
//
// The grouped variant expects the child table sorted by the images of u's bag neighbours
// (tuple_sort), so entries that differ only in trial, colour set or other slots come in runs.
// In every tile the first entry of each run computes the run's candidate list once (adjacency
// to every bag neighbour's image and the degree filter) into shared memory, and each entry of
// the run then only tests its own colour set.  A tile whose lists overflow the shared buffer is
// processed entry by entry instead.

template <typename K, int BLOCK, int VCAP>
struct IntroSmem {
  long long off[BLOCK + 1];
  long long warp[BLOCK / 32];
  K key[BLOCK];
  u64 cnt[BLOCK];
  u64 tup[BLOCK];
  int rs[BLOCK];
  int anc[BLOCK];
  int head[BLOCK];
  int hvc[BLOCK];
  int hst[BLOCK];
  int wc[BLOCK / 32];
  int hmax[BLOCK / 32];
  u64 red[BLOCK / 32];
  u64 newbase;
  int vbuf[VCAP];
};

// chunked append: a block reserves output slots kAppendChunk at a time from a global cursor
constexpr u64 kAppendChunk = 2048;

struct EmitState {
  u64 produced = 0, fresh = 0, examined = 0, cursor = 0;
  u64 chunk_base = 0, chunk_fill = kAppendChunk;  // block-uniform
  bool full = false;
};

template <typename K, int MODE, int BLOCK, typename S>
__device__ __forceinline__ void emit(const IntroArgs &a, S &sm, EmitState &st, bool valid, K okey,
                                     u64 oc) {
  if (MODE == 0) {
    st.produced += valid;
  } else if (MODE == 1) {
    int tot;
    const int rank = block_flag_rank<BLOCK>(valid, sm.wc, tot);
    u64 pos = 0;
    if (a.cursor) {  // chunked append (planned capacities): one atomic per chunk
      const u64 idx = st.chunk_fill + (u64)rank;
      const bool spill = st.chunk_fill + (u64)tot > kAppendChunk;  // block-uniform
      if (spill) {
        if (threadIdx.x == 0) sm.newbase = atomicAdd(a.cursor, kAppendChunk);
        __syncthreads();
      }
      const u64 nb = spill ? sm.newbase : 0;
      pos = idx < kAppendChunk ? st.chunk_base + idx : nb + (idx - kAppendChunk);
      if (spill) {
        st.chunk_base = nb;
        st.chunk_fill = st.chunk_fill + (u64)tot - kAppendChunk;
      } else {
        st.chunk_fill += (u64)tot;
      }
    } else {  // exact bases from the count pass
      pos = st.cursor + (u64)rank;
      st.cursor += (u64)tot;
    }
    if (valid) {
      ++st.produced;
      if (pos < a.out.cap)
        store_slot(reinterpret_cast<Slot<K> *>(a.out.slots), pos,
                   a.proj_q >= 0 ? key_remove(okey, a.L, a.proj_q) : okey, oc);
      else st.full = true;
    }
  } else if (valid) {
    ++st.produced;
    if (!st.full) {  // a full table takes no more probes: the run is repeated
      int r = hash_add(reinterpret_cast<Slot<K> *>(a.out.slots), a.out.cap,
                       key_remove(okey, a.L, a.q), oc);
      if (r > 0) ++st.fresh;
      if (r < 0) st.full = true;
    }
  }
}

// index e of the entry whose candidate range [off[e], off[e+1]) holds j
template <int BLOCK>
__device__ __forceinline__ int owner(const long long *off, long long j) {
  int lo = 0, hi = BLOCK - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= j) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// entry by entry: every candidate of every entry is checked in full (the tile's entries are in
// sm.key / sm.cnt)
template <typename K, int MODE, int BLOCK, typename S>
__device__ __forceinline__ void plain_tile(const IntroArgs &a, S &sm, EmitState &st) {
  const K key = sm.key[threadIdx.x];
  long long nc = 0;
  int rs = -1, anc = -1;
  if (key != 0) {
    if (a.nnb == 0) {
      nc = a.G.n;
    } else {
      int best = INT_MAX;
      for (int j = 0; j < a.nnb; ++j) {
        int w = key_slot(key, a.L, a.nb_slot[j]);
        int r0 = a.G.row_ptr[w], d = a.G.row_ptr[w + 1] - r0;
        if (d < best) {
          best = d;
          rs = r0;
          anc = j;
        }
      }
      nc = best;
    }
  }
  sm.rs[threadIdx.x] = rs;
  sm.anc[threadIdx.x] = anc;
  block_exclusive_scan<BLOCK>(nc, sm.off, sm.warp);
  const long long total = sm.off[BLOCK];
  if (threadIdx.x == 0) st.examined += (u64)total;  // block-uniform: count once
  for (long long j0 = 0; j0 < total; j0 += BLOCK) {
    const long long j = j0 + threadIdx.x;
    bool valid = false;
    K okey = 0;
    u64 oc = 0;
    if (j < total) {
      const int e = owner<BLOCK>(sm.off, j);
      const long long r = j - sm.off[e];
      const int v = sm.rs[e] >= 0 ? __ldg(a.G.col + sm.rs[e] + r) : (int)r;
      const K ekey = sm.key[e];
      const int t = key_trial(ekey, a.L);
      const int cv = a.G.colors[(u64)t * (u64)a.G.n + (u64)v];
      valid = !((key_mask(ekey, a.L) >> cv) & 1u);
      if (valid && a.degF) valid = a.G.deg8[v] >= a.degF;
      if (valid && a.G.allow) valid = (a.G.allow[v] & a.ubit) != 0;
      if (valid) {
        const int an = sm.anc[e];
        for (int q = 0; q < a.nnb && valid; ++q)
          if (q != an) valid = adjacent(a.G, key_slot(ekey, a.L, a.nb_slot[q]), v);
      }
      if (valid) {
        okey = key_insert(ekey, a.L, a.p, v) | ((K)1 << cv);
        oc = sm.cnt[e];
      }
    }
    emit<K, MODE, BLOCK>(a, sm, st, valid, okey, oc);
  }
}

template <typename K>
__device__ __forceinline__ u64 nb_tuple(K key, const IntroArgs &a) {
  u64 t = 0;
  for (int j = 0; j < a.nnb; ++j) t = (t << a.L.nb) | (u64)key_slot(key, a.L, a.nb_slot[j]);
  return t;
}

// candidate lists shared by runs of equal bag-neighbour images; false if they overflowed
template <typename K, int MODE, int BLOCK, int VCAP, typename S>
__device__ __forceinline__ bool grouped_tile(const IntroArgs &a, S &sm, EmitState &st) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const K key = sm.key[tid];
  const u64 tup = key != 0 ? nb_tuple(key, a) : ~0ull;
  sm.tup[tid] = tup;
  __syncthreads();
  const bool head = key != 0 && (tid == 0 || sm.tup[tid - 1] != tup);
  // the run head of every entry: inclusive max-scan of (head ? tid : -1)
  int h = head ? tid : -1;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, h, o);
    if (lane >= o) h = max(h, y);
  }
  if (lane == 31) sm.hmax[w] = h;
  long long nc = 0;
  int rs = -1, anc = -1;
  if (head) {
    int best = INT_MAX;
    for (int j = 0; j < a.nnb; ++j) {
      int wv = key_slot(key, a.L, a.nb_slot[j]);
      int r0 = a.G.row_ptr[wv], d = a.G.row_ptr[wv + 1] - r0;
      if (d < best) {
        best = d;
        rs = r0;
        anc = j;
      }
    }
    nc = best;
  }
  sm.rs[tid] = rs;
  sm.anc[tid] = anc;
  sm.hvc[tid] = 0;
  __syncthreads();
  for (int i = 0; i < w; ++i) h = max(h, sm.hmax[i]);
  sm.head[tid] = h;
  block_exclusive_scan<BLOCK>(nc, sm.off, sm.warp);
  const long long total = sm.off[BLOCK];
  if (threadIdx.x == 0) st.examined += (u64)total;  // block-uniform: count once
  int vtotal = 0;
  for (long long j0 = 0; j0 < total; j0 += BLOCK) {
    const long long j = j0 + tid;
    bool ok = false;
    int e = 0, v = 0;
    if (j < total) {
      e = owner<BLOCK>(sm.off, j);
      v = __ldg(a.G.col + sm.rs[e] + (j - sm.off[e]));
      ok = (a.degF == 0 || a.G.deg8[v] >= a.degF) &&
           (!a.G.allow || (a.G.allow[v] & a.ubit));
      if (ok) {
        const K ekey = sm.key[e];
        const int an = sm.anc[e];
        for (int q = 0; q < a.nnb && ok; ++q)
          if (q != an) ok = adjacent(a.G, key_slot(ekey, a.L, a.nb_slot[q]), v);
      }
    }
    int tot;
    const int rank = block_flag_rank<BLOCK>(ok, sm.wc, tot);
    if (ok) {
      const int pos = vtotal + rank;
      if (pos < VCAP) sm.vbuf[pos] = v;
      atomicAdd(&sm.hvc[e], 1);
    }
    vtotal += tot;
  }
  if (vtotal > VCAP) return false;  // uniform across the block
  __syncthreads();
  // each head's list starts after the lists of the heads before it (stream order)
  block_exclusive_scan<BLOCK>(sm.hvc[tid], sm.off, sm.warp);
  sm.hst[tid] = (int)sm.off[tid];
  __syncthreads();
  const int hd = sm.head[tid];
  const long long mine = key != 0 ? sm.hvc[hd] : 0;
  block_exclusive_scan<BLOCK>(mine, sm.off, sm.warp);
  const long long total2 = sm.off[BLOCK];
  for (long long j0 = 0; j0 < total2; j0 += BLOCK) {
    const long long j = j0 + tid;
    bool valid = false;
    K okey = 0;
    u64 oc = 0;
    if (j < total2) {
      const int e = owner<BLOCK>(sm.off, j);
      const int v = sm.vbuf[sm.hst[sm.head[e]] + (int)(j - sm.off[e])];
      const K ekey = sm.key[e];
      const int t = key_trial(ekey, a.L);
      const int cv = a.G.colors[(u64)t * (u64)a.G.n + (u64)v];
      valid = !((key_mask(ekey, a.L) >> cv) & 1u);
      if (valid) {
        okey = key_insert(ekey, a.L, a.p, v) | ((K)1 << cv);
        oc = sm.cnt[e];
      }
    }
    emit<K, MODE, BLOCK>(a, sm, st, valid, okey, oc);
  }
  return true;
}

template <typename K, int MODE, int BLOCK, int GROUPED>
__global__ void __launch_bounds__(BLOCK) intro_kernel(IntroArgs a, u64 *blk_count,
                                                      const u64 *blk_base) {
  constexpr int VCAP = GROUPED ? 2048 : 1;
  __shared__ IntroSmem<K, BLOCK, VCAP> sm;
  const Slot<K> *in = reinterpret_cast<const Slot<K> *>(a.in.slots);
  const u64 bound = block_run_failed(a.err) ? 0 : table_bound<K>(a.in);
  EmitState st;
  if (MODE == 1) st.cursor = blk_base[blockIdx.x];
  for (u64 base = (u64)blockIdx.x * BLOCK; base < bound; base += (u64)gridDim.x * BLOCK) {
    const u64 i = base + threadIdx.x;
    K key = 0;
    u64 c = 0;
    if (i < bound) load_slot(in, i, key, c);
    sm.key[threadIdx.x] = key;
    sm.cnt[threadIdx.x] = c;
    if (!GROUPED || !grouped_tile<K, MODE, BLOCK, VCAP>(a, sm, st))
      plain_tile<K, MODE, BLOCK>(a, sm, st);
    __syncthreads();  // the next tile overwrites the shared arrays
  }
  if (MODE == 1 && a.cursor && st.chunk_fill < kAppendChunk) {
    // the unused tail of this block's last chunk becomes holes
    Slot<K> *out = reinterpret_cast<Slot<K> *>(a.out.slots);
    for (u64 j = st.chunk_fill + threadIdx.x; j < kAppendChunk; j += BLOCK)
      if (st.chunk_base + j < a.out.cap) store_slot(out, st.chunk_base + j, (K)0, 0ull);
  }
  if (st.full) atomicOr(a.err, kErrOverflow);
  if (MODE == 0) {
    u64 s = block_sum<BLOCK>(st.produced, sm.red);
    u64 x = block_sum<BLOCK>(st.examined, sm.red);
    if (threadIdx.x == 0) {
      blk_count[blockIdx.x] = s;
      if (x) atomicAdd(a.cand, x);
    }
  } else if (MODE == 1) {
    if (a.valid) {
      u64 s = block_sum<BLOCK>(st.produced, sm.red);
      if (threadIdx.x == 0 && s) atomicAdd(a.valid, s);
    }
    if (a.cand) {
      u64 x = block_sum<BLOCK>(st.examined, sm.red);
      if (threadIdx.x == 0 && x) atomicAdd(a.cand, x);
    }
  } else if (MODE == 2) {
    if (a.cand) {
      u64 x = block_sum<BLOCK>(st.examined, sm.red);
      if (threadIdx.x == 0 && x) atomicAdd(a.cand, x);
    }
    u64 s = block_sum<BLOCK>(st.produced, sm.red);
    if (threadIdx.x == 0 && s) atomicAdd(a.valid, s);
    u64 f = block_sum<BLOCK>(st.fresh, sm.red);
    if (threadIdx.x == 0 && f) atomicAdd(a.out.count, f);
  }
}

// ---- introduce, warp by warp (planned capacities, vertex with at most one bag neighbour) ------
// Each warp takes 32 child entries at a time, scans their candidate counts with shuffles and
// walks the concatenated candidate lists 32 at a time; a lane finds the entry owning its
// candidate by a five-step binary search over the warp's prefix sums.  Outputs go to per-warp
// chunks of the output (MODE 1) or into the parent forget's hash table (MODE 2).  No block
// barrier is involved.
// A warp reserves a.chunk output slots at a time (a power of two in [32, 256], chosen by the
// planner from the table's planned size so that the holes left in the warps' last chunks stay a
// small part of the table).
// Each lane first builds its entry's output key with the new vertex's field left zero (the
// vertex inserted at slot p and, when the entries are written projected, the parent forget's
// slot removed), so that a candidate only ORs in its vertex and its colour bit.

__device__ __forceinline__ u64 shfl_key(u64 v, int src) {
  return __shfl_sync(0xffffffffu, v, src);
}
__device__ __forceinline__ u128 shfl_key(u128 v, int src) {
  const u64 lo = __shfl_sync(0xffffffffu, (u64)v, src);
  const u64 hi = __shfl_sync(0xffffffffu, (u64)(v >> 64), src);
  return ((u128)hi << 64) | (u128)lo;
}

// The output key of an introduce for a child entry `key` with the new vertex's field zero: the
// vertex inserted at slot p, then slot q removed when the parent forget's projection is applied
// (q < 0: none; q == p: the new vertex is forgotten at once, so only its colour enters the key).
template <typename K>
__device__ __forceinline__ K intro_base(K key, const KeyLayout &L, int p, int q) {
  if (q == p) return key;
  const K b = key_insert(key, L, p, 0);
  return q >= 0 ? key_remove(b, L, q) : b;
}
// bit position of the new vertex in that output key, -1 when it is forgotten at once
__device__ __forceinline__ int intro_vshift(const KeyLayout &L, int p, int q) {
  if (q == p) return -1;
  return L.k + (q >= 0 && q < p ? p - 1 : p) * L.nb;
}
// the output key of candidate v with colour cv
template <typename K>
__device__ __forceinline__ K intro_out(K base, int vsh, int v, int cv) {
  return base | (vsh >= 0 ? (K)(unsigned)v << vsh : (K)0) | ((K)1 << cv);
}

// Appends the warp's valid outputs (already projected) in chunks (MODE 1) or adds them into the
// hashed output (MODE 2).
template <typename K, int MODE>
__device__ __forceinline__ void warp_emit(const IntroArgs &a, bool valid, K okey, u64 oc,
                                          int lane, unsigned lt, u64 &cbase, u64 &cfill,
                                          u64 &produced, u64 &fresh, bool &full) {
  Slot<K> *out = reinterpret_cast<Slot<K> *>(a.out.slots);
  if (MODE == 1) {
    const u64 chunk = a.chunk;
    const unsigned bal = __ballot_sync(0xffffffffu, valid);
    if (!bal) return;
    const u64 tot = __popc(bal);
    const u64 idx = cfill + __popc(bal & lt);
    u64 nb = 0;
    const bool spill = cfill + tot > chunk;
    if (spill) {
      if (lane == 0) nb = atomicAdd(a.cursor, chunk);
      nb = __shfl_sync(0xffffffffu, nb, 0);
    }
    if (valid) {
      const u64 pos = idx < chunk ? cbase + idx : nb + (idx - chunk);
      ++produced;
      if (pos < a.out.cap) store_slot(out, pos, okey, oc);
      else full = true;
    }
    if (spill) {
      cbase = nb;
      cfill = cfill + tot - chunk;
    } else {
      cfill += tot;
    }
  } else if (valid) {
    ++produced;
    if (!full) {
      const int r = hash_add(out, a.out.cap, okey, oc);
      if (r > 0) ++fresh;
      if (r < 0) full = true;
    }
  }
}

// I: integer type of candidate positions within a window (int when 32 * n < 2^31).
template <typename K, int MODE, typename I>
__global__ void __launch_bounds__(256, 4) intro_warp_kernel(IntroArgs a) {
  const Slot<K> *in = reinterpret_cast<const Slot<K> *>(a.in.slots);
  Slot<K> *out = reinterpret_cast<Slot<K> *>(a.out.slots);
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const u64 warps = (u64)gridDim.x * (blockDim.x / 32);
  const u64 wid = (u64)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const u64 bound = warp_run_failed(a.err) ? 0 : table_bound<K>(a.in);
  const int q = MODE == 2 ? a.q : a.proj_q;
  const int vsh = intro_vshift(a.L, a.p, q);
  const u64 n = (u64)a.G.n;
  const u64 chunk = a.chunk;
  u64 cbase = 0, cfill = chunk;  // warp-uniform chunk state
  u64 produced = 0, fresh = 0, examined = 0;
  bool full = false;
  // the next window's records are loaded while the current one is expanded
  K nkey = 0;
  u64 nc_ = 0;
  if (wid * 32 + lane < bound) load_slot(in, wid * 32 + lane, nkey, nc_);
  for (u64 base = wid * 32; base < bound; base += warps * 32) {
    const K key = nkey;
    const u64 c = nc_;
    {
      const u64 i2 = base + warps * 32 + lane;
      nkey = 0;
      nc_ = 0;
      if (i2 < bound) load_slot(in, i2, nkey, nc_);
    }
    I nc = 0;
    int rs = 0;
    K ob = 0;          // output key without the new vertex
    uint32_t cm = 0;   // colour set
    u64 crow = 0;      // first colour of the entry's trial
    if (key != 0) {
      if (a.nnb == 0) {
        nc = (I)a.G.n;
      } else {
        const int w = key_slot(key, a.L, a.nb_slot[0]);
        rs = a.G.row_ptr[w];
        nc = a.G.row_ptr[w + 1] - rs;
      }
      ob = intro_base(key, a.L, a.p, q);
      cm = key_mask(key, a.L);
      crow = (u64)key_trial(key, a.L) * n;
    }
    I incl = nc;
    for (int o = 1; o < 32; o <<= 1) {
      const I y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const I excl = incl - nc;
    const I total = __shfl_sync(0xffffffffu, incl, 31);
    if (lane == 0) examined += (u64)total;
    for (I j0 = 0; j0 < total; j0 += 32) {
      const I j = j0 + lane;
      // owner: smallest lane o with incl[o] > j
      int lo = 0, hi = 31;
#pragma unroll
      for (int step = 0; step < 5; ++step) {
        const int mid = (lo + hi) >> 1;
        const I v = __shfl_sync(0xffffffffu, incl, mid);
        if (v > j) hi = mid;
        else lo = mid + 1;
      }
      const int o = lo;
      const K eb = shfl_key(ob, o);
      const u64 ec = __shfl_sync(0xffffffffu, c, o);
      const int ers = __shfl_sync(0xffffffffu, rs, o);
      const I eexcl = __shfl_sync(0xffffffffu, excl, o);
      const uint32_t ecm = __shfl_sync(0xffffffffu, cm, o);
      const u64 ecrow = __shfl_sync(0xffffffffu, crow, o);
      bool valid = false;
      K okey = 0;
      if (j < total) {
        const I r = j - eexcl;
        const int v = a.nnb ? __ldg(a.G.col + ers + r) : (int)r;
        const int cv = a.G.colors[ecrow + (u64)v];
        valid = !((ecm >> cv) & 1u);
        if (valid && a.degF) valid = a.G.deg8[v] >= a.degF;
        if (valid && a.G.allow) valid = (a.G.allow[v] & a.ubit) != 0;
        if (valid) okey = intro_out(eb, vsh, v, cv);
      }
      warp_emit<K, MODE>(a, valid, okey, ec, lane, lt, cbase, cfill, produced, fresh, full);
    }
  }
  if (MODE == 1 && cfill < chunk)  // the unused tail of the warp's last chunk: holes
    for (u64 j = cfill + lane; j < chunk; j += 32)
      if (cbase + j < a.out.cap) store_slot(out, cbase + j, (K)0, 0ull);
  if (full) atomicOr(a.err, kErrOverflow);
  for (int o = 16; o > 0; o >>= 1) {
    produced += __shfl_down_sync(0xffffffffu, produced, o);
    fresh += __shfl_down_sync(0xffffffffu, fresh, o);
  }
  if (lane == 0) {
    if (a.valid && produced) atomicAdd(a.valid, produced);
    if (MODE == 2 && fresh) atomicAdd(a.out.count, fresh);
    if (a.cand && examined) atomicAdd(a.cand, examined);
  }
}

// ---- grouped introduce, warp by warp (planned capacities) -----------------------------------
// The child comes in runs of equal images of u's bag neighbours (sorted or clustered by them).
// Each warp takes a contiguous range of windows of 32 consecutive entries.  The first entry of
// every run in a window leads: the warp walks the lead's anchor list 32 candidates at a time,
// keeps those adjacent to every bag neighbour's image (and passing the degree filter and the
// allowed mappings) in a per-warp buffer, and every entry of the run then only tests its own
// colour set against that list.  A window that begins inside the run the previous window ended
// in takes that run's list as it is: two buffers alternate, the one holding the carried list
// being left alone while the window's new lists are built in the other.  A window whose new
// lists do not fit a buffer is processed entry by entry.
constexpr int kGroupCap = 256;  // candidate-list buffer per warp (two of them)

// Per host vertex w (one thread) and every trial: counts of w's neighbours by colour, four
// colours to a 64-bit word (16-bit fields), for the chained introduce's counted entries.
__global__ void __launch_bounds__(256) nb_colour_hist_kernel(GraphDev G, int trials, int degF,
                                                             uint32_t ubit, u64 *hist,
                                                             u64 *cand) {
  u64 seen = 0;
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < G.n; w += gridDim.x * blockDim.x) {
    const int r0 = G.row_ptr[w], r1 = G.row_ptr[w + 1];
    for (int t = 0; t < trials; ++t) {
      const uint8_t *col = G.colors + (u64)t * (u64)G.n;
      u64 h0 = 0, h1 = 0, h2 = 0, h3 = 0;
      for (int r = r0; r < r1; ++r) {
        const int v = __ldg(G.col + r);
        if (degF && G.deg8[v] < degF) continue;
        if (G.allow && !(G.allow[v] & ubit)) continue;
        const int c = col[v];
        const u64 one = 1ull << (16 * (c & 3));
        h0 += (c >> 2) == 0 ? one : 0;
        h1 += (c >> 2) == 1 ? one : 0;
        h2 += (c >> 2) == 2 ? one : 0;
        h3 += (c >> 2) == 3 ? one : 0;
      }
      u64 *o = hist + ((u64)t * (u64)G.n + (u64)w) * 4;
      reinterpret_cast<ulonglong2 *>(o)[0] = make_ulonglong2(h0, h1);
      reinterpret_cast<ulonglong2 *>(o)[1] = make_ulonglong2(h2, h3);
    }
    seen += (u64)(r1 - r0) * (u64)trials;
  }
  for (int o = 16; o > 0; o >>= 1) seen += __shfl_down_sync(0xffffffffu, seen, o);
  if ((threadIdx.x & 31) == 0 && seen) atomicAdd(cand, seen);
}

// x1's extensions of an entry with colour set cm from the colour counts of its anchor image
__device__ __forceinline__ u64 hist_count(const u64 *h, uint32_t cm, int k) {
  const ulonglong2 a = __ldg(reinterpret_cast<const ulonglong2 *>(h));
  const ulonglong2 b = __ldg(reinterpret_cast<const ulonglong2 *>(h) + 1);
  const u64 w[4] = {a.x, a.y, b.x, b.y};
  u64 sum = 0;
#pragma unroll
  for (int c = 0; c < 16; ++c)
    if (c < k && !((cm >> c) & 1u)) sum += (w[c >> 2] >> (16 * (c & 3))) & 0xFFFFull;
  return sum;
}

// x1's candidates of one y entry (chained introduce): the adjacency list of the bag neighbour
// image with the fewest neighbours
template <typename K>
__device__ __forceinline__ void chain_anchor(const IntroArgs &a, K key, int &rs, int &d,
                                             int &anc) {
  rs = 0;
  d = 0;
  anc = 0;
  if (key == 0) return;
  int best = INT_MAX;
  for (int j = 0; j < a.c_nnb; ++j) {
    const int w = key_slot(key, a.L, a.c_nb_slot[j]);
    const int r0 = a.G.row_ptr[w], dd = a.G.row_ptr[w + 1] - r0;
    if (dd < best) {
      best = dd;
      rs = r0;
      anc = j;
    }
  }
  d = best;
}

// x1's rule for candidate v of y entry `key` (colour set cm): colour not in the set, degree
// filter, allowed mapping, adjacent to every bag neighbour image but the anchor's
template <typename K>
__device__ __forceinline__ bool chain_ok(const IntroArgs &a, K key, uint32_t cm, int v, int cv,
                                         int anc) {
  if ((cm >> cv) & 1u) return false;
  if (a.c_degF && a.G.deg8[v] < a.c_degF) return false;
  if (a.G.allow && !(a.G.allow[v] & a.c_ubit)) return false;
  for (int j = 0; j < a.c_nnb; ++j)
    if (j != anc && !adjacent(a.G, key_slot(key, a.L, a.c_nb_slot[j]), v)) return false;
  return true;
}

template <typename K, int MODE, bool CHAIN = false>
__global__ void __launch_bounds__(256, CHAIN ? 3 : 4) intro_group_warp_kernel(IntroArgs a) {
  __shared__ int s_buf[8][2 * kGroupCap];
  const Slot<K> *in = reinterpret_cast<const Slot<K> *>(a.in.slots);
  Slot<K> *out = reinterpret_cast<Slot<K> *>(a.out.slots);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  int *bufs = s_buf[wib];
  const u64 warps = (u64)gridDim.x * (blockDim.x / 32);
  const u64 wid = (u64)blockIdx.x * (blockDim.x / 32) + wib;
  const u64 bound = warp_run_failed(a.err) ? 0 : table_bound<K>(a.in);
  const u64 nwin = (bound + 31) / 32, per = (nwin + warps - 1) / warps;
  const u64 w0 = min(nwin, wid * per), w1 = min(nwin, w0 + per);
  const int q = MODE == 2 ? a.q : a.proj_q;
  const int vsh = intro_vshift(a.L, a.p, q);
  const u64 n = (u64)a.G.n;
  const u64 chunk = a.chunk;
  u64 cbase = 0, cfill = chunk;
  u64 produced = 0, fresh = 0, examined = 0, produced1 = 0;
  bool full = false;
  // the run the previous window ended in (warp-uniform): its tuple and its list
  // bufs[cb * kGroupCap + cs .. + cl) (cl < 0: none)
  u64 ctup = ~0ull;
  int cb = 0, cs = 0, cl = -1;
  // the next window's records are loaded while the current one is processed
  K nkey = 0;
  u64 nc_ = 0;
  if (w0 < w1 && w0 * 32 + lane < bound) load_slot(in, w0 * 32 + lane, nkey, nc_);
  for (u64 win = w0; win < w1; ++win) {
    const K key = nkey;
    const u64 c = nc_;
    {
      const u64 i2 = (win + 1) * 32 + lane;
      nkey = 0;
      nc_ = 0;
      if (win + 1 < w1 && i2 < bound) load_slot(in, i2, nkey, nc_);
    }
    const u64 tup = key != 0 ? nb_tuple(key, a) : ~0ull;
    const u64 up = __shfl_up_sync(0xffffffffu, tup, 1);
    const bool lead = key != 0 && (lane == 0 ? (cl < 0 || tup != ctup) : up != tup);
    const unsigned leads = __ballot_sync(0xffffffffu, lead);
    const int nbuf = cb ^ 1;  // the new lists go where the carried one is not
    int *nb_base = bufs + nbuf * kGroupCap;
    // candidate lists of the window's new runs, one after the other in the new buffer
    int lstart = 0, llen = 0;  // held by lead lanes
    int used = 0;              // warp-uniform
    bool overflow = false;
    for (unsigned rest = leads; rest; rest &= rest - 1) {
      const int l = __ffs(rest) - 1;
      const K lkey = shfl_key(key, l);
      int best = INT_MAX, rs = 0, anc = 0;
      for (int j = 0; j < a.nnb; ++j) {
        const int w = key_slot(lkey, a.L, a.nb_slot[j]);
        const int r0 = a.G.row_ptr[w], d = a.G.row_ptr[w + 1] - r0;
        if (d < best) {
          best = d;
          rs = r0;
          anc = j;
        }
      }
      if (lane == 0) examined += (u64)best;
      // two bag neighbours, the other one of degree <= 32: its adjacency list is held one entry
      // a lane and every candidate is compared against it by shuffles instead of a binary
      // search in global memory
      int ob = 0, od = 33;
      if (a.nnb == 2) {
        const int w2 = key_slot(lkey, a.L, a.nb_slot[1 - anc]);
        ob = a.G.row_ptr[w2];
        od = a.G.row_ptr[w2 + 1] - ob;
      }
      const bool inreg = od <= 32;
      const int bv = (inreg && lane < od) ? __ldg(a.G.col + ob + lane) : -1;
      const int start = used;
      for (int j0 = 0; j0 < best; j0 += 32) {
        const int j = j0 + lane;
        bool ok = false;
        int v = 0;
        if (j < best) {
          v = __ldg(a.G.col + rs + j);
          ok = (a.degF == 0 || a.G.deg8[v] >= a.degF) &&
               (!a.G.allow || (a.G.allow[v] & a.ubit));
          if (!inreg)
            for (int qq = 0; qq < a.nnb && ok; ++qq)
              if (qq != anc) ok = adjacent(a.G, key_slot(lkey, a.L, a.nb_slot[qq]), v);
        }
        if (inreg) {  // every lane takes part in the shuffles
          bool hit = false;
          for (int qq = 0; qq < od; ++qq) hit |= __shfl_sync(0xffffffffu, bv, qq) == v;
          ok = ok && hit;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, ok);
        const int pos = used + __popc(bal & lt);
        if (ok && pos < kGroupCap) nb_base[pos] = v;
        used += __popc(bal);
      }
      if (used > kGroupCap) overflow = true;
      if (lane == l) {
        lstart = start;
        llen = used - start;
      }
    }
    __syncwarp();
    if (!overflow) {
      // each entry takes the list of the last lead at or before it; entries before the first
      // lead continue the carried run
      const unsigned mine = leads & (lt | (1u << lane));
      const int from = mine ? 31 - __clz(mine) : 0;
      // every lane takes part in both shuffles (a full-mask shuffle in a branch is undefined)
      int s0 = __shfl_sync(0xffffffffu, lstart, from);
      int n0 = __shfl_sync(0xffffffffu, llen, from);
      const int *lst = nb_base;
      if (!mine) {
        lst = bufs + cb * kGroupCap;
        s0 = cs;
        n0 = cl < 0 ? 0 : cl;
      }
      if (key == 0) n0 = 0;
      int nmax = n0;
      for (int o = 16; o > 0; o >>= 1) nmax = max(nmax, __shfl_xor_sync(0xffffffffu, nmax, o));
      const uint32_t cm = key_mask(key, a.L);
      const u64 crow = key != 0 ? (u64)key_trial(key, a.L) * n : 0;
      if constexpr (CHAIN) {
        // every x1 extension (entry, v1) of this entry is counted; those with a nonempty u2 list
        // are extended by it at once
        int r1, d1, anc1;
        chain_anchor(a, key, r1, d1, anc1);
        // u2 candidates of the run whose colour is not in this entry's set: only those can
        // extend one of its x1 entries (the set only grows with v1's colour)
        int nv = 0;
        for (int r = 0; r < nmax; ++r)
          if (r < n0 && !((cm >> a.G.colors[crow + (u64)lst[s0 + r]]) & 1u)) ++nv;
        if (a.c_hist && key != 0 && nv == 0) {
          // none: the entry's x1 extensions are only counted, from the colour counts of its
          // anchor image
          const u64 w1 = (u64)key_slot(key, a.L, a.c_nb_slot[anc1]);
          produced1 += hist_count(a.c_hist + ((u64)key_trial(key, a.L) * n + w1) * 4, cm,
                                  a.L.k);
          d1 = 0;
        }
        if (nv == 0) n0 = 0;  // no pair can be valid
        int dmax = d1, dsum = d1;
        for (int o = 16; o > 0; o >>= 1) {
          dmax = max(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
          dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
        }
        if (lane == 0) examined += (u64)dsum;
        const K b1 = key != 0 ? intro_base(key, a.L, a.c_p, -1) : (K)0;
        const int vsh1 = intro_vshift(a.L, a.c_p, -1);
        for (int j = 0; j < dmax; ++j) {
          bool ok1 = false;
          int v1 = 0, cv1 = 0;
          if (j < d1) {
            v1 = __ldg(a.G.col + r1 + j);
            cv1 = a.G.colors[crow + (u64)v1];
            ok1 = chain_ok(a, key, cm, v1, cv1, anc1);
          }
          produced1 += ok1 ? 1u : 0u;
          const bool pair = ok1 && n0 > 0;
          if (!__any_sync(0xffffffffu, pair)) continue;
          int m = pair ? n0 : 0;
          for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
          const uint32_t cm1 = cm | (1u << cv1);
          const K k1 = pair ? intro_out(b1, vsh1, v1, cv1) : (K)0;
          for (int r = 0; r < m; ++r) {
            bool valid = false;
            K okey = 0;
            if (pair && r < n0) {
              const int v = lst[s0 + r];
              const int cv = a.G.colors[crow + (u64)v];
              valid = !((cm1 >> cv) & 1u);
              if (valid) okey = intro_out(intro_base(k1, a.L, a.p, q), vsh, v, cv);
            }
            warp_emit<K, MODE>(a, valid, okey, c, lane, lt, cbase, cfill, produced, fresh, full);
          }
        }
        nmax = 0;  // the plain loop below has nothing left to do
      }
      for (int r = 0; r < nmax; ++r) {
        bool valid = false;
        K okey = 0;
        if (r < n0) {
          const int v = lst[s0 + r];
          const int cv = a.G.colors[crow + (u64)v];
          valid = !((cm >> cv) & 1u);
          // most candidates of a closing step clash in colour: the output key is built only
          // for the valid ones
          if (valid) okey = intro_out(intro_base(key, a.L, a.p, q), vsh, v, cv);
        }
        warp_emit<K, MODE>(a, valid, okey, c, lane, lt, cbase, cfill, produced, fresh, full);
      }
      // carry the run of the window's last entry: a new one, or the carried one continued
      if (leads) {
        const int l = 31 - __clz(leads);
        cb = nbuf;
        cs = __shfl_sync(0xffffffffu, lstart, l);
        cl = __shfl_sync(0xffffffffu, llen, l);
      }
      ctup = __shfl_sync(0xffffffffu, tup, 31);
      if (ctup == ~0ull) cl = -1;
    } else {  // entry by entry, every check in full
      int best = INT_MAX, rs = 0, anc = 0;
      if (key != 0)
        for (int j = 0; j < a.nnb; ++j) {
          const int w = key_slot(key, a.L, a.nb_slot[j]);
          const int r0 = a.G.row_ptr[w], d = a.G.row_ptr[w + 1] - r0;
          if (d < best) {
            best = d;
            rs = r0;
            anc = j;
          }
        }
      const int nc = key != 0 ? best : 0;
      int nmax = nc;
      for (int o = 16; o > 0; o >>= 1) nmax = max(nmax, __shfl_xor_sync(0xffffffffu, nmax, o));
      const uint32_t cm = key_mask(key, a.L);
      const u64 crow = key != 0 ? (u64)key_trial(key, a.L) * n : 0;
      if constexpr (CHAIN) {
        // every x1 extension, then every u2 candidate of the entry's own anchor list with all
        // of x2's checks
        int r1, d1, anc1;
        chain_anchor(a, key, r1, d1, anc1);
        int dmax = d1, dsum = d1, nsum = 0;
        for (int o = 16; o > 0; o >>= 1) {
          dmax = max(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
          dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
        }
        const K b1 = key != 0 ? intro_base(key, a.L, a.c_p, -1) : (K)0;
        const int vsh1 = intro_vshift(a.L, a.c_p, -1);
        for (int j = 0; j < dmax; ++j) {
          bool ok1 = false;
          int v1 = 0, cv1 = 0;
          if (j < d1) {
            v1 = __ldg(a.G.col + r1 + j);
            cv1 = a.G.colors[crow + (u64)v1];
            ok1 = chain_ok(a, key, cm, v1, cv1, anc1);
          }
          produced1 += ok1 ? 1u : 0u;
          const bool pair = ok1 && nc > 0;
          if (!__any_sync(0xffffffffu, pair)) continue;
          nsum += pair ? nc : 0;
          const uint32_t cm1 = cm | (1u << cv1);
          const K k1 = pair ? intro_out(b1, vsh1, v1, cv1) : (K)0;
          for (int r = 0; r < nmax; ++r) {
            bool valid = false;
            K okey = 0;
            if (pair && r < nc) {
              const int v = __ldg(a.G.col + rs + r);
              const int cv = a.G.colors[crow + (u64)v];
              valid = !((cm1 >> cv) & 1u);
              if (valid && a.degF) valid = a.G.deg8[v] >= a.degF;
              if (valid && a.G.allow) valid = (a.G.allow[v] & a.ubit) != 0;
              for (int qq = 0; qq < a.nnb && valid; ++qq)
                if (qq != anc) valid = adjacent(a.G, key_slot(key, a.L, a.nb_slot[qq]), v);
              if (valid) okey = intro_out(intro_base(k1, a.L, a.p, q), vsh, v, cv);
            }
            warp_emit<K, MODE>(a, valid, okey, c, lane, lt, cbase, cfill, produced, fresh, full);
          }
        }
        for (int o = 16; o > 0; o >>= 1) nsum += __shfl_xor_sync(0xffffffffu, nsum, o);
        if (lane == 0) examined += (u64)(dsum + nsum);
        nmax = 0;
      }
      for (int j = 0; j < nmax; ++j) {
        bool valid = false;
        K okey = 0;
        if (j < nc) {
          const int v = __ldg(a.G.col + rs + j);
          const int cv = a.G.colors[crow + (u64)v];
          valid = !((cm >> cv) & 1u);
          if (valid && a.degF) valid = a.G.deg8[v] >= a.degF;
          if (valid && a.G.allow) valid = (a.G.allow[v] & a.ubit) != 0;
          for (int qq = 0; qq < a.nnb && valid; ++qq)
            if (qq != anc) valid = adjacent(a.G, key_slot(key, a.L, a.nb_slot[qq]), v);
          if (valid) okey = intro_out(intro_base(key, a.L, a.p, q), vsh, v, cv);
        }
        warp_emit<K, MODE>(a, valid, okey, c, lane, lt, cbase, cfill, produced, fresh, full);
      }
      cl = -1;  // no list to carry
    }
    __syncwarp();  // the buffers are rewritten by the next window
  }
  if (MODE == 1 && cfill < chunk)
    for (u64 j = cfill + lane; j < chunk; j += 32)
      if (cbase + j < a.out.cap) store_slot(out, cbase + j, (K)0, 0ull);
  if (full) atomicOr(a.err, kErrOverflow);
  for (int o = 16; o > 0; o >>= 1) {
    produced += __shfl_down_sync(0xffffffffu, produced, o);
    fresh += __shfl_down_sync(0xffffffffu, fresh, o);
    if (CHAIN) produced1 += __shfl_down_sync(0xffffffffu, produced1, o);
  }
  if (lane == 0) {
    if (CHAIN && a.c_valid && produced1) atomicAdd(a.c_valid, produced1);
    if (a.valid && produced) atomicAdd(a.valid, produced);
    if (MODE == 2 && fresh) atomicAdd(a.out.count, fresh);
    if (a.cand && examined) atomicAdd(a.cand, examined);
  }
}

// A wait of the kind the sort passes' look-back makes, on a word that nothing sets: each
// thread polls it at most `polls` times, then records a timeout in the error word and returns.
__global__ void wait_probe_kernel(const u64 *flag, unsigned polls, int *err) {
  for (unsigned i = 0; i < polls; ++i)
    if (__ldcv(flag) != 0) return;
  atomicOr(err, kErrTimeout);
}

// exclusive scan of the per-block counts (one block of 1024 threads); bases and the grand total
__global__ void __launch_bounds__(1024) scan_blocks_kernel(const u64 *cnt, int nblk, u64 *base,
                                                           u64 *total) {
  block_scan_array(cnt, base, (u64)nblk, total);
}

// ---- forget: project out slot q and aggregate into a hash table ---------------------------
template <typename K, int BLOCK>
__global__ void __launch_bounds__(BLOCK) forget_kernel(ForgetArgs a) {
  __shared__ u64 s_red[BLOCK / 32];
  const Slot<K> *in = reinterpret_cast<const Slot<K> *>(a.in.slots);
  Slot<K> *out = reinterpret_cast<Slot<K> *>(a.out.slots);
  const u64 bound = block_run_failed(a.err) ? 0 : table_bound<K>(a.in);
  const u64 ocap = a.out.cap;
  u64 fresh = 0;
  bool full = false;
  for (u64 i = blockIdx.x * (u64)BLOCK + threadIdx.x; i < bound; i += (u64)gridDim.x * BLOCK) {
    K key;
    u64 c;
    load_slot(in, i, key, c);
    if (key == 0 || full) continue;
    int r = hash_add(out, ocap, key_remove(key, a.L, a.q), c);
    if (r > 0) ++fresh;
    if (r < 0) full = true;
  }
  if (full) atomicOr(a.err, kErrOverflow);
  u64 f = block_sum<BLOCK>(fresh, s_red);
  if (threadIdx.x == 0 && f) atomicAdd(a.out.count, f);
}

// ---- join: chain the build child's entries by bag mapping, then probe with the other -------
template <typename K>
__device__ __forceinline__ K phi_key(K key, const KeyLayout &L) {
  // colour set cleared; bit 0 marks an occupied index slot
  return (key & ~(K)((1ull << L.k) - 1ull)) | (K)1;
}

template <typename K, int BLOCK>
__global__ void __launch_bounds__(BLOCK) join_build_kernel(JoinArgs a) {
  const Slot<K> *bt = reinterpret_cast<const Slot<K> *>(a.build.slots);
  Slot<K> *idx = reinterpret_cast<Slot<K> *>(a.index);
  const u64 bound = block_run_failed(a.err) ? 0 : table_bound<K>(a.build);
  const u64 icap = a.index_cap;
  bool full = false;
  for (u64 i = blockIdx.x * (u64)BLOCK + threadIdx.x; i < bound; i += (u64)gridDim.x * BLOCK) {
    K key;
    u64 c;
    load_slot(bt, i, key, c);
    if (key == 0 || full) continue;
    long long h = hash_claim(idx, icap, phi_key(key, a.L));
    if (h < 0) {
      full = true;
      continue;
    }
    a.next[i] = atomicExch(&idx[h].cnt, (u64)(i + 1));
  }
  if (full) atomicOr(a.err, kErrOverflow);
}

template <typename K, int MODE, int BLOCK>
__global__ void __launch_bounds__(BLOCK) join_probe_kernel(JoinArgs a) {
  __shared__ u64 s_red[BLOCK / 32];
  const Slot<K> *bt = reinterpret_cast<const Slot<K> *>(a.build.slots);
  const Slot<K> *pt = reinterpret_cast<const Slot<K> *>(a.probe.slots);
  const Slot<K> *idx = reinterpret_cast<const Slot<K> *>(a.index);
  Slot<K> *out = reinterpret_cast<Slot<K> *>(a.out.slots);
  const u64 bound = block_run_failed(a.err) ? 0 : table_bound<K>(a.probe);
  const u64 icap = a.index_cap, ocap = a.out.cap;
  const K cmask = (K)((1ull << a.L.k) - 1ull);
  u64 pairs = 0, fresh = 0;
  bool full = false;
  for (u64 i = blockIdx.x * (u64)BLOCK + threadIdx.x; i < bound; i += (u64)gridDim.x * BLOCK) {
    K key;
    u64 c2;
    load_slot(pt, i, key, c2);
    if (key == 0) continue;
    long long h = hash_find(idx, icap, phi_key(key, a.L));
    if (h < 0) continue;
    const int t = key_trial(key, a.L);
    uint32_t bagc = 0;
    for (int s = 0; s < a.b; ++s)
      bagc |= 1u << a.G.colors[(u64)t * (u64)a.G.n + (u64)key_slot(key, a.L, s)];
    const uint32_t C2 = key_mask(key, a.L);
    K hk;
    u64 e;
    load_slot(idx, (u64)h, hk, e);
    while (e) {
      K k1;
      u64 c1;
      load_slot(bt, e - 1, k1, c1);
      const uint32_t C1 = key_mask(k1, a.L);
      if ((C1 & C2) == bagc) {
        ++pairs;
        if (MODE == 1 && !full) {
          int r = hash_add(out, ocap, (key & ~cmask) | (K)(C1 | C2), c1 * c2);
          if (r > 0) ++fresh;
          if (r < 0) full = true;
        }
      }
      e = a.next[e - 1];
    }
  }
  if (full) atomicOr(a.err, kErrOverflow);
  if (MODE == 0) {
    u64 s = block_sum<BLOCK>(pairs, s_red);
    if (threadIdx.x == 0 && s) atomicAdd(a.pairs, s);
  } else {
    u64 f = block_sum<BLOCK>(fresh, s_red);
    if (threadIdx.x == 0 && f) atomicAdd(a.out.count, f);
  }
}

// ---- root: per trial, exists = root table nonempty, count = sum of its counts --------------
template <typename K>
__global__ void root_kernel(RootArgs a) {
  const Slot<K> *in = reinterpret_cast<const Slot<K> *>(a.in.slots);
  const u64 bound = table_bound<K>(a.in);
  for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < bound;
       i += (u64)gridDim.x * blockDim.x) {
    K key;
    u64 c;
    load_slot(in, i, key, c);
    if (key == 0) continue;
    int t = key_trial(key, a.L);
    a.exists[t] = 1u;
    atomicAdd(&a.count[t], c);
  }
}

// ---- unpack a table for inspection ----------------------------------------------------------
template <typename K>
__global__ void unpack_kernel(KeyLayout L, TableDesc t, int b, int32_t *trial, int32_t *phi,
                              uint32_t *mask, u64 *cnt, u64 *n_out, u64 cap) {
  const Slot<K> *in = reinterpret_cast<const Slot<K> *>(t.slots);
  const u64 bound = table_bound<K>(t);
  for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < bound;
       i += (u64)gridDim.x * blockDim.x) {
    K key;
    u64 c;
    load_slot(in, i, key, c);
    if (key == 0) continue;
    u64 pos = atomicAdd(n_out, 1ull);
    if (pos >= cap) continue;
    trial[pos] = key_trial(key, L);
    for (int s = 0; s < b; ++s) phi[pos * b + s] = key_slot(key, L, s);
    mask[pos] = key_mask(key, L);
    cnt[pos] = c;
  }
}

int grid_for(const DevInfo &d, int block) {
  int per_sm = d.blocks_per_sm * 256 / block;
  if (per_sm < 1) per_sm = 1;
  return d.sms * per_sm;
}

template <typename K, int BLOCK>
int intro_dispatch(cudaStream_t s, const DevInfo &d, int mode, int grouped, const IntroArgs &a,
                   u64 *blk_count, const u64 *blk_base) {
  int grid = grid_for(d, BLOCK);
#define CC_LAUNCH(M, G) intro_kernel<K, M, BLOCK, G><<<grid, BLOCK, 0, s>>>(a, blk_count, blk_base)
  if (grouped) {
    if (mode == 0) CC_LAUNCH(0, 1);
    else if (mode == 1) CC_LAUNCH(1, 1);
    else CC_LAUNCH(2, 1);
  } else {
    if (mode == 0) CC_LAUNCH(0, 0);
    else if (mode == 1) CC_LAUNCH(1, 0);
    else CC_LAUNCH(2, 0);
  }
#undef CC_LAUNCH
  return (int)cudaGetLastError();
}

}  // namespace

size_t slot_bytes(int kw) { return kw == 1 ? sizeof(Slot<u64>) : sizeof(Slot<u128>); }
size_t index_slot_bytes(int kw) { return slot_bytes(kw); }

int intro_grid(const DevInfo &d, int block) { return grid_for(d, block); }

int launch_color(cudaStream_t s, const DevInfo &d, uint8_t *out, int32_t n, int32_t trials,
                 int32_t k, uint64_t seed, int32_t t0) {
  if ((u64)n * (u64)trials == 0) return 0;
  color_kernel<<<d.sms * 4, 256, 0, s>>>(out, n, trials, k, (uint32_t)seed,
                                         (uint32_t)(seed >> 32), (uint32_t)t0);
  return (int)cudaGetLastError();
}

int launch_leaf(cudaStream_t s, const DevInfo &d, int kw, const LeafArgs &a) {
  if ((u64)a.G.n * (u64)a.trials == 0) return 0;
  int grid = grid_for(d, 256);
  if (kw == 1) leaf_kernel<u64, 256><<<grid, 256, 0, s>>>(a);
  else leaf_kernel<u128, 256><<<grid, 256, 0, s>>>(a);
  return (int)cudaGetLastError();
}

int launch_intro_blk(cudaStream_t s, const DevInfo &d, int kw, int mode, int grouped,
                     int block, const IntroArgs &a, u64 *blk) {
  int grid = grid_for(d, block);
  u64 *cnt = blk, *base = blk + grid, *total = blk + 2 * grid;
  int r = 0;
#define CC_INTRO(B)                                                                \
  if (block == B) {                                                                \
    r = kw == 1 ? intro_dispatch<u64, B>(s, d, mode, grouped, a, cnt, base)        \
                : intro_dispatch<u128, B>(s, d, mode, grouped, a, cnt, base);      \
  } else
  CC_INTRO(128) CC_INTRO(256) CC_INTRO(512) { return (int)cudaErrorInvalidValue; }
#undef CC_INTRO
  if (r) return r;
  if (mode == 0) {
    scan_blocks_kernel<<<1, 1024, 0, s>>>(cnt, grid, base, total);
    r = (int)cudaGetLastError();
  }
  return r;
}

__global__ void deg8_kernel(const int32_t *row_ptr, int32_t n, uint8_t *deg8) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const int d = row_ptr[v + 1] - row_ptr[v];
    deg8[v] = (uint8_t)(d < 255 ? d : 255);
  }
}

// Allowed-mapping masks of one slice of a run: pattern vertex u (bit ubit) may be mapped only to
// host vertices v with v mod slices == slice; every other bit comes from base (all ones when
// base is null).
__global__ void slice_mask_kernel(const uint32_t *base, int32_t n, uint32_t ubit, int32_t slices,
                                  int32_t slice, uint32_t *out) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const uint32_t m = base ? base[v] : 0xFFFFFFFFu;
    out[v] = v % slices == slice ? m : (m & ~ubit);
  }
}

int launch_slice_mask(cudaStream_t s, const DevInfo &d, const uint32_t *base, int32_t n,
                      uint32_t ubit, int32_t slices, int32_t slice, uint32_t *out) {
  if (n > 0) slice_mask_kernel<<<d.sms * 4, 256, 0, s>>>(base, n, ubit, slices, slice, out);
  return (int)cudaGetLastError();
}

int launch_deg8(cudaStream_t s, const DevInfo &d, const int32_t *row_ptr, int32_t n,
                uint8_t *deg8) {
  if (n > 0) deg8_kernel<<<d.sms * 4, 256, 0, s>>>(row_ptr, n, deg8);
  return (int)cudaGetLastError();
}

int launch_intro_group_warp(cudaStream_t s, const DevInfo &d, int kw, int mode,
                            const IntroArgs &a) {
  const int grid = d.sms * d.blocks_per_sm;
  if (kw == 1) {
    if (mode == 1) intro_group_warp_kernel<u64, 1><<<grid, 256, 0, s>>>(a);
    else intro_group_warp_kernel<u64, 2><<<grid, 256, 0, s>>>(a);
  } else {
    if (mode == 1) intro_group_warp_kernel<u128, 1><<<grid, 256, 0, s>>>(a);
    else intro_group_warp_kernel<u128, 2><<<grid, 256, 0, s>>>(a);
  }
  return (int)cudaGetLastError();
}

int launch_nb_colour_hist(cudaStream_t s, const DevInfo &d, const GraphDev &G, int trials,
                          int degF, uint32_t ubit, unsigned long long *hist,
                          unsigned long long *cand) {
  const int grid = std::max(1, std::min(d.sms * 8, (G.n + 255) / 256));
  nb_colour_hist_kernel<<<grid, 256, 0, s>>>(G, trials, degF, ubit, hist, cand);
  return (int)cudaGetLastError();
}

int launch_intro_chain(cudaStream_t s, const DevInfo &d, int kw, const IntroArgs &a) {
  const int grid = d.sms * d.blocks_per_sm;
  if (kw == 1) intro_group_warp_kernel<u64, 1, true><<<grid, 256, 0, s>>>(a);
  else intro_group_warp_kernel<u128, 1, true><<<grid, 256, 0, s>>>(a);
  return (int)cudaGetLastError();
}

int launch_intro_warp(cudaStream_t s, const DevInfo &d, int kw, int mode, const IntroArgs &a) {
  const int grid = d.sms * d.blocks_per_sm;
  // a window's candidates number at most 32 * n (no bag neighbour: every vertex per entry)
  const bool narrow = (long long)a.G.n * 32 < (1ll << 31);
#define CC_IW(K, M)                                                         \
  if (narrow) intro_warp_kernel<K, M, int><<<grid, 256, 0, s>>>(a);         \
  else intro_warp_kernel<K, M, long long><<<grid, 256, 0, s>>>(a)
  if (kw == 1) {
    if (mode == 1) {
      CC_IW(u64, 1);
    } else {
      CC_IW(u64, 2);
    }
  } else {
    if (mode == 1) {
      CC_IW(u128, 1);
    } else {
      CC_IW(u128, 2);
    }
  }
#undef CC_IW
  return (int)cudaGetLastError();
}

int launch_wait_probe(cudaStream_t s, const unsigned long long *flag, unsigned polls,
                      int *err) {
  wait_probe_kernel<<<1, 32, 0, s>>>(flag, polls, err);
  return (int)cudaGetLastError();
}

int launch_forget(cudaStream_t s, const DevInfo &d, int kw, int block, const ForgetArgs &a) {
  (void)block;
  int grid = grid_for(d, 256);
  if (kw == 1) forget_kernel<u64, 256><<<grid, 256, 0, s>>>(a);
  else forget_kernel<u128, 256><<<grid, 256, 0, s>>>(a);
  return (int)cudaGetLastError();
}

int launch_join(cudaStream_t s, const DevInfo &d, int kw, int phase, int block,
                const JoinArgs &a) {
  (void)block;
  int grid = grid_for(d, 256);
  if (phase == 0) {
    if (kw == 1) join_build_kernel<u64, 256><<<grid, 256, 0, s>>>(a);
    else join_build_kernel<u128, 256><<<grid, 256, 0, s>>>(a);
  } else if (phase == 1) {
    if (kw == 1) join_probe_kernel<u64, 0, 256><<<grid, 256, 0, s>>>(a);
    else join_probe_kernel<u128, 0, 256><<<grid, 256, 0, s>>>(a);
  } else {
    if (kw == 1) join_probe_kernel<u64, 1, 256><<<grid, 256, 0, s>>>(a);
    else join_probe_kernel<u128, 1, 256><<<grid, 256, 0, s>>>(a);
  }
  return (int)cudaGetLastError();
}

int launch_root(cudaStream_t s, const DevInfo &d, int kw, const RootArgs &a) {
  int grid = d.sms;
  if (kw == 1) root_kernel<u64><<<grid, 256, 0, s>>>(a);
  else root_kernel<u128><<<grid, 256, 0, s>>>(a);
  return (int)cudaGetLastError();
}

int launch_unpack(cudaStream_t s, const DevInfo &d, int kw, const KeyLayout &L,
                  const TableDesc &t, int b, unsigned long long cap, int32_t *trial,
                  int32_t *phi, uint32_t *mask, unsigned long long *cnt,
                  unsigned long long *n_out) {
  int grid = d.sms * 2;
  if (kw == 1)
    unpack_kernel<u64><<<grid, 256, 0, s>>>(L, t, b, trial, phi, mask, cnt, n_out, cap);
  else
    unpack_kernel<u128><<<grid, 256, 0, s>>>(L, t, b, trial, phi, mask, cnt, n_out, cap);
  return (int)cudaGetLastError();
}

}  // namespace cc
