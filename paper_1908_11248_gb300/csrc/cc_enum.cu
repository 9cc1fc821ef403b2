// Result reconstruction (Section 4) on the device.
//
// The paper's R(x, M) walks the nice decomposition from the root, asking each node's child
// table how a (mapping, colour set) pair arose, and glues the answers.  Here the same walk is
// breadth-first over the nodes in pre-order: a state is (trial, colour set C still to account
// for, stack of colour sets owed to the second children of enclosing joins, partial map Phi).
// Stepping a state through node x (next node in pre-order is x's first child, or, after a leaf,
// the second child of the innermost pending join):
//   forget u    : one state per vertex v with (Phi + u->v restricted to the child bag, C) in
//                 the child table; Phi(u) = v
//   introduce u : C loses the colour of Phi(u)
//   join        : one state per split C = C' | C'' with C' & C'' the bag's colours, (phi, C') in
//                 the first child's table and (phi, C'') in the second's; C'' is pushed
//   leaf        : pops the next colour set (or, at the last leaf, the state is a full embedding)
// Every state is extendable to at least one embedding, so the state count never exceeds the
// final number of embeddings.  The union over trials is then sorted lexicographically (LSD
// radix sort over the columns) and repeats are dropped.
//
// Membership "(t, phi, C) in D_y" is answered per table layout: a leaf table is indexed by
// (t, v); hashed tables are probed; sorted tables are binary-searched in their sort order; an
// introduce node, whose table need not be stored, is resolved by checking its rule (colour,
// degree filter, adjacency to the bag neighbours) and descending to its child.
#include <cstdint>

#include "cc_device.cuh"
#include "cc_internal.h"

namespace cc {
namespace {

using namespace dev;

__device__ __forceinline__ int colour_of(const GraphDev &G, int t, int v) {
  return G.colors[(u64)t * (u64)G.n + (u64)v];
}

template <typename SK, typename K>
__device__ bool sorted_contains(const Slot<K> *s, u64 count, const SortSpec &sp, K key) {
  const SK q = sort_key<SK>(key, sp);
  u64 lo = 0, hi = count;
  while (lo < hi) {
    const u64 mid = (lo + hi) >> 1;
    K km;
    u64 c;
    load_slot(s, mid, km, c);
    const SK sm = sort_key<SK>(km, sp);
    if (sm < q) lo = mid + 1;
    else hi = mid;
  }
  if (lo >= count) return false;
  K kl;
  u64 c;
  load_slot(s, lo, kl, c);
  return kl == key;
}

template <typename K>
__device__ bool member(const EnumArgs &a, int y, K key) {
  for (int depth = 0; depth < 2 * kMaxBag + 8; ++depth) {
    const EnumNode &nd = a.nodes[y];
    if (nd.type == 1) {  // introduce: check its rule, then look in the child
      const int v = key_slot(key, a.L, nd.p);
      const int cv = colour_of(a.G, key_trial(key, a.L), v);
      if (!((key_mask(key, a.L) >> cv) & 1u)) return false;
      if (nd.degF && a.G.row_ptr[v + 1] - a.G.row_ptr[v] < nd.degF) return false;
      if (a.G.allow && !((a.G.allow[v] >> nd.vertex) & 1u)) return false;
      const K k2 = key_remove(key, a.L, nd.p) & ~((K)1 << cv);
      for (int j = 0; j < nd.nnb; ++j)
        if (!adjacent(a.G, key_slot(k2, a.L, nd.nb_slot[j]), v)) return false;
      key = k2;
      y = nd.child0;
      continue;
    }
    const Slot<K> *s = reinterpret_cast<const Slot<K> *>(nd.slots);
    if (nd.type == 0) {  // leaf: record (t, v) sits at t * n + v
      const u64 idx = (u64)key_trial(key, a.L) * (u64)a.G.n + (u64)key_slot(key, a.L, 0);
      K kk;
      u64 c;
      load_slot(s, idx, kk, c);
      return kk == key;
    }
    if (nd.hashed) return hash_find(s, nd.cap, key) >= 0;
    if (nd.sorted)
      return nd.spec.bits + nd.spec.hbits <= 64
                 ? sorted_contains<u64>(s, nd.count, nd.spec, key)
                 : sorted_contains<u128>(s, nd.count, nd.spec, key);
    return false;
  }
  return false;
}

template <typename K>
__device__ __forceinline__ K key_of(const EnumArgs &a, const EnumNode &nd, int t, uint32_t C,
                                    const int *phi) {
  K key = (K)C;
  for (int s = 0; s < nd.b; ++s) key |= (K)(unsigned)phi[nd.bag[s]] << (a.L.k + s * a.L.nb);
  if (a.L.tb) key |= (K)(unsigned)t << a.L.tpos;
  return key;
}

// state layout: [0] trial, [1] colour set, [2] stack depth, [3, 3+D) stack, [3+D, 3+D+nF) Phi
template <typename K, int MODE>
__global__ void enum_step_kernel(EnumArgs a) {
  const EnumNode &nd = a.nodes[a.x];
  for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < a.n_in;
       i += (u64)gridDim.x * blockDim.x) {
    const int *st = a.in + i * (u64)a.R;
    const int t = st[0];
    const uint32_t C = (uint32_t)st[1];
    const int sp = st[2];
    const int *phi = st + 3 + a.D;
    u64 made = 0;
    const u64 base = MODE ? a.off[i] : 0;
    // emits a copy of this state with colour set C2, stack depth sp2 (push >= 0 pushes it
    // first) and Phi(u) = v when u >= 0
    auto emit = [&](uint32_t C2, int sp2, long long push, int u, int v) {
      if (MODE == 1) {
        int *o = a.out + (base + made) * (u64)a.R;
        for (int j = 0; j < a.R; ++j) o[j] = st[j];
        o[1] = (int)C2;
        if (push >= 0) o[3 + sp] = (int)push;
        o[2] = sp2;
        if (u >= 0) o[3 + a.D + u] = v;
      }
      ++made;
    };
    if (nd.type == 2) {  // forget u: every v completing (phi + u->v, C) in the child table
      const int u = nd.vertex;
      const EnumNode &ch = a.nodes[nd.child0];
      int best = INT_MAX, rs = 0;
      for (int j = 0; j < nd.nnb; ++j) {
        const int w = phi[nd.nb_slot[j]];  // F-vertex ids for forget nodes
        const int r0 = a.G.row_ptr[w], d = a.G.row_ptr[w + 1] - r0;
        if (d < best) {
          best = d;
          rs = r0;
        }
      }
      const int ncand = nd.nnb ? best : a.G.n;
      int work[kMaxBag + 32];
      for (int f = 0; f < a.nF; ++f) work[f] = phi[f];
      for (int j = 0; j < ncand; ++j) {
        const int v = nd.nnb ? __ldg(a.G.col + rs + j) : j;
        if (!((C >> colour_of(a.G, t, v)) & 1u)) continue;
        work[u] = v;
        if (member<K>(a, nd.child0, key_of<K>(a, ch, t, C, work))) emit(C, sp, -1, u, v);
      }
    } else if (nd.type == 1) {  // introduce u: its colour leaves C
      emit(C & ~(1u << colour_of(a.G, t, phi[nd.vertex])), sp, -1, -1, 0);
    } else if (nd.type == 3) {  // join: split the private colours between the children
      const EnumNode &y = a.nodes[nd.child0];
      const EnumNode &z = a.nodes[nd.child1];
      uint32_t bagc = 0;
      for (int s = 0; s < nd.b; ++s) bagc |= 1u << colour_of(a.G, t, phi[nd.bag[s]]);
      const uint32_t P = C & ~bagc;
      const int need = y.vstar - nd.b;
      int bit[32], nbits = 0;
      for (int q = 0; q < 32; ++q)
        if (P >> q & 1u) bit[nbits++] = q;
      if (need >= 0 && need <= nbits) {
        // subsets of P of size `need`, as index masks in increasing order (Gosper's hack)
        unsigned long long m = need ? ((1ull << need) - 1ull) : 0ull;
        const unsigned long long end = 1ull << nbits;
        while (true) {
          uint32_t A = 0;
          for (int q = 0; q < nbits; ++q)
            if (m >> q & 1ull) A |= 1u << bit[q];
          const uint32_t C1 = bagc | A, C2 = bagc | (P & ~A);
          if (member<K>(a, nd.child0, key_of<K>(a, y, t, C1, phi)) &&
              member<K>(a, nd.child1, key_of<K>(a, z, t, C2, phi)))
            emit(C1, sp + 1, (long long)C2, -1, 0);
          if (m == 0) break;
          const unsigned long long low = m & (~m + 1ull), r = m + low;
          m = (((r ^ m) >> 2) / low) | r;
          if (m >= end) break;
        }
      }
    } else {  // leaf: the next node is the second child of the innermost pending join
      if (sp > 0) emit((uint32_t)st[3 + sp - 1], sp - 1, -1, -1, 0);
      else emit(C, sp, -1, -1, 0);
    }
    if (MODE == 0) a.cnt[i] = (unsigned)made;
  }
}

// root states: one per root entry (t, C)
template <typename K>
__global__ void enum_init_kernel(EnumArgs a, const void *root, u64 bound, unsigned long long *n) {
  const Slot<K> *s = reinterpret_cast<const Slot<K> *>(root);
  for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < bound;
       i += (u64)gridDim.x * blockDim.x) {
    K key;
    u64 c;
    load_slot(s, i, key, c);
    if (key == 0) continue;
    const u64 pos = atomicAdd(n, 1ull);
    if (pos >= a.n_in) continue;  // capacity of the first state array
    int *o = a.out + pos * (u64)a.R;
    o[0] = key_trial(key, a.L);
    o[1] = (int)key_mask(key, a.L);
    o[2] = 0;
    for (int j = 3; j < a.R; ++j) o[j] = -1;
  }
}

// exclusive scan of n u32 values into u64 offsets; total at off[n]
__global__ void block_sums_kernel(const unsigned *v, u64 n, u64 per, u64 *sums) {
  const u64 lo = blockIdx.x * per, hi = min(n, lo + per);
  u64 s = 0;
  for (u64 i = lo + threadIdx.x; i < hi; i += blockDim.x) s += v[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __shared__ u64 w[32];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    u64 t = 0;
    for (unsigned q = 0; q < blockDim.x / 32; ++q) t += w[q];
    sums[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(1024) scan_small_kernel(u64 *v, int m, u64 *total) {
  block_scan_array(v, v, (u64)m, total);
}

// each block scans its range sequentially in chunks of blockDim (one block per range)
__global__ void block_scan_kernel(const unsigned *v, u64 n, u64 per, const u64 *sums, u64 *off) {
  __shared__ u64 s[1024];
  const u64 lo = blockIdx.x * per, hi = min(n, lo + per);
  u64 run = sums[blockIdx.x];
  for (u64 b = lo; b < hi; b += blockDim.x) {
    const u64 i = b + threadIdx.x;
    const u64 x = i < hi ? v[i] : 0;
    s[threadIdx.x] = x;
    __syncthreads();
    for (unsigned o = 1; o < blockDim.x; o <<= 1) {
      u64 y = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
      __syncthreads();
      s[threadIdx.x] += y;
      __syncthreads();
    }
    if (i < hi) off[i] = run + s[threadIdx.x] - x;
    run += s[blockDim.x - 1];
    __syncthreads();
  }
}

// ---- lexicographic sort of rows (LSD radix over columns, 8 bits per pass) -----------------
// perm holds row indices; a pass orders them stably by one byte of one column
__global__ void rows_hist_kernel(const int *rows, int nF, const unsigned *perm, u64 n, int col,
                                 int shift, u64 *hist) {
  __shared__ unsigned h[256];
  for (int d = threadIdx.x; d < 256; d += blockDim.x) h[d] = 0;
  __syncthreads();
  const u64 G = gridDim.x, chunk = (n + G - 1) / G;
  const u64 lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  for (u64 i = lo + threadIdx.x; i < hi; i += blockDim.x)
    atomicAdd(&h[((unsigned)rows[(u64)perm[i] * nF + col] >> shift) & 255u], 1u);
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[(u64)d * G + blockIdx.x] = h[d];
}

__global__ void __launch_bounds__(256) rows_row_scan_kernel(u64 *hist, int G) {
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

__global__ void __launch_bounds__(256) rows_digit_base_kernel(u64 *hist, int G) {
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

__global__ void __launch_bounds__(256) rows_scatter_kernel(const int *rows, int nF,
                                                           const unsigned *perm, u64 n, int col,
                                                           int shift, const u64 *off,
                                                           unsigned *out) {
  constexpr int W = 8;
  __shared__ unsigned s_wc[W][256];
  __shared__ unsigned s_run[256];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  s_run[tid] = 0;
  for (int x = 0; x < W; ++x) s_wc[x][tid] = 0;
  __syncthreads();
  const u64 G = gridDim.x, chunk = (n + G - 1) / G;
  const u64 lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  for (u64 base = lo; base < hi; base += 256) {
    const u64 i = base + tid;
    const bool valid = i < hi;
    const unsigned p = valid ? perm[i] : 0u;
    const int d = valid ? (int)(((unsigned)rows[(u64)p * nF + col] >> shift) & 255u) : 256 + lane;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && lane == __ffs(peers) - 1) s_wc[w][d] = __popc(peers);
    __syncthreads();
    unsigned acc = s_run[tid];
    for (int x = 0; x < W; ++x) {
      unsigned c = s_wc[x][tid];
      s_wc[x][tid] = acc;
      acc += c;
    }
    s_run[tid] = acc;
    __syncthreads();
    if (valid) out[off[(u64)d * G + blockIdx.x] + off[256 * G + d] + s_wc[w][d] + rank] = p;
    __syncthreads();
    for (int x = 0; x < W; ++x) s_wc[x][tid] = 0;
    __syncthreads();
  }
}

// each row (the images of F-vertices 0..nF-1) replaced by its vertex set in increasing order
__global__ void rows_canon_kernel(int *rows, int nF, u64 n) {
  for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < n;
       i += (u64)gridDim.x * blockDim.x) {
    int *r = rows + i * (u64)nF;
    for (int a = 1; a < nF; ++a) {  // insertion sort, n_F <= 32
      const int v = r[a];
      int b = a - 1;
      while (b >= 0 && r[b] > v) {
        r[b + 1] = r[b];
        --b;
      }
      r[b + 1] = v;
    }
  }
}

// rows of the final states, and the identity permutation
__global__ void rows_extract_kernel(const int *states, u64 n, int R, int D, int nF, int *rows,
                                    unsigned *perm) {
  for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < n;
       i += (u64)gridDim.x * blockDim.x) {
    for (int f = 0; f < nF; ++f) rows[i * nF + f] = states[i * (u64)R + 3 + D + f];
    perm[i] = (unsigned)i;
  }
}

// 1 where a row differs from its predecessor in sorted order
__global__ void rows_heads_kernel(const int *rows, int nF, const unsigned *perm, u64 n,
                                  unsigned *flag) {
  for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < n;
       i += (u64)gridDim.x * blockDim.x) {
    unsigned h = 1;
    if (i > 0) {
      const int *a = rows + (u64)perm[i] * nF, *b = rows + (u64)perm[i - 1] * nF;
      h = 0;
      for (int f = 0; f < nF; ++f) h |= a[f] != b[f];
    }
    flag[i] = h;
  }
}

__global__ void rows_gather_kernel(const int *rows, int nF, const unsigned *perm, u64 n,
                                   const unsigned *flag, const u64 *off, u64 limit, int *out) {
  for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < n;
       i += (u64)gridDim.x * blockDim.x) {
    if (!flag[i] || off[i] >= limit) continue;
    for (int f = 0; f < nF; ++f) out[off[i] * nF + f] = rows[(u64)perm[i] * nF + f];
  }
}

}  // namespace

int enum_grid(const DevInfo &d) { return d.sms * 8; }

int launch_enum_init(cudaStream_t s, const DevInfo &d, int kw, const EnumArgs &a,
                     const void *root, unsigned long long bound, unsigned long long *n) {
  if (kw == 1) enum_init_kernel<u64><<<d.sms, 256, 0, s>>>(a, root, bound, n);
  else enum_init_kernel<u128><<<d.sms, 256, 0, s>>>(a, root, bound, n);
  return (int)cudaGetLastError();
}

int launch_enum_step(cudaStream_t s, const DevInfo &d, int kw, int mode, const EnumArgs &a) {
  if (a.n_in == 0) return 0;
  const int grid = enum_grid(d);
  if (kw == 1) {
    if (mode == 0) enum_step_kernel<u64, 0><<<grid, 128, 0, s>>>(a);
    else enum_step_kernel<u64, 1><<<grid, 128, 0, s>>>(a);
  } else {
    if (mode == 0) enum_step_kernel<u128, 0><<<grid, 128, 0, s>>>(a);
    else enum_step_kernel<u128, 1><<<grid, 128, 0, s>>>(a);
  }
  return (int)cudaGetLastError();
}

size_t scan_scratch_words(const DevInfo &d) { return (size_t)d.sms * 2 + 2; }

int launch_scan_u32(cudaStream_t s, const DevInfo &d, const unsigned *v, unsigned long long n,
                    unsigned long long *off, unsigned long long *scratch) {
  // scratch: block sums (sms * 2 words) then the total
  const int nb = d.sms * 2;
  const u64 per = (n + nb - 1) / nb;
  u64 *sums = scratch, *total = scratch + nb;
  if (n == 0) return (int)cudaMemsetAsync(off, 0, sizeof(u64), s);
  block_sums_kernel<<<nb, 256, 0, s>>>(v, n, per, sums);
  scan_small_kernel<<<1, 1024, 0, s>>>(sums, nb, total);
  block_scan_kernel<<<nb, 1024, 0, s>>>(v, n, per, sums, off);
  cudaMemcpyAsync(off + n, total, sizeof(u64), cudaMemcpyDeviceToDevice, s);
  return (int)cudaGetLastError();
}

int launch_rows_canon(cudaStream_t s, const DevInfo &d, int *rows, int nF,
                      unsigned long long n) {
  if (n) rows_canon_kernel<<<d.sms * 4, 256, 0, s>>>(rows, nF, n);
  return (int)cudaGetLastError();
}

int launch_rows_extract(cudaStream_t s, const DevInfo &d, const int *states,
                        unsigned long long n, int R, int D, int nF, int *rows, unsigned *perm) {
  if (n) rows_extract_kernel<<<d.sms * 4, 256, 0, s>>>(states, n, R, D, nF, rows, perm);
  return (int)cudaGetLastError();
}

int launch_rows_sort(cudaStream_t s, const DevInfo &d, const int *rows, int nF, int nb,
                     unsigned long long n, unsigned *perm, unsigned *tmp, unsigned long long *hist,
                     unsigned **result) {
  const int G = d.sms * 2;
  unsigned *in = perm, *out = tmp;
  if (n > 1) {
    for (int col = nF - 1; col >= 0; --col)
      for (int shift = 0; shift < nb; shift += 8) {
        rows_hist_kernel<<<G, 256, 0, s>>>(rows, nF, in, n, col, shift, hist);
        rows_row_scan_kernel<<<256, 256, 0, s>>>(hist, G);
        rows_digit_base_kernel<<<1, 256, 0, s>>>(hist, G);
        rows_scatter_kernel<<<G, 256, 0, s>>>(rows, nF, in, n, col, shift, hist, out);
        unsigned *t = in;
        in = out;
        out = t;
      }
  }
  *result = in;
  return (int)cudaGetLastError();
}

int launch_rows_heads(cudaStream_t s, const DevInfo &d, const int *rows, int nF,
                      const unsigned *perm, unsigned long long n, unsigned *flag) {
  if (n) rows_heads_kernel<<<d.sms * 4, 256, 0, s>>>(rows, nF, perm, n, flag);
  return (int)cudaGetLastError();
}

int launch_rows_gather(cudaStream_t s, const DevInfo &d, const int *rows, int nF,
                       const unsigned *perm, unsigned long long n, const unsigned *flag,
                       const unsigned long long *off, unsigned long long limit, int *out) {
  if (n && limit) rows_gather_kernel<<<d.sms * 4, 256, 0, s>>>(rows, nF, perm, n, flag, off, limit, out);
  return (int)cudaGetLastError();
}

}  // namespace cc
