// Internal types shared by the host runtime (cc_host.cpp) and the device kernels
// (cc_kernels.cu).  Not part of the public ABI (include/cc.h).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace cc {

constexpr int kMaxBag = 8;  // largest bag |V_x| handled by the kernels (treewidth <= 7)

// device error word bits (OR-ed by kernels, read by the host after a run)
constexpr int kErrOverflow = 1;   // an append table or hash table ran out of slots
constexpr int kErrProbe = 2;      // a hash probe sequence wrapped the whole table
constexpr int kErrTimeout = 4;    // a bounded device wait gave up

// Bit layout of a packed table key (64 or 128 bits):
//   bits [0, k)                 colour set C (bit i = colour i)
//   bits [k + i*nb, k+(i+1)*nb) G-vertex of bag slot i (slots in increasing F-vertex order)
//   bits [tpos, tpos + tb)      trial index
// A valid key never has C == 0, so the all-zero key marks an empty hash slot.
struct KeyLayout {
  int k;     // colours
  int nb;    // bits per vertex id
  int tpos;  // first trial bit = k + max_bag * nb
  int tb;    // trial bits
};

// One table: `slots` holds Slot64 (key, count) or Slot128 (key, count, pad) records.  A dense
// table holds its entries in [0, min(*count, cap)); a hashed table has holes (key 0) anywhere
// in [0, cap) and *count is its number of distinct keys.
struct TableDesc {
  void *slots;
  unsigned long long cap;
  unsigned long long *count;  // device counter
  int hashed;
};

struct GraphDev {
  const int32_t *row_ptr;  // n + 1
  const int32_t *col;      // row_ptr[n]
  const uint8_t *colors;   // trials * n
  int32_t n;
  const uint8_t *deg8;     // min(degree, 255) per vertex (pattern degrees are below 32)
  const uint32_t *allow;   // per vertex, bit u: F-vertex u may be mapped there (null: any)
};

struct LeafArgs {
  GraphDev G;
  KeyLayout L;
  int trials;
  int degF;  // minimum host degree (degree filter), 0 = off
  TableDesc out;
  int *err;
  uint32_t ubit;  // 1 << (the leaf's F-vertex), tested against G.allow
};

struct IntroArgs {
  GraphDev G;
  KeyLayout L;
  TableDesc in;
  int b_in;                  // child bag size
  int p;                     // slot of the introduced vertex u in the new bag
  int nnb;                   // bag neighbours of u in F[V_x]
  int nb_slot[kMaxBag];      // their slots in the child bag
  int degF;                  // minimum host degree of u's image (0 = off)
  TableDesc out;             // dense (mode 1) or hashed (mode 2) output
  int q;                     // mode 2: slot (in the new bag) of the vertex the parent forgets
  int proj_q;                // mode 1: if >= 0, write keys with this slot removed
  unsigned long long *cursor;  // mode 1: non-null = chunked append from this cursor (no bases)
  unsigned long long *valid; // modes 1, 2: number of introduce entries produced (if non-null)
  unsigned long long *cand;  // mode 0: number of candidate vertices examined
  int *err;
  uint32_t ubit;             // 1 << u, tested against G.allow
  unsigned chunk;            // warp kernels, mode 1: slots a warp reserves at a time (32..256)
  // chained introduce (launch_intro_chain): the input is the child y of a lower introduce x1
  // whose table is not stored; the fields above describe the upper introduce x2 (its bag
  // neighbours' slots counted in y's bag), these the lower one
  int c_p;                   // slot of x1's vertex in x1's bag
  int c_nnb;                 // bag neighbours of x1's vertex (at least one)
  int c_nb_slot[kMaxBag];    // their slots in y's bag
  int c_degF;                // degree filter of x1's vertex (0 = off)
  uint32_t c_ubit;           // 1 << x1's vertex, tested against G.allow
  unsigned long long *c_valid;  // number of x1 entries (|D_x1|), counted, not written
  // non-null (x1 with one bag neighbour, k <= 16): per trial t and host vertex w, sixteen
  // 16-bit counts of w's neighbours of each colour that pass x1's degree filter and allowed
  // mappings (launch_nb_colour_hist); an entry whose run has no x2 candidate then counts its x1
  // extensions from them instead of walking w's adjacency
  const unsigned long long *c_hist;
};

struct ForgetArgs {
  KeyLayout L;
  TableDesc in;
  int b_in;
  int q;  // slot of the forgotten vertex in the child bag
  TableDesc out;
  int *err;
};

struct JoinArgs {
  GraphDev G;
  KeyLayout L;
  TableDesc build;      // child whose entries are chained by bag mapping
  TableDesc probe;      // the other child
  int b;                // bag size
  void *index;          // hashed (phi-key, head) records, capacity index_cap
  unsigned long long index_cap;
  unsigned long long *next;  // per build slot: next chained slot + 1 (0 ends a chain)
  TableDesc out;        // hashed output (mode 1)
  unsigned long long *pairs;  // mode 0: number of matching (C', C'') pairs
  int *err;
};

struct RootArgs {
  KeyLayout L;
  TableDesc in;
  unsigned int *exists;      // per trial
  unsigned long long *count; // per trial
};

// launch configuration derived once per device
struct DevInfo {
  int sms = 0;
  int blocks_per_sm = 4;
};

// ---- launchers (cc_kernels.cu); return a cudaError_t as int ---------------------------------
// colours of trials t0 .. t0+trials-1 (Philox counter (v, t0 + t, 0, 0)) into out[t][v]
int launch_color(cudaStream_t s, const DevInfo &d, uint8_t *out, int32_t n, int32_t trials,
                 int32_t k, uint64_t seed, int32_t t0 = 0);
int launch_leaf(cudaStream_t s, const DevInfo &d, int kw, const LeafArgs &a);
// Introduce in three modes: 0 counts valid extensions per block into blk[0, grid) and writes
// exclusive bases to blk[grid, 2*grid) and the total to blk[2*grid]; 1 writes them densely at
// those bases; 2 adds them, projected by the parent forget, into a hashed table.  Modes 0 and 1
// of one node must use the same block size (and so the same grid).
// `grouped` selects candidate lists shared by runs of equal bag-neighbour images (the child
// table must then be sorted by those images, see launch_tuple_sort).
int intro_grid(const DevInfo &d, int block);
int launch_intro_blk(cudaStream_t s, const DevInfo &d, int kw, int mode, int grouped, int block,
                     const IntroArgs &a, unsigned long long *blk);
// Sort order of table records: the G-vertices of bag slots order[0..nsl) first (most
// significant); with full = 1 the remaining slots order[nsl..b) follow, then the trial and the
// colour set, so that equal keys are adjacent.  bits = total sort-key bits.
struct SortSpec {
  KeyLayout L;
  int b;
  int nsl;
  int order[kMaxBag];
  int full;
  int bits;
  // bucketed order (hbits > 0): the top hbits of a hash of the first hslots slots of `order`
  // (of the whole key when hslots == 0) come before everything else, so equal keys and equal
  // images of those slots stay together while buckets spread evenly
  int hbits;
  int hslots;
};
// Stable LSD radix sort of the nonempty records of `src` (n_src slots, n of them nonempty) into
// buf_a / buf_b (n records each); *which (0 or 1) names the buffer holding the result.  hist
// needs 256 * sort_grid(d) + 512 words.
int sort_grid(const DevInfo &d);
int sort_passes(const SortSpec &sp);
// Scratch of a one-sweep sort: 256 digit counts per pass, a tile counter per pass, and 256
// look-back words per tile of the largest pass (max_tiles >= records / sweep_tile(kw) + 1).
struct SweepScratch {
  unsigned long long *ghist;
  unsigned *tile_ctr;
  unsigned long long *status;
  unsigned long long max_tiles;
  int *err;
  int tma;  // 1: passes stream their next tile into shared memory by bulk copy
};
int sweep_tile(int kw);
// Lets the bulk-copy sort passes use more than 48 KB of shared memory; call once per device
// before the first sort (returns a cudaError_t as int).
int prepare_sort_kernels();
// The record counts live on the device: the first pass scans min(*n_src, src_cap) slots of
// src (holes skipped), later passes *n records.  buf_a / buf_b hold buf_cap records.
int launch_sort_records(cudaStream_t s, const DevInfo &d, int kw, const SortSpec &sp,
                        const void *src, const unsigned long long *n_src,
                        unsigned long long src_cap, const unsigned long long *n,
                        unsigned long long buf_cap, void *buf_a, void *buf_b,
                        unsigned long long *hist, int *which, const SweepScratch *sw);
// Bucketed merge of a forget's records (cc_part.cu): the nonempty records of src (scan bound
// *n_src, at most src_cap slots) merged by key into dst (room for dst_cap records, *dst_count
// receives the merged count), sorted by (bucket, full key order) for a spec with sp.full = 1 and
// sp.hbits = part_bucket_bits(records) (at most 20).  mid, and spare when sp.hbits > 10, are
// record spaces of space_cap >= records slots; src must hold at least that many slots too (it is
// reused as scratch).  The scratch words:
struct PartScratch {
  unsigned *hist;     // 2^hbits bucket sizes
  unsigned long long *base;    // 2^hbits + 1 bucket starts (the last: the record count)
  unsigned long long *cur1;    // 2^(first split's bits) cursors
  unsigned long long *cur2;    // 2^hbits cursors
  unsigned long long *status;  // 2^hbits look-back words
  unsigned *claim;    // bucket counter
  unsigned long long *scan;    // scan_scratch_words(d) words
  int *err;           // the run's error word (a look-back wait that gave up sets kErrTimeout)
};
int part_bucket_bits(unsigned long long records, int kw);
// lets the split and bucket-sort kernels use more than 48 KB of shared memory (once per device)
int prepare_part_kernels();
int launch_part_merge(cudaStream_t s, const DevInfo &d, int kw, const SortSpec &sp,
                      const void *src, const unsigned long long *n_src,
                      unsigned long long src_cap, void *mid, void *spare,
                      unsigned long long space_cap, const PartScratch &ps, void *dst,
                      unsigned long long dst_cap, unsigned long long *dst_count);
// One record per run of equal keys of the sorted `src` (min(*n, n_cap) records) with the summed
// count, written densely to dst (room for n_cap records); *count receives the number of runs.
// blk needs 2 * sort_grid(d) + 1 words.  With from_s non-null the records carry full sort keys of
// that order (a one-sweep sort leaves them so) and are written back as packed keys.
int launch_reduce(cudaStream_t s, const DevInfo &d, int kw, const void *src,
                  const unsigned long long *n, unsigned long long n_cap, unsigned long long *blk,
                  void *dst, unsigned long long *count, const SortSpec *from_s,
                  bool narrow = false);
// True when a one-sweep sort (sort_sweep 1) of 128-bit-key records by a full order of at most
// 64 bits moves 16-byte (sort key, count) records from its first pass on: the reduce that
// follows must then be given narrow = true.
bool sort_narrows(int kw, const SortSpec &sp, int sort_sweep);
// Introduce of a vertex with at most one bag neighbour, warp by warp, for planned runs: mode 1
// appends in per-warp chunks from a.cursor (holes left where chunks are not filled), mode 2
// adds into the parent forget's hash table.
int launch_intro_warp(cudaStream_t s, const DevInfo &d, int kw, int mode, const IntroArgs &a);
// one warp polls *flag (which nothing sets) `polls` times, then sets kErrTimeout in *err
int launch_wait_probe(cudaStream_t s, const unsigned long long *flag, unsigned polls, int *err);
// allowed-mapping masks restricting the pattern vertex of bit ubit to the host vertices
// v = slice (mod slices), other bits from base (null: all allowed)
int launch_slice_mask(cudaStream_t s, const DevInfo &d, const uint32_t *base, int32_t n,
                      uint32_t ubit, int32_t slices, int32_t slice, uint32_t *out);
int launch_deg8(cudaStream_t s, const DevInfo &d, const int32_t *row_ptr, int32_t n,
                uint8_t *deg8);
// Grouped introduce (child sorted by bag-neighbour images), warp by warp, for planned runs;
// modes as launch_intro_warp.
// Two introduces in one pass (planned capacities, mode 1): x1 = introduce u1 over y, then x2 =
// introduce u2 over x1, u2 not adjacent to u1 and y in runs of equal images of u2's bag
// neighbours.  x1's entries are generated and counted (into c_valid) but not stored; each is
// extended by the run's shared list of u2's candidates and x2's entries are appended as in
// launch_intro_group_warp.
int launch_intro_chain(cudaStream_t s, const DevInfo &d, int kw, const IntroArgs &a);
// hist[(t * n + w) * 4 .. + 4): colour c's count in 16-bit field c of the four words, over w's
// neighbours v with deg(v) >= degF and bit `ubit` of allow[v] (when G.allow); adds the
// adjacency entries read (trials times 2m) to *cand.  Degrees must be below 65536.
int launch_nb_colour_hist(cudaStream_t s, const DevInfo &d, const GraphDev &G, int trials,
                          int degF, uint32_t ubit, unsigned long long *hist,
                          unsigned long long *cand);
int launch_intro_group_warp(cudaStream_t s, const DevInfo &d, int kw, int mode,
                            const IntroArgs &a);
int launch_forget(cudaStream_t s, const DevInfo &d, int kw, int block, const ForgetArgs &a);
int launch_join(cudaStream_t s, const DevInfo &d, int kw, int phase, int block,
                const JoinArgs &a);  // phase 0 build, 1 count pairs, 2 write
int launch_root(cudaStream_t s, const DevInfo &d, int kw, const RootArgs &a);
int launch_unpack(cudaStream_t s, const DevInfo &d, int kw, const KeyLayout &L,
                  const TableDesc &t, int b, unsigned long long cap, int32_t *trial,
                  int32_t *phi, uint32_t *mask, unsigned long long *cnt,
                  unsigned long long *n_out);

// ---- reconstruction (cc_enum.cu) ---------------------------------------------------------
// A node as the top-down walk sees it, with its stored table (if any).
struct EnumNode {
  int type, child0, child1, vertex;
  int b;                  // bag size
  int bag[kMaxBag];       // F-vertices of the bag, slot order
  int p;                  // introduce: slot of the introduced vertex
  int nnb;                // introduce: bag neighbours (child-bag slots in nb_slot);
  int nb_slot[kMaxBag];   // forget: F-neighbours of the forgotten vertex in the bag (F-vertex ids)
  int degF;               // introduce: degree filter bound (0 = off)
  int vstar;              // |V*_x|
  const void *slots;      // stored table (leaf: indexed by trial * n + v)
  unsigned long long cap, count;
  int hashed, sorted;
  SortSpec spec;          // order of a sorted table
};

struct EnumArgs {
  GraphDev G;
  KeyLayout L;
  const EnumNode *nodes;  // device array
  int x;                  // node processed by this step
  int nF, R, D;           // state = R ints: trial, colour set, depth, stack[D], Phi[nF]
  const int *in;
  unsigned long long n_in;
  int *out;
  const unsigned long long *off;  // write pass: first output state of each input state
  unsigned *cnt;                  // count pass: output states per input state
};

int launch_enum_init(cudaStream_t s, const DevInfo &d, int kw, const EnumArgs &a,
                     const void *root, unsigned long long bound, unsigned long long *n);
int launch_enum_step(cudaStream_t s, const DevInfo &d, int kw, int mode, const EnumArgs &a);
size_t scan_scratch_words(const DevInfo &d);
// exclusive scan of n u32 values into off[0..n) and the total into off[n]
int launch_scan_u32(cudaStream_t s, const DevInfo &d, const unsigned *v, unsigned long long n,
                    unsigned long long *off, unsigned long long *scratch);
int launch_rows_extract(cudaStream_t s, const DevInfo &d, const int *states,
                        unsigned long long n, int R, int D, int nF, int *rows, unsigned *perm);
// every row sorted in place into increasing order (the vertex set of an embedding)
int launch_rows_canon(cudaStream_t s, const DevInfo &d, int *rows, int nF,
                      unsigned long long n);
// lexicographic order of the rows (nF ints each, values < 2^nb) as a permutation; *result is
// perm or tmp.  hist needs 256 * 2 * sms words.
int launch_rows_sort(cudaStream_t s, const DevInfo &d, const int *rows, int nF, int nb,
                     unsigned long long n, unsigned *perm, unsigned *tmp, unsigned long long *hist,
                     unsigned **result);
int launch_rows_heads(cudaStream_t s, const DevInfo &d, const int *rows, int nF,
                      const unsigned *perm, unsigned long long n, unsigned *flag);
int launch_rows_gather(cudaStream_t s, const DevInfo &d, const int *rows, int nF,
                       const unsigned *perm, unsigned long long n, const unsigned *flag,
                       const unsigned long long *off, unsigned long long limit, int *out);

size_t slot_bytes(int kw);       // bytes of one table record for 1- or 2-word keys
size_t index_slot_bytes(int kw); // bytes of one join-index record

}  // namespace cc
