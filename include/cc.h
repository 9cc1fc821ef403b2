/*
 * cc.h -- C ABI of the GB300 colour-coding library for subgraph isomorphism (SubIso) and
 * subgraph enumeration (SubEnum), after Malik, Suchy and Valla, arXiv 1908.11248.
 *
 * The method (paper Sections 2-4): colour the host graph G at random with k colours (Section
 * 2.1), run a dynamic programme bottom-up over a nice tree decomposition of the pattern F whose
 * tables hold the nonzero configurations (bag mapping phi, colour set C) of every node
 * (Section 3.1: leaf, introduce, forget and join rules), test the root (a solution exists iff the
 * root table is nonempty), and reconstruct the embeddings top-down (Section 4).  This library
 * extends the Boolean table of the paper to uint64 counts of colourful embeddings (mod 2^64);
 * the set of nonzero configurations is exactly the paper's.
 *
 * Conventions
 *   - Every function returns CC_OK (0) or a negative error code; no exception crosses the ABI.
 *   - Pointers named h_* are HOST pointers and are only read or written during the call (the
 *     library copies inputs in).  Pointers named d_* are DEVICE pointers of the context's GPU.
 *   - Graph vertices are int32 ids 0..n-1; pattern vertices 0..n_F-1 with n_F <= 32.
 *   - Colours are 0-based; bit i of a colour set is colour i (Section 3.2).  k >= n_F, k <= 32.
 *   - One context is driven by one host thread at a time, except the cc_serve_* functions,
 *     which are thread-safe.
 *   - All device work is ordered on the stream given to cc_create, in the order of the calls
 *     (a replayed graph's branches fork from it and join it again); a running server issues its
 *     queries on streams of its own.
 */
#ifndef CC_H
#define CC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------------------------ */
#define CC_OK 0
#define CC_EINVAL (-1)     /* malformed argument: bad CSR, bad decomposition, k < n_F, ...     */
#define CC_ENOMEM (-2)     /* the device arena cannot hold the request                          */
#define CC_ECAPACITY (-3)  /* a table outgrew its planned capacity; nothing partial is returned */
#define CC_ETIMEOUT (-4)   /* a bounded device-side wait or a host wait ran out                 */
#define CC_ECUDA (-5)      /* a CUDA runtime call failed                                        */
#define CC_ENOTFOUND (-6)  /* unknown pattern, colouring, run or ticket id                      */
#define CC_EKEYWIDTH (-7)  /* trial, bag-mapping and colour-set bits do not fit in 128 bits     */
#define CC_EBUSY (-8)      /* the context is serving: only cc_serve_* and the pattern calls run */
#define CC_ECANCELED (-9)  /* a served query was dropped before it started (cc_serve_cancel)     */

/* Static text for an error code. */
const char *cc_strerror(int code);

/* ---- context ------------------------------------------------------------------------------ */
typedef struct cc_ctx cc_ctx;

/* Creates a context on CUDA device `device`, issuing all work on `cuda_stream` (a cudaStream_t,
 * NULL for the legacy default stream).  Device memory: if d_arena is non-NULL the context
 * sub-allocates every device buffer from [d_arena, d_arena + arena_bytes), which stays owned by
 * the caller and must outlive the context; if d_arena is NULL the context allocates an arena of
 * arena_bytes itself (cudaMalloc) and frees it in cc_destroy.  Errors: CC_EINVAL (bad device or
 * arena_bytes == 0), CC_ECUDA, CC_ENOMEM. */
int cc_create(cc_ctx **out, int device, void *cuda_stream, void *d_arena, size_t arena_bytes);

/* Waits for the context's stream, stops a running server and frees the context. */
int cc_destroy(cc_ctx *ctx);

/* ---- host graph G (paper Section 1.2: undirected and simple) ------------------------------- */
/* Loads G from host CSR: h_row_ptr[n+1] (h_row_ptr[0] == 0, nondecreasing) and
 * h_col[h_row_ptr[n]].  Every row must be strictly increasing, hold no self loop, and the
 * adjacency must be symmetric; anything else is CC_EINVAL.  Replaces a previous graph and
 * releases every run and colouring made on it.  n may be 0 (no vertex). */
int cc_load_graph(cc_ctx *ctx, int32_t n, const int32_t *h_row_ptr, const int32_t *h_col);

/* ---- pattern F and its decomposition (Sections 1.2 and 3) ---------------------------------- */
/* A tree decomposition (Section 1.2, Definition of tree decomposition): num_bags bags, bag i
 * holding h_bag_vtx[h_bag_ptr[i] .. h_bag_ptr[i+1]), h_parent[i] its parent bag or -1 for the
 * single root.  Bags must be nonempty. */
typedef struct {
  int32_t num_bags;
  const int32_t *h_bag_ptr;
  const int32_t *h_bag_vtx;
  const int32_t *h_parent;
} cc_td;

/* Loads F (n_F vertices, m_F undirected edges h_edges[2*m_F]) with decomposition `td`, or, if
 * td is NULL, with a minimum-width decomposition computed from elimination orderings
 * (Section 3, O(n_F^2 2^n_F) for n_F <= 20, a greedy min-fill ordering above).  The
 * decomposition is converted to a nice one (Section 1.2, leaf bags of size one, empty root of
 * degree one): children taken in increasing id, forgets before introduces, each in increasing
 * vertex order, several children joined left-deep.  Errors: CC_EINVAL for n_F outside 1..32,
 * an edge out of range or a loop, or a td that is not a tree decomposition of F. */
int cc_load_pattern(cc_ctx *ctx, int32_t n_F, int32_t m_F, const int32_t *h_edges,
                    const cc_td *td, int32_t *pattern_id);

/* A pattern whose embeddings must also respect allowed mappings (Section 3.2, masking
 * unprofitable mappings: the extended input names, for each vertex of the network, the pattern
 * vertices that may be mapped to it).  h_allow[n] (n of the loaded graph): bit u of h_allow[v]
 * lets F-vertex u be mapped to host vertex v.  Tables, counts and enumerations then count only
 * maps that respect it (the degree filter still applies on top).  Otherwise as cc_load_pattern.
 * The masks belong to the graph loaded now: runs of the pattern fail with CC_EINVAL once a graph
 * of other content is loaded.  Errors: as cc_load_pattern, CC_EINVAL (no graph, h_allow NULL),
 * CC_EBUSY, CC_ENOMEM, CC_ECUDA. */
int cc_load_pattern_masked(cc_ctx *ctx, int32_t nF, int32_t mF, const int32_t *h_edges,
                           const cc_td *td, const uint32_t *h_allow, int32_t *pattern_id);

/* Host-only (no context, no GPU): the nice decomposition cc_load_pattern would build for F and
 * td (td NULL: minimum width), in the layout of cc_pattern_nodes.  Arrays hold max_nodes nodes
 * (h_bag_ptr max_nodes+1, h_bag_vtx max_nodes*n_F).  *num_nodes and *width receive its size and
 * width.  Errors: as cc_load_pattern; CC_ECAPACITY if it has more than max_nodes nodes. */
int cc_nice_decomposition(int32_t n_F, int32_t m_F, const int32_t *h_edges, const cc_td *td,
                          int32_t max_nodes, int32_t *h_type, int32_t *h_child0,
                          int32_t *h_child1, int32_t *h_vertex, int32_t *h_bag_ptr,
                          int32_t *h_bag_vtx, int32_t *num_nodes, int32_t *width);

/* Host-only: CC_OK if (n, h_row_ptr, h_col) is a valid simple undirected CSR graph (the checks of
 * cc_load_graph), CC_EINVAL otherwise. */
int cc_check_graph(int32_t n, const int32_t *h_row_ptr, const int32_t *h_col);

/* Node count and width (largest bag size minus one) of a loaded pattern's nice decomposition. */
int cc_pattern_info(cc_ctx *ctx, int32_t pattern_id, int32_t *num_nodes, int32_t *width);

/* The nice decomposition in post-order (root last).  type: 0 leaf, 1 introduce, 2 forget,
 * 3 join; child0/child1 node ids or -1; vertex: leaf, introduced or forgotten F-vertex (-1 for
 * join); bag of node i is h_bag_vtx[h_bag_ptr[i] .. h_bag_ptr[i+1]) in increasing order.
 * Arrays: num_nodes entries, h_bag_ptr num_nodes+1, h_bag_vtx num_nodes*n_F. */
int cc_pattern_nodes(cc_ctx *ctx, int32_t pattern_id, int32_t *h_type, int32_t *h_child0,
                     int32_t *h_child1, int32_t *h_vertex, int32_t *h_bag_ptr,
                     int32_t *h_bag_vtx);

/* ---- colourings (Section 2.1) ------------------------------------------------------------- */
/* Draws `trials` random k-colourings of the loaded graph on the device: the colour of vertex v in
 * trial t is floor(x * k / 2^32) where x is the first output word of Philox4x32-10 (Salmon et
 * al., SC'11) at counter (v, t, 0, 0) and key (low 32 bits of seed, high 32 bits of seed).
 * Errors: CC_EINVAL (no graph, trials < 1, k outside 1..32). */
int cc_color(cc_ctx *ctx, uint64_t seed, int32_t trials, int32_t k, int32_t *coloring_id);

/* Uses explicit colourings h_colors[trials * n] (row t = trial t, values < k). */
int cc_set_colors(cc_ctx *ctx, const uint8_t *h_colors, int32_t trials, int32_t k,
                  int32_t *coloring_id);

/* Copies a colouring back to the host (h_out[trials * n]). */
int cc_get_colors(cc_ctx *ctx, int32_t coloring_id, uint8_t *h_out);

/* Frees a colouring (runs made from it keep their own reference until released). */
int cc_release_colors(cc_ctx *ctx, int32_t coloring_id);

/* ---- the dynamic programme (Section 3.1) -------------------------------------------------- */
typedef struct {
  int32_t degree_filter; /* map y to x only if deg_G(x) >= deg_F(y) (Section 3.2); 1 = on     */
  int32_t retain;        /* keep every node table for cc_enumerate / cc_table_dump            */
  int32_t fuse;          /* introduce followed by forget: 0 each node stores its own table;   */
                         /* 1 the introduce adds its entries, projected, into the forget's     */
                         /*   hash table; 2 (default) it writes them projected and densely,    */
                         /*   they are sorted and equal keys reduced.  With 1 and 2 the        */
                         /*   introduce's table is never stored (its size is still counted)    */
  int32_t use_graph;     /* 1: replay the node kernels from a captured CUDA graph when the     */
                         /*    plan's capacities are known (falls back to planning otherwise)  */
  float load_factor;     /* hash-table fill target in (0, 0.9]; 0 = library default           */
  int32_t block;         /* threads per block of the node kernels (128, 256 or 512)           */
  int32_t profile;       /* 1: time every kernel launch with CUDA events (cc_run_timings)     */
  int32_t group;         /* 1: an introduce whose vertex has >= 2 bag neighbours first sorts   */
                         /*    its child by their images and shares candidate lists per run    */
  int32_t sort_sweep;    /* 1: radix sorts take all digit counts in one read and one kernel   */
                         /*    per pass (decoupled look-back); 2: as 1, each block bringing its */
                         /*    next tile into shared memory by bulk copy while it works on the  */
                         /*    current one; 0: histogram+scan+scatter passes; 3: a forget after */
                         /*    an introduce merges by buckets (a hash of the next introduce's   */
                         /*    bag-neighbour images split the records, each bucket is sorted    */
                         /*    and merged in shared memory), other sorts as 1                    */
  int32_t distance_prune; /* 1: an introduced vertex with no bag neighbour takes only the host */
                         /*    vertices within distance dist_F(w, u) of phi(w), w the bag vertex */
                         /*    nearest to it in F (Section 3.2, mapping expansion); root results */
                         /*    are unchanged, tables shrink                                      */
  int32_t max_slices;    /* most slices a single trial that does not fit may be split into     */
                         /*    (CC_MODE_SLICED); 0 = 4096                                        */
  int32_t part_bits;     /* sort_sweep 3: log2 of the bucket count (1..20); 0 = from the size  */
                         /*    of the table, about 1024 records a bucket                         */
  int32_t chain;         /* 1 (default): in planned runs, an introduce whose parent introduces */
                         /*    a vertex not adjacent to its own, with >= 2 bag neighbours whose */
                         /*    images the child's runs share, runs in one pass with that parent: */
                         /*    its entries are generated, counted and extended at once, and its */
                         /*    table is never stored (its size is still counted; enumeration   */
                         /*    resolves introduce nodes by their rule, Section 4)              */
} cc_run_opts;

/* Fills *opts with the defaults (degree_filter 1, retain 0, fuse 2, use_graph 0, load factor
 * 0.5, block 256, profile 0, group 1, sort_sweep 1, distance_prune 0, max_slices 0,
 * part_bits 0). */
void cc_default_opts(cc_run_opts *opts);

/* Runs the DP of pattern `pattern_id` for every trial of colouring `coloring_id` (all trials in
 * the same launches: the trial index is part of every table key).  Requires k >= n_F.  On
 * success *run_id names the result; per-trial results stay on the device until read.  When all
 * trials together do not fit the arena and no tables are to be kept (retain 0), the trials run in
 * halves, recursively, until they fit (trial streaming; cc_run_mode gives CC_MODE_STREAMED), and
 * a single trial that does not fit runs in slices by the image of one pattern vertex
 * (CC_MODE_SLICED).  Errors: CC_EINVAL, CC_ENOTFOUND, CC_ENOMEM (arena too small even for one
 * trial in opts->max_slices slices: nothing is kept),
 * CC_EKEYWIDTH (ceil(log2 trials) + width_bags * ceil(log2 n) + k > 128), CC_ECUDA. */
int cc_run_dp(cc_ctx *ctx, int32_t pattern_id, int32_t coloring_id, const cc_run_opts *opts,
              int32_t *run_id);

/* Runs several (pattern, colouring) DPs with one set of options (the batched execution of
 * Section 5's many queries over one graph).  With opts->use_graph, retain 0 and profile 0, the
 * requests that have been planned (an earlier run of the same pattern, graph content, trials,
 * colours and options) run as parallel branches of captured CUDA graphs (up to 64 branches a
 * graph; a set whose memory does not fit at once is split in halves), each branch in device
 * memory reserved for its graph; a graph is kept per request list and replayed, its colours
 * copied in first.  A request that outgrows its graph's capacities makes the library drop the
 * graph and run its requests again directly.  The other requests run one after the other on the
 * context's stream (which plans them).  h_run_ids[npat] out; on error no run is kept.  Errors as
 * cc_run_dp. */
int cc_run_batch(cc_ctx *ctx, int32_t npat, const int32_t *h_pattern_ids,
                 const int32_t *h_coloring_ids, const cc_run_opts *opts, int32_t *h_run_ids);

/* Autotuner: the running time depends on the decomposition supplied rather than on the
 * treewidth of F (section on obtaining a nice tree decomposition), and beyond its width on the
 * order of its nodes and on how the node rules are carried out.  Times the
 * DP of pattern `pattern_id` under colouring `coloring_id` (each candidate: one run that plans,
 * then the best wall time of `repeats` planned runs, results read back) and picks, by coordinate
 * descent from *base (NULL: cc_default_opts; retain, profile and use_graph are cleared):
 *   - the node schedule: the pattern's tree decomposition rooted at each of its bags in turn
 *     (at most max_schedules distinct nice decompositions, the loaded one first; each other one
 *     is loaded as a new pattern, which the context keeps);
 *   - fuse (2, 1, 0), block (256, 128, 512), load_factor (0.5, 0.35, 0.7), sort_sweep (1, 0)
 *     and group (1, 0), one option at a time.
 * Every candidate's per-trial counts and exists flags must equal the first's (otherwise
 * CC_ECUDA).  Out: *best_opts, *best_pattern_id (use it with the options), *best_ms (may be
 * NULL) and *configs_tried (may be NULL).  Errors: CC_EINVAL, CC_ENOTFOUND, CC_EBUSY, and those
 * of cc_run_dp. */
int cc_autotune(cc_ctx *ctx, int32_t pattern_id, int32_t coloring_id, const cc_run_opts *base,
                int32_t max_schedules, int32_t repeats, cc_run_opts *best_opts,
                int32_t *best_pattern_id, float *best_ms, int32_t *configs_tried);

/* ---- repetition to an error bound (Section 2.1) ------------------------------------------- */
/* Number of colourings after which a present copy of a pattern with n_F vertices is missed with
 * probability at most epsilon when k = n_F: ceil(e^{n_F} * ln(1/epsilon)) (clamped to INT32_MAX);
 * -1 if n_F < 1 or epsilon is not in (0, 1).  Host only. */
int32_t cc_solve_trials(int32_t n_F, double epsilon);

/* The paper's whole solve: colours the graph again and again (trial t of the solve by Philox
 * counter (v, t, 0, 0) under `seed`, so the solve equals one run over all its trials) in batches
 * of `batch` trials, up to min(cc_solve_trials(n_F, epsilon), max_trials) trials, with
 * cc_default_opts.  limit == 0 (decision, SubIso): stops after the first batch in which a trial
 * finds a colourful copy.  limit > 0 (enumeration, SubEnum): runs every trial, keeps each batch's
 * tables and merges its embeddings, each once: h_out[limit][n_F] receives the *n_out
 * lexicographically smallest distinct embeddings found.  *found = 1 if any trial found a copy;
 * *trials_run the trials run; *estimate (may be NULL) the mean count over the trials divided by
 * (k)_{n_F}/k^{n_F}, an unbiased estimate of the number of embeddings.  Batches run with tables
 * kept (limit > 0) must fit the arena whole.  Errors: CC_EINVAL, CC_ENOTFOUND, CC_EBUSY,
 * CC_ENOMEM, CC_EKEYWIDTH, CC_ECUDA. */
int cc_solve(cc_ctx *ctx, int32_t pattern_id, uint64_t seed, int32_t k, double epsilon,
             int32_t batch, int32_t max_trials, uint64_t limit, int32_t *h_out, uint64_t *n_out,
             uint8_t *found, int32_t *trials_run, double *estimate);

/* How a run was executed. */
#define CC_MODE_EXACT 0   /* count passes size every table exactly (first run of a plan key) */
#define CC_MODE_PLANNED 1 /* capacities from the plan, appends in chunks, no host reads */
#define CC_MODE_GRAPH 2   /* planned, replayed from a captured CUDA graph */
#define CC_MODE_STREAMED 3 /* all trials together did not fit: ran in chunks of trials (halved
                            * until they fit); counts, exists flags and table sizes as for one
                            * run, no tables kept */
#define CC_MODE_SLICED 4   /* as CC_MODE_STREAMED, and a single trial did not fit either: it ran
                            * in s slices, slice i restricting the vertex of the decomposition's
                            * first leaf to host vertices v = i (mod s) through allowed-mapping
                            * masks (Section 3.2); the embeddings split by that vertex's image,
                            * so counts (summed mod 2^64) and exists flags are exact, while table
                            * sizes are sums over slices (an upper bound for nodes whose bag
                            * lacks that vertex); s doubles from 2 until every slice fits, at most
                            * max_slices of the run's options (then CC_ENOMEM) */

/* *mode = one of CC_MODE_* for run `run_id`.  Errors: CC_EINVAL, CC_ENOTFOUND. */
int cc_run_mode(cc_ctx *ctx, int32_t run_id, int32_t *mode);

/* Per trial: 1 if a colourful copy of F exists (the root table is nonempty), else 0. */
int cc_decide(cc_ctx *ctx, int32_t run_id, uint8_t *h_exists);

/* Per trial: number of colourful embeddings Phi: V(F) -> V(G) (labelled maps, so every copy
 * counts |Aut(F)| times), mod 2^64. */
int cc_count(cc_ctx *ctx, int32_t run_id, uint64_t *h_counts);

/* Table sizes |D_x| summed over trials, one per node (h_sizes[num_nodes]), and their sum. */
int cc_table_stats(cc_ctx *ctx, int32_t run_id, uint64_t *h_sizes, uint64_t *h_total);

/* Copies the table of node `node` (run made with retain = 1 and fuse = 0, or a node whose table
 * was stored) to the host, unpacked: for entry i, h_trial[i], the bag tuple
 * h_phi[i*b .. i*b+b) (b = bag size, bag order increasing), h_mask[i] and h_cnt[i].  Arrays
 * must hold `capacity` entries; *n_out gets the entry count (CC_ECAPACITY if it exceeds
 * capacity).  Entries come in no particular order. */
int cc_table_dump(cc_ctx *ctx, int32_t run_id, int32_t node, uint64_t capacity,
                  int32_t *h_trial, int32_t *h_phi, uint32_t *h_mask, uint64_t *h_cnt,
                  uint64_t *n_out);

/* Result reconstruction (Section 4) on the device for a run made with retain = 1: the union
 * over the run's trials of all colourful embeddings, without repeats, sorted lexicographically
 * by (Phi(0), ..., Phi(n_F-1)), truncated to `limit` rows written to h_out[limit * n_F].
 * *n_out = rows written, *n_total = distinct embeddings before truncation.  Errors:
 * CC_EINVAL (run not retained), CC_ENOMEM (the embeddings do not fit the arena). */
int cc_enumerate(cc_ctx *ctx, int32_t run_id, uint64_t limit, int32_t *h_out, uint64_t *n_out,
                 uint64_t *n_total);

/* As cc_enumerate, counting occurrences that differ in their vertex sets (the switch of
 * Section 5.2: non-induced occurrences and automorphisms map the pattern onto the same vertex
 * set in several ways): each embedding is replaced by its image set in increasing vertex order,
 * and h_out receives the `limit` lexicographically smallest distinct sets; *n_total = distinct
 * vertex sets.  Errors as cc_enumerate. */
int cc_enumerate_sets(cc_ctx *ctx, int32_t run_id, uint64_t limit, int32_t *h_out,
                      uint64_t *n_out, uint64_t *n_total);

/* Frees a run's tables and results. */
int cc_release(cc_ctx *ctx, int32_t run_id);

/* Kernel kinds reported by cc_run_timings. */
#define CC_K_COLOR 0
#define CC_K_LEAF 1
#define CC_K_INTRO_COUNT 2
#define CC_K_INTRO_WRITE 3
#define CC_K_INTRO_FUSED 4
#define CC_K_FORGET 5
#define CC_K_JOIN_BUILD 6
#define CC_K_JOIN_COUNT 7
#define CC_K_JOIN_WRITE 8
#define CC_K_ROOT 9
#define CC_K_SORT 10   /* all passes of one radix sort of a table's records */
#define CC_K_REDUCE 11 /* reduce-by-key of sorted records (a forget's merge) */
#define CC_K_MERGE 12  /* a forget's whole bucketed merge (sort_sweep 3): split, sort, merge */
#define CC_K_INTRO_CHAIN 13 /* two introduces in one pass (option chain); node = the upper one */

/* Per-launch device times of a run made with profile = 1, in launch order: node id, kernel
 * kind (CC_K_*), milliseconds between CUDA events recorded on the context's stream just before
 * and just after the launch, and the number of candidate vertices the launch examined
 * (introduce kinds; 0 otherwise).  Arrays hold `capacity` entries; *n_out gets the launch
 * count (CC_ECAPACITY if it exceeds capacity). */
int cc_run_timings(cc_ctx *ctx, int32_t run_id, int32_t capacity, int32_t *h_node,
                   int32_t *h_kind, float *h_ms, uint64_t *h_candidates, int32_t *n_out);

/* Failure detection check (no counterpart in the paper): every device-side wait of the library
 * (the sort passes' look-back, the bulk-copy barriers) polls a bounded number of times, then
 * records CC_ETIMEOUT in the run's error word and returns, leaving the context usable.  This call
 * makes one such wait run out on purpose: a warp polls a device word that nothing sets, `polls`
 * times, and the error word is read back.  Returns CC_ETIMEOUT when the wait gave up as it
 * should; CC_EINVAL (polls 0), CC_EBUSY, CC_ENOMEM, CC_ECUDA otherwise. */
int cc_probe_bounded_wait(cc_ctx *ctx, uint32_t polls);

/* Context counters: kernel launches issued since cc_create, arena bytes in use and arena size. */
int cc_context_stats(cc_ctx *ctx, uint64_t *kernel_launches, uint64_t *arena_used,
                     uint64_t *arena_size);

/* ---- a count that allocates no device memory (the paper has no counterpart) --------------- */
/* Size of the fixed device array cc_count_noalloc works in. */
#define CC_NOALLOC_BYTES (64ull << 20)

/* For callers that cannot allocate device memory: processes whose device memory belongs to
 * another allocator that must not be bypassed (a framework's caching pool, a fixed partition of
 * the GPU), and code loaded into such processes with no allocator of its own to call.
 * Returns what cc_count and cc_decide return for graph (n, h_row_ptr, h_col), pattern (n_F, m_F,
 * h_edges, td) and cc_color(seed, trials, k) under cc_default_opts, computing everything inside
 * one CC_NOALLOC_BYTES device array that is part of the library image (every GPU that loads the
 * library holds it until exit); the caller passes only host inputs and the host outputs
 * h_counts[trials] and h_exists[trials].  The call copies its inputs from (pageable) host memory
 * on `cuda_stream`, waits for that stream between steps and returns when the results are on the
 * host.  On a stream that is being captured into a CUDA graph it does nothing and returns
 * CC_EINVAL.  The first call on a device looks up the array's device address.  Every call
 * shares the array and leaves its contents behind (each call clears what it needs); calls whose
 * work overlaps on one GPU race and must be serialised by the caller.  Errors: CC_ENOMEM when
 * the graph and colourings (4(n+1) + 4*h_row_ptr[n] + n(1 + trials) bytes plus under 1 MiB of
 * fixed state) or later the tables do not fit the array; CC_EINVAL as above; otherwise those of
 * the calls it stands for. */
int cc_count_noalloc(int device, void *cuda_stream, int32_t n, const int32_t *h_row_ptr,
                     const int32_t *h_col, int32_t n_F, int32_t m_F, const int32_t *h_edges,
                     const cc_td *td, uint64_t seed, int32_t trials, int32_t k,
                     uint64_t *h_counts, uint8_t *h_exists);

/* ---- serving: a resident graph, queries admitted by table memory, batched as they arrive --- */
/* Many pattern queries against the loaded graph (Section 5 runs every query of a data set on one
 * host graph).  cc_serve_start starts a server thread that from then on alone issues the
 * context's device work: until cc_serve_stop, every other call on the context returns CC_EBUSY
 * except cc_serve_*, cc_load_pattern, cc_pattern_info, cc_pattern_nodes and cc_context_stats
 * (which may be called from any thread).  Queries wait in submission order.  The server admits
 * the next one while one of max_inflight execution slots (each a CUDA stream; 0 = 8, at most
 * 64) is free and the table memory its plan needs fits within mem_budget bytes of the arena
 * (0 = half the free arena) beside the queries already running, so that queries arriving while
 * others run share the GPU with them.  Each query colours the graph (cc_color with its seed,
 * trials and k) and runs the DP with cc_default_opts inside its own arena range, reserved at
 * admission and trimmed to what its kernels use.  A query whose (pattern, trials, k) has no
 * plan yet runs exactly, synchronously on its slot while the other slots keep running; later
 * ones of the same key run planned, and one that outgrows its plan runs again exactly.  A query
 * whose tables do not fit the budget while running alone runs as cc_run_dp would (its trials in
 * chunks, a single trial in slices by the image of one pattern vertex), synchronously; only if
 * that fails too does it end with CC_ENOMEM, and later queries of its key are refused with
 * CC_ENOMEM at once.  A query with limit > 0 keeps its tables and, once its DP is done,
 * reconstructs the `limit` lexicographically smallest distinct embeddings over its trials
 * (cc_enumerate), synchronously on its slot; such a query must fit without slicing.  Results
 * are those of cc_count, cc_decide and cc_enumerate for the same inputs, whatever else runs.
 * Errors: CC_EINVAL (no graph, bad max_inflight), CC_EBUSY (already serving), CC_ECUDA. */
int cc_serve_start(cc_ctx *ctx, size_t mem_budget, int32_t max_inflight);

/* Queues a query of pattern `pattern_id` under colouring (seed, trials, k) and returns at once
 * with *ticket; limit > 0 also asks for its first `limit` embeddings.  A bad pattern id or
 * k < n_F is reported by the query's status.  Thread-safe.  Errors: CC_EINVAL (not serving or
 * stopping, trials < 1, k outside [1, 32]). */
int cc_serve_submit(cc_ctx *ctx, int32_t pattern_id, uint64_t seed, int32_t trials, int32_t k,
                    uint64_t limit, int64_t *ticket);

/* Polls a ticket: *done = 0 while it waits or runs.  Once done, *status is its result code and,
 * if that is CC_OK, h_counts[trials] and h_exists[trials] hold its counts and exists flags,
 * h_rows[limit * n_F] its embeddings (lexicographic, without repeats) and *n_rows their number
 * (0 when the query's limit was 0), and *latency_ns the time from submission to completion; any
 * output pointer may be NULL.  The ticket is then forgotten (a later poll gives CC_ENOTFOUND).
 * Thread-safe. */
int cc_serve_poll(cc_ctx *ctx, int64_t ticket, int32_t *done, int32_t *status,
                  uint64_t *h_counts, uint8_t *h_exists, int32_t *h_rows, uint64_t *n_rows,
                  int64_t *latency_ns);

/* Server counters since it last started: queries submitted and completed, the most queries seen
 * running at once, the most arena bytes they held at once, exact runs (first queries of a key
 * and reruns), reruns of queries that outgrew their plan, and queries that ran split (their
 * tables did not fit the budget whole).  Any pointer may be NULL.  Errors: CC_EINVAL,
 * CC_ENOTFOUND (the context never served). */
int cc_serve_stats(cc_ctx *ctx, uint64_t *submitted, uint64_t *completed, int32_t *inflight_max,
                   uint64_t *reserved_max, uint64_t *exact_runs, uint64_t *reruns,
                   uint64_t *sliced);

/* Drops every query submitted so far that has not started: each ends with status CC_ECANCELED
 * (its ticket is polled as usual); queries already running finish.  Lets a caller bound a
 * session by time when some queries are far costlier than others (a query that runs split
 * holds the GPU alone until it ends).  *n_cancelled (may be NULL) = queries dropped.  Errors:
 * CC_EINVAL (not serving). */
int cc_serve_cancel(cc_ctx *ctx, uint64_t *n_cancelled);

/* Stops the server after the queued and running queries finish; results not yet polled stay
 * available.  Returns CC_OK if no server runs. */
int cc_serve_stop(cc_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* CC_H */
