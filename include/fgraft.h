/*
 * fgraft.h -- C ABI of the GB300 FGraft builder (libfgraft.so).
 *
 * The builder of "Batched Feedback and the Random-Access Wall in
 * Search-Based Graph Construction", Section 3: a scaffold S_0 made of the
 * union of T spatial-approximation trees (symmetrised), then B synchronous
 * blocks (block(p) = p mod B) in which every point of the block beam-searches
 * the frozen substrate S_b with itself as the query (width ef_h, entering at
 * the tree roots) and the expanded vertices are occlusion-pruned (alpha) into
 * the point's own row of at most R ids; after each block
 *     S_{b+1} = S_b U {(p,u),(u,p) : u in A[p], p in block b}.
 * The final graph is the harvested rows symmetrised and re-pruned, plus the
 * tree-0 spine.  By Proposition 1 the graph is a function of
 * (data, seed, T, R, ef_h, alpha, B) only; this library produces the same
 * bits at every launch configuration.
 *
 * Conventions (all entry points):
 *  - Every pointer is a CUDA device pointer owned by the caller unless a
 *    comment says "host".  The library allocates device memory only inside
 *    fgraft_build_scaffold (the index) and frees it in fgraft_index_destroy.
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL = the legacy default
 *    stream) and is asynchronous unless a host output is requested, in which
 *    case the call synchronises `stream` before returning.
 *  - Arguments are checked before anything is launched.  Errors are returned
 *    as fgraft_status and described by fgraft_last_error(); no entry point
 *    aborts, traps or prints.
 *  - Distances (delta): squared L2 for FGRAFT_L2_F32 and FGRAFT_L2_U8,
 *    1 - <x,y> for FGRAFT_ANGULAR_F32 (unit vectors; the paper L2-normalises
 *    angular data, Section 2).  Float32 distances follow one fixed summation
 *    order (32 virtual lanes, lane l owning elements 128k + 4l + c, fused
 *    multiply-add per element, xor-butterfly combine), uint8 distances are
 *    exact integers.  Every ordering is by the pair (delta, id).
 *  - Vectors: X holds n rows of d elements (float32 or uint8) with a row
 *    stride of ld elements; ld * element size must be a multiple of 16 and X
 *    16-byte aligned; elements past d in a row are ignored.  uint8 needs
 *    d <= 256 (exact float conversion of the distance); float32 d <= 1024.
 *  - Ids are int32; n < 2^31 - 1.  Rows are padded with -1.
 */
#ifndef FGRAFT_H
#define FGRAFT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* fgraft_stream; /* same type as cudaStream_t */

typedef enum {
  FGRAFT_OK = 0,
  FGRAFT_EINVAL = 1,    /* bad argument; nothing was launched */
  FGRAFT_ENOMEM = 2,    /* a device allocation failed */
  FGRAFT_ECUDA = 3,     /* a CUDA runtime call failed (message has the CUDA error) */
  FGRAFT_EOVERFLOW = 4, /* an output capacity was too small, or a search outgrew its scratch */
  FGRAFT_ETIMEOUT = 5   /* a tensor-core kernel's bounded wait for its MMA
                           products gave up (see fgraft_tune_mma_wait); the
                           kernel drained its products in flight, freed its
                           tensor memory and returned, so the CUDA context
                           stays usable; the outputs of that call (and of an
                           index's blocks harvested since) are unspecified */
} fgraft_status;

typedef enum { FGRAFT_L2_F32 = 0, FGRAFT_ANGULAR_F32 = 1, FGRAFT_L2_U8 = 2 } fgraft_metric;

/* Build parameters, named as in Section 3. */
typedef struct {
  int32_t T;       /* SAT trees in the scaffold, 1 <= T <= 64 and T <= n */
  int32_t R;       /* degree bound of a harvested row, 1 <= R <= 1024 */
  int32_t ef_h;    /* harvest beam width, 1 <= ef_h <= 128 */
  int32_t B;       /* blocks; 0 or 1 = one frozen block (Graft) */
  float alpha;     /* occlusion factor on the unsquared distance, >= 0 */
  uint64_t seed;   /* keys the tree roots */
  int32_t metric;  /* fgraft_metric */
} fgraft_params;

/* Distance-evaluation counters (Section 2: work is the count of distance
 * evaluations, each one counted).
 * Defined by the algorithm, so a correct build reports the same numbers at
 * every launch configuration:
 *  sat_evals          per SAT node with m points below it and k children:
 *                     m + k(k-1)/2 + (m-k)k
 *  harvest_evals      sum over harvested points of the size of the visited
 *                     set of their beam (tree roots included)
 *  prune_evals        sum over kept candidates of the alive candidates
 *                     examined in the removal pass that follows the keep
 *                     (no pass after the R-th keep)
 *  final_prune_evals  sum over rows of |C(u) U spine(u)| plus the removal
 *                     passes of the rows that are re-pruned
 *  expansions         sum of the expanded-set sizes
 *  ids_scanned        neighbour ids read by the harvest (measurement only;
 *                     depends on the substrate's layout, not on the method)
 *  reruns             harvest queries re-run on global-memory scratch because
 *                     their visited set outgrew shared memory (measurement) */
typedef struct {
  uint64_t sat_evals;
  uint64_t harvest_evals;
  uint64_t prune_evals;
  uint64_t final_prune_evals;
  uint64_t expansions;
  uint64_t ids_scanned;
  uint64_t reruns;
} fgraft_counters;

typedef struct fgraft_index fgraft_index; /* opaque */

/* Scaffold S_0 (Section 1: T spatial-approximation trees [Navarro 2002];
 * Section 3: S_0 joins the edges of the T trees and adds every reverse
 * edge).
 * Root t is splitmix64(seed ^ (0x9E3779B97F4A7C15 * (t+1)) + j) mod n for
 * the smallest j >= 0 giving a root distinct from roots 0..t-1 (keyed
 * randomness, Proposition 1).  A SAT node a holding points P sorts P by
 * (delta(x,a), id); x becomes a child iff delta(x,a) < delta(x,b) for every
 * earlier child b; every other point goes to its closest child by
 * (delta, id).
 * X is borrowed, not copied: it must stay valid and unchanged until
 * fgraft_index_destroy.  On success *out owns the scaffold, the row storage
 * for the harvest and all scratch.  counters (host, optional) receives the
 * index's cumulative counters after a stream synchronisation.  The call
 * synchronises `stream` once per tree level. */
fgraft_status fgraft_build_scaffold(const void* X, int64_t n, int32_t d, int64_t ld,
                                    const fgraft_params* params, fgraft_stream stream,
                                    fgraft_index** out, fgraft_counters* counters);

/* Harvest block b (Section 3): every point p with p mod B == b (all points
 * when B <= 1) searches S_b and writes its pruned row A[p] (at most R ids in
 * keep order = (delta, id) order, -1 padded); then S_{b+1} is formed.
 * Blocks must be harvested in order 0, 1, .., B-1 (EINVAL otherwise);
 * harvesting block b again after a later block is not allowed.  Needs no
 * host synchronisation unless counters (host, optional) is given, so the
 * B calls can be captured in a CUDA graph. */
fgraft_status fgraft_harvest_block(fgraft_index* ix, int32_t b, fgraft_stream stream,
                                   fgraft_counters* counters);

/* Block b of several independent indices at once (many builds of the same
 * schedule, for example one per data shard or tenant): every index must be
 * at block b (0..B-1 in order, as for fgraft_harvest_block) and appear once.
 * The indices are grouped by kernel shape (metric, lane groups of the
 * dimension, pool slots of ef_h, 16-byte chunks per row); each group of up
 * to 64 indices takes ONE persistent search launch whose work items are the
 * (index, search) pairs of all of them, claimed from one counter, each with
 * its index's descriptor.  The per-warp layout of that launch is common to
 * the group (a shared-memory hash sized by occupancy, 4 warps per CTA,
 * register gathers; visited sets outgrowing the hash go on in global bitmaps
 * sized for the largest index, kept on the device for the process).  Then,
 * per index, the re-run pass, the prune and the reverse lists run on
 * `stream` as for fgraft_harvest_block.  Each index's rows equal those of
 * its own fgraft_harvest_block call.  Nothing is synchronised on the host;
 * not for use during stream capture (the bitmaps may be reallocated).  The
 * paper has no counterpart; it runs one build at a time. */
fgraft_status fgraft_harvest_block_multi(fgraft_index* const* ixs, int32_t nix, int32_t b,
                                         fgraft_stream stream);

/* All blocks in order, then the final graph; with use_graph != 0 the block
 * loop is captured once as a CUDA graph and replayed.  Equivalent to B calls
 * of fgraft_harvest_block followed by fgraft_prune with no outputs. */
fgraft_status fgraft_harvest_all(fgraft_index* ix, int32_t use_graph, fgraft_stream stream,
                                 fgraft_counters* counters);

/* Final graph (Section 3: rows made symmetric, pruned again, joined with the
 * parent/child edges of tree 0).  C(u) = A[u] U {p : u in A[p]}; when |C(u)| > R
 * the row is the occlusion prune of C(u) to R, otherwise C(u); then the
 * tree-0 parent and children of u are added and the row is sorted by
 * (delta(u,v), id).  The index keeps the result for fgraft_search; it is
 * computed once per index (by this call or by fgraft_harvest_all), and later
 * calls only copy it out.  out_offsets (n+1 int64) and out_ids (cap int32)
 * are optional device outputs (both NULL: keep internally only); when cap is
 * too small the call returns EOVERFLOW and writes the size needed to
 * *needed (host, optional).  Requires every block to have been harvested. */
fgraft_status fgraft_prune(fgraft_index* ix, fgraft_stream stream, fgraft_counters* counters,
                           int64_t* out_offsets, int32_t* out_ids, int64_t cap, int64_t* needed);

/* Stand-alone batched occlusion prune (Section 3, after FANNG and DiskANN).
 * List i belongs to point owner[i] and holds cand_ids[cand_off[i] ..
 * cand_off[i+1]); the owner itself and repeated ids are dropped, the rest is
 * sorted by (delta(owner, c), id) and pruned with alpha to at most R kept
 * ids, written to out_ids[i*R ..] (-1 padded) with the count in out_cnt[i].
 * X as in fgraft_build_scaffold.  Lists of any length are accepted; the
 * scratch is allocated stream-ordered for the longest one. */
fgraft_status fgraft_prune_lists(const void* X, int64_t n, int32_t d, int64_t ld, int32_t metric,
                                 const int32_t* owner, const int64_t* cand_off,
                                 const int32_t* cand_ids, int64_t nlists, float alpha, int32_t R,
                                 int32_t* out_ids, int32_t* out_cnt, fgraft_stream stream);

/* The list prune above, for callers that cannot allocate device memory at
 * the moment they prune: a serving loop whose latency budget has no room for
 * an allocator call (or for its failure under memory pressure), and a host
 * application that has already handed all device memory to its own pool
 * allocator.  The paper has no counterpart: this is a property of the
 * library, not of the method.
 * Same arguments and results as fgraft_prune_lists, with fixed limits:
 * nlists <= 65536 (EINVAL otherwise, before any work) and at most 4096
 * candidates per list, counted before the owner and repeats are dropped
 * (EINVAL after the call; the rows of such lists are then unspecified, the
 * other rows are correct).  The scratch is one file-scope device array of
 * about 2.4 MiB that every device loading the library keeps until the
 * process exits.  The first call on a device looks up that array's device
 * address once (cudaGetSymbolAddress).  Every call shares the array and it
 * keeps the last call's contents: each call clears what must start at zero,
 * and calls whose work overlaps on the GPU (other streams, other host
 * threads) race on it.  The call synchronises `stream` before returning, to
 * report over-long lists.  It calls no cudaMalloc, cudaFree or allocating
 * library routine. */
fgraft_status fgraft_prune_lists_noalloc(const void* X, int64_t n, int32_t d, int64_t ld,
                                         int32_t metric, const int32_t* owner,
                                         const int64_t* cand_off, const int32_t* cand_ids,
                                         int64_t nlists, float alpha, int32_t R, int32_t* out_ids,
                                         int32_t* out_cnt, fgraft_stream stream);

/* Exact k nearest neighbours of points (Section 2: local completeness, the
 * fraction of a point's true 10-NN that sit in its adjacency row, needs them
 * for every point).  For each point i = row0 .. row0 + nrows - 1, the k
 * smallest (delta(x_i, x_j), j) over all j != i in [0, n), delta the
 * canonical float32 distance: the brute force of Section 2 restricted to the
 * points themselves.  out_ids / out_dist (device, nrows*k, row r = point
 * row0 + r): ids ascending by (delta, id), -1 / +inf past n - 1 neighbours.
 * Computed as a dense product on the tensor cores: all rows rounded to BF16,
 * a Gram pass that finds each row's k-th smallest approximate distance, a
 * second that collects every column within twice the row's rounding bound
 * of it, then the canonical rerank of the collected columns (a row that
 * collected more than 256 scans all n points), so the result equals the
 * float32 brute force exactly.  float32 metrics, 1 <= k <= 32.  stats (host,
 * optional, 4 doubles): canonical evaluations of the rerank, rows that
 * scanned every point, filter and rerank kernel milliseconds.  Scratch
 * (about 256 bytes per point plus 1 KB per query row, at most 64 MB of it)
 * is allocated stream-ordered; the call synchronises `stream` once per
 * 65,536 rows to check its bounded waits (FGRAFT_ETIMEOUT). */
fgraft_status fgraft_knn_exact(const void* X, int64_t n, int32_t d, int64_t ld, int32_t metric,
                               int64_t row0, int64_t nrows, int32_t k, int32_t* out_ids,
                               float* out_dist, double* stats, fgraft_stream stream);

/* Visited-set log (Section 5.5, Table 6: the sets V_i whose overlap decides
 * whether co-scheduled searches could share their work).  Runs the harvest
 * searches of the next block -- the substrate S_b with b = the blocks
 * harvested so far (fgraft_index_sizes) -- for the np query points listed
 * in points (device, int32 ids), and records for each the vertices it
 * evaluates: out_ids[i*cap ..] (device, np*cap int32) receives, in the
 * order of insertion into the visited set, the first min(|V_i|, cap) of them
 * (the tree roots first), and out_cnt[i] (device, np int32) receives |V_i|,
 * or -1 when points[i] is not in [0, n).  A point of block b gets exactly the
 * set its own harvest search evaluates (the harvest's `harvest_evals` sums
 * these sizes); other points are searched on S_b all the same.  Nothing of
 * the index changes: no row, prune or counter of the build.  The call
 * synchronises `stream` to check the searches' scratch (FGRAFT_EOVERFLOW as
 * for the harvest).  np < 2^31, cap >= 1. */
fgraft_status fgraft_harvest_visited(fgraft_index* ix, const int32_t* points, int64_t np,
                                     int32_t cap, int32_t* out_ids, int32_t* out_cnt,
                                     fgraft_stream stream);

/* Query search (Section 2: beam search over the final graph, graded against
 * a brute-force key).  The same beam as the harvest, width ef_s, entering at
 * the T roots; out_ids/out_dist (nq*k) get the first k pool entries (-1 /
 * +inf when fewer were reached); out_evals (nq, optional) the number of
 * distance evaluations of each query.  Q: nq rows of d elements of the
 * index's element type, stride ldq elements (16-byte rule as for X).
 * Requires fgraft_prune to have run.  1 <= k <= ef_s <= 128. */
fgraft_status fgraft_search(fgraft_index* ix, const void* Q, int64_t nq, int64_t ldq, int32_t k,
                            int32_t ef_s, int32_t* out_ids, float* out_dist, uint32_t* out_evals,
                            fgraft_stream stream);

/* Dense-block ceiling (Section 5.3: the pair set fixed in advance that a
 * blocked kernel evaluates at arithmetic rate).  block_ids holds nb blocks of
 * bs ids (-1 = padding; ids of a block distinct).  For every valid member i
 * of a block and every other valid member j, delta(x_i, x_j) is taken, and
 * out_ids/out_dist (nb*bs*k) receive the k smallest (delta, id) per row
 * (-1 / +inf fill).  The result is the canonical float32 top-k whatever the
 * precision:
 *   precision 0  every pair in the canonical float32 order (CUDA cores;
 *                uint8 rows: exact integer distances);
 *   precision 1  BF16 tensor-core filter (tcgen05, FP32 accumulation) on the
 *                block centred on its mean, then every pair within twice a
 *                rounding-error bound of the k-th approximate distance is
 *                recomputed in the canonical order;
 *   precision 2  the same with an FP8 (E4M3) filter, each centred row scaled
 *                so that its largest magnitude is 448 (kind::f8f6f4); its
 *                bound is about 16 times wider, so more pairs are recomputed.
 * The bound of a row comes from the rows' actual rounding residuals
 * (|<q_i,q_j> - <x_i,x_j>| <= |x_i - q_i| max|q| + |x_i| max|x - q|, plus
 * the FP32 accumulation and the canonical float32 rounding), times 2.
 * stats (host, optional, 6 doubles; the call then synchronises `stream`):
 * fraction of pairs recomputed, filter-kernel ms, rerank ms, prep ms
 * (precisions 1 and 2; zeros for precision 0).  When stats[4] is nonzero on
 * entry, stats[4] and stats[5] return, over the recomputed pairs, the largest
 * |approximate - float64| as a fraction of the row's bound and the largest
 * |canonical float32 - float64| (the float64 check slows the rerank).
 * Precisions 1 and 2 take float32 metrics only; bs <= 1024,
 * k <= 64, nb <= 65535.  Precisions 1 and 2 allocate their scratch
 * stream-ordered (about 2 MB per block for up to 64 blocks at a time) and
 * synchronise `stream` once per 64 blocks to check their bounded waits
 * (FGRAFT_ETIMEOUT). */
fgraft_status fgraft_dense_block_dist(const void* X, int64_t n, int32_t d, int64_t ld,
                                      int32_t metric, const int32_t* block_ids, int64_t nb,
                                      int32_t bs, int32_t k, int32_t precision, int32_t* out_ids,
                                      float* out_dist, double* stats, fgraft_stream stream);

/* The dense-block ceiling without any selection (Section 5.3: the blocked
 * kernel's raw pair rate): the tensor-core Gram matrix of every block in
 * BF16 (precision 1) or FP8 (precision 2) on the centred rows, turned into
 * approximate distances and reduced to the smallest one per row:
 * out_min[b * bs + i] = min over valid j != i of the approximate
 * delta(x_i, x_j) (+inf for padding rows and single-member blocks).  The
 * same kernel as the filter of fgraft_dense_block_dist, one pass instead of
 * three.  ms (host, optional) receives the Gram kernel's time; the call then
 * synchronises `stream`.  Arguments as for fgraft_dense_block_dist;
 * float32 metrics only. */
fgraft_status fgraft_dense_block_gram(const void* X, int64_t n, int32_t d, int64_t ld,
                                      int32_t metric, const int32_t* block_ids, int64_t nb,
                                      int32_t bs, int32_t precision, float* out_min, double* ms,
                                      fgraft_stream stream);

/* Inspection: copies of the index's state into caller buffers (device).
 * roots: T; parents: T*n (parent of every point in each tree, -1 at the
 * root); s_offsets: n+1 and s_ids: scaffold size (fgraft_index_sizes);
 * rows: n*R and counts: n (harvested rows).  Any pointer may be NULL. */
fgraft_status fgraft_index_copy(const fgraft_index* ix, int32_t* roots, int32_t* parents,
                                int64_t* s_offsets, int32_t* s_ids, int32_t* rows,
                                int32_t* counts, fgraft_stream stream);

/* Sizes (host outputs): n, T, R, scaffold entries, final-graph entries
 * (0 before fgraft_prune), blocks harvested so far.  Any pointer may be
 * NULL.  Synchronises nothing. */
fgraft_status fgraft_index_sizes(const fgraft_index* ix, int64_t* n, int32_t* T, int32_t* R,
                                 int64_t* scaffold_nnz, int64_t* final_nnz,
                                 int32_t* blocks_done);

/* Cumulative counters of the index (host output; synchronises `stream`). */
fgraft_status fgraft_index_counters(fgraft_index* ix, fgraft_stream stream,
                                    fgraft_counters* counters);

/* Harvest launch configuration (measurement and tuning; results do not
 * depend on it).  The visited set of a search is an n-bit shared-memory
 * bitmap when that is no larger than the hash, else a bucketed hash of
 * 2^hash_log2 slots; giving hash_log2 (7 <= k <= 14) selects the hash of
 * that size.  warps_per_cta: 1..4.  overflow_mode: what a search does when
 * its visited set outgrows the hash: 1 moves it to a per-warp n-bit bitmap
 * in global memory and continues (default), 2 abandons the query and runs it
 * again on global-memory scratch after the launch.  0 leaves a value
 * unchanged. */
fgraft_status fgraft_index_tune(fgraft_index* ix, int32_t hash_log2, int32_t warps_per_cta,
                                int32_t overflow_mode);

/* Autotuner (not in the paper: a property of this implementation).  Times
 * the harvest of a calibration sample -- the first `sample` searches in
 * claim order of the index's next block b (the blocks harvested so far, or
 * block 0 when all are), each with its occlusion prune, on the substrate
 * S_b -- under every
 * candidate launch configuration, keeps the fastest for this index and
 * records it in the process's tuning table under (metric, d, ef_h, R,
 * ceil(log2 n), T, B); later fgraft_build_scaffold calls of the same shape
 * start from it.  The settings: warps (searches) per CTA 4, 2, 1; visited sets by
 * the occupancy rule or in a shared-memory hash of 2^9..2^12 slots;
 * overflowing searches continuing in a global bitmap or re-run; candidate
 * rows gathered into registers by the lane groups or bulk-copied (TMA) into
 * a shared buffer of 32 rows per search (rows of at most 64 chunks); the
 * bitmap visited tests of 1 or 2 chunks of 32 ids issued together.  The
 * search is coordinate descent from the defaults (4, occupancy rule, global
 * bitmap, registers, 2), each setting in turn over its options, two rounds;
 * each candidate is timed as the fastest of three runs of the sample.  The
 * searches of later blocks scan longer neighbour lists (S_b grows with b),
 * so a sample from a middle block represents the whole harvest better than
 * block 0: harvest some blocks of a scratch index first.  Results never
 * depend on the settings: the sample's rows receive their final values (its
 * block's harvest writes the same) and nothing else of the index changes.
 * chosen (host, optional) receives the settings and the microseconds per
 * sample search with them and with the default settings.  Call it before
 * capturing the harvest in a graph; it synchronises `stream`. */
typedef struct {
  int32_t warps_per_cta;
  int32_t hash_log2;      /* 0: the occupancy rule */
  int32_t overflow_mode;  /* 1: continue in a global bitmap, 2: re-run */
  int32_t gather;         /* 0: registers, 1: bulk copies into shared memory */
  int32_t id_batch;       /* 1 or 2 chunks of ids per round of bitmap tests */
  float us_per_query;
  float default_us_per_query;
} fgraft_tuning;
fgraft_status fgraft_index_autotune(fgraft_index* ix, int32_t sample, fgraft_stream stream,
                                    fgraft_tuning* chosen);

/* Explicit harvest launch settings for an index (tuning; results do not
 * depend on them); the timing fields of t are ignored.  EINVAL for a
 * setting out of range (gather = 1 needs rows of at most 64 chunks). */
fgraft_status fgraft_index_set_tuning(fgraft_index* ix, const fgraft_tuning* t);

/* The process's tuning table as a JSON file (path: host string):
 * {"fgraft_tuning": 1, "entries": [{"metric", "d", "ef_h", "R", "log2_n", "T",
 * "B", "warps_per_cta", "hash_log2", "overflow_mode", "gather", "id_batch",
 * "us_per_query"}, ..]} ("gather" and "id_batch" optional: 0 and 2).
 * Loading adds or replaces entries (EINVAL on an unreadable file or an
 * entry with a missing field or a setting out of range, table unchanged). */
fgraft_status fgraft_tuning_table_save(const char* path);
fgraft_status fgraft_tuning_table_load(const char* path);

/* Tensor-core configuration for later builds, harvests and final graphs in
 * this process (tuning; results do not depend on it).  With tensor_cores = 1
 * (the default), under a float32 metric, the dominance tests of an occlusion
 * prune of at most 128 candidates and the SAT's closest-child choices are
 * decided from TF32 Gram tiles computed by tcgen05.mma, and every decision
 * the Gram value cannot fix within its error bound is recomputed in canonical
 * float32 (the prune of Section 3 and the tree of Section 1 are unchanged);
 * with 0 every distance is computed in canonical float32 by lane groups.
 * FGRAFT_EINVAL for other values. */
fgraft_status fgraft_tune_prune(int32_t tensor_cores);

/* Scaffold degree cap for later fgraft_build_scaffold calls in this process
 * (Section 6: the ablation the paper reports as negative).  With cap > 0
 * every row of S_0 longer than cap keeps its cap nearest entries by
 * (delta(u, v), v), rows sorted by id; the final graph's tree-0 spine and the
 * entry roots are unchanged.  0 (the default) turns it off.  The distances
 * the cap evaluates are not in any counter.  FGRAFT_EINVAL for cap < 0. */
fgraft_status fgraft_tune_scaffold_cap(int32_t cap);

/* Failure handling (tuning and tests; results do not depend on it unless a
 * wait gives up).  Every kernel that waits on the tensor cores (the TF32
 * prune of Section 3, the SAT's closest-child choice of Section 1, the dense
 * blocks of Section 5.3) polls its MMA-completion barrier at most `polls`
 * times (the prune bounds by the same count the waits with which its compute
 * threads and its walker warp pass list slots to each other) before it gives
 * up, sets an error flag, waits for its products in
 * flight with the full bound (2^22 polls), frees its tensor memory and
 * returns; the call that reads the flag returns FGRAFT_ETIMEOUT
 * (fgraft_build_scaffold, fgraft_harvest_block with counters, fgraft_prune,
 * fgraft_index_counters, fgraft_dense_block_dist).  polls = 0 gives up at
 * the first wait, which tests that path without a fault; -1 restores the
 * default of 2^22 polls.  Applies to later launches in this process.
 * FGRAFT_EINVAL for polls < -1. */
fgraft_status fgraft_tune_mma_wait(int32_t polls);

/* SAT launch configuration for later fgraft_build_scaffold calls in this
 * process (tuning; results do not depend on it): tree nodes holding at least
 * big_node_min points are split across many CTAs, one launch per child
 * selection, until the list of points no child has rejected yet is at most
 * finish_len long for every such node; then one CTA per node finishes the
 * selection.  Smaller nodes get one CTA each from the start.
 * Defaults 16384 and 512; big_node_min >= 2, finish_len >= 1; 0 leaves a
 * value unchanged. */
fgraft_status fgraft_tune_sat(int32_t big_node_min, int32_t finish_len);

/* Harvest schedule for later fgraft_build_scaffold calls in this process
 * (tuning; the rows of a block are independent given S_b, Section 4, so the
 * graph does not depend on it).  With coherent = 1 the searches of each
 * block are claimed in a preorder of SAT tree 0, so the searches in flight
 * together are neighbours that evaluate many of the same targets (Section
 * 5.5, Table 6) and share their loads through the L2 cache; with 0 they run
 * in id order; with 2 (the default) the preorder is used when the vectors
 * are larger than the device's L2 cache.  The schedule falls back to id
 * order when B > 64 or tree 0 is deeper than 4096.  FGRAFT_EINVAL for other
 * values. */
fgraft_status fgraft_tune_schedule(int32_t coherent);

/* The schedule of an index (inspection).  pre (device, n int32): the place
 * of every point in the preorder of tree 0; qorder (device, n int32): for
 * blocks b = 0..B-1 one after another, the indices i of the points
 * b + i * B of block b in the order their searches are claimed.  Both are
 * left untouched, and *coherent (host, optional) is 0, when the index runs
 * in id order; otherwise *coherent is 1.  Any pointer may be NULL. */
fgraft_status fgraft_index_schedule(const fgraft_index* ix, int32_t* pre, int32_t* qorder,
                                    int32_t* coherent, fgraft_stream stream);

/* Measurement hooks (results never depend on them).
 * fgraft_index_profile: with enable != 0, every later harvest of a block
 * records a CUDA event pair around its harvest kernel on the launching
 * stream (inside a captured graph too).
 * fgraft_index_harvest_ms: synchronises `stream` and returns in *ms the sum
 * of those kernel durations over the blocks harvested so far, in *launches
 * (optional) their number, and in *prune_ms (optional) the summed time from
 * the end of each harvest kernel to the end of its block's prune kernel (the
 * re-run pass and the occlusion prune).
 * fgraft_kernel_launches: kernels launched by the library in this process
 * so far (a graph replay counts the kernels it holds). */
fgraft_status fgraft_index_profile(fgraft_index* ix, int32_t enable);
fgraft_status fgraft_index_harvest_ms(fgraft_index* ix, fgraft_stream stream, double* ms,
                                      int32_t* launches, double* prune_ms);
uint64_t fgraft_kernel_launches(void);

void fgraft_index_destroy(fgraft_index* ix);

/* Message of the last non-OK status returned on this host thread. */
const char* fgraft_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FGRAFT_H */
