// Host-side declarations shared by the translation units of libfgraft.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

namespace fg {

// Status plumbing: the C ABI maps these to fgraft_status.
struct Err {
  int code;  // fgraft_status value
  std::string msg;
};

void set_error(int code, const std::string& msg);

// Process-wide count of kernel launches issued by the library (measurement).
void note_launch(uint64_t k = 1);
uint64_t launch_count();
void set_launch_count(uint64_t v);
int cuda_fail(cudaError_t e, const char* what);
// Raises the dynamic shared memory limit of kernel fn on the current device
// to at least bytes; never lowers it, since a graph captured earlier may
// launch the same kernel with more.
cudaError_t raise_smem_limit(const void* fn, int bytes);

#define FG_STR2(x) #x
#define FG_STR(x) FG_STR2(x)
#define FG_CUDA(call)                                                                 \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call " at " __FILE__ ":" FG_STR(__LINE__)); \
  } while (0)

// Vector layout of a point set for the kernels.
struct VecLayout {
  const char* X;
  int64_t n;
  int32_t d;
  int64_t ld_bytes;
  int32_t metric;
  int32_t nchunks;  // 16-byte chunks covering d elements
  int32_t G, K;     // lanes per vector and chunks per lane
};

// Picks the lane-group shape for a metric and dimension; false if unsupported.
bool choose_shape(int metric, int d, int* G, int* K);

// Exclusive scan of n uint32 counts into n+1 int64 offsets (out[n] = total).
// tmp must hold scan_tmp_elems(n) int64.
int64_t scan_tmp_elems(int64_t n);
int scan_u32(const uint32_t* in, int64_t* out, int64_t n, int64_t* tmp, cudaStream_t s);

// SAT forest: parents [T*n] (-1 at each root), sat work counter added to ctr.
struct SatScratch {
  int32_t* node_of;     // T*n
  uint32_t* kcnt;       // T*n (zero on entry and exit)
  int64_t* kstart;      // T*n + 1
  int32_t* item_pt;     // T*n
  uint64_t* lst;        // 2*T*n (open lists)
  uint64_t* best;       // T*n
  int32_t* kid;         // T*n (children of a node at the start of its item range)
  int32_t* seg_k;       // like seg_start (children per node)
  int64_t* seg_start;   // T*n + T*n/big_min + 1 (small nodes first, big ones from T*n)
  int32_t* seg_len;     // same
  int32_t* seg_node;    // same
  int32_t* seg_tree;    // same
  uint32_t* nseg;       // 7: tiny, big nodes of the level, error flag, other nodes,
                        //    tensor-core timeout flag, most points of other / big nodes
  int64_t* scan_tmp;
  int32_t big_min;      // nodes with at least this many points use the multi-CTA path
  int32_t* big_list;    // segment index of each big node
  uint64_t* big_keys;   // 3 per big node
  uint32_t* big_kcount; // 1 per big node
  uint32_t* big_lens;   // 3 per big node
  int32_t finish_len;   // open lists this short finish in one CTA per node
};
int sat_forest(const VecLayout& L, int T, const int32_t* roots_d, int32_t* parents,
               SatScratch& S, unsigned long long* ctr_sat, cudaStream_t s);

// Scaffold CSR from the parents of T trees (rows sorted by id, no repeats;
// with cap > 0 a row longer than cap keeps its cap nearest entries, Section
// 6).  tmp_off: n+1, tmp_ids: 2*T*n, ucnt: n, deg: n.  On return *nnz_out
// holds the size and s_ids (allocated here with cudaMalloc) the ids.
int scaffold_csr(int64_t n, int T, const int32_t* parents, int64_t* s_off, int32_t** s_ids,
                 int64_t* nnz_out, uint32_t* deg, int64_t* tmp_off, int32_t* tmp_ids,
                 int64_t* scan_tmp, cudaStream_t s, const VecLayout* L, int cap);

// Reverse lists of the rows of blocks 0..b: r_off (n+1), r_ids (<= n*R);
// with Ad and r_d given, r_d[k] = delta(u, r_ids[k]) beside each reverse id
// (the distance its row holds: the canonical distance is symmetric).
int reverse_rows(int64_t n, int R, int nb, int b, const int32_t* A, const int32_t* cnt,
                 uint32_t* rcnt, uint32_t* rcur, int64_t* r_off, int32_t* r_ids,
                 int64_t* scan_tmp, cudaStream_t s, const float* Ad = nullptr,
                 float* r_d = nullptr);

// Final graph (rows of all blocks symmetrised, re-pruned when over R, tree-0
// spine added, sorted).  f_ids is (re)allocated here.  Ad / r_d (optional):
// the distances beside the rows' and the reverse lists' ids, so that the
// candidate keys need no evaluation.
int final_graph(const VecLayout& L, int R, float alpha2, const int32_t* A, const int32_t* cnt,
                const int64_t* r_off, const int32_t* r_ids, const int32_t* parent0,
                int64_t* f_off, int32_t** f_ids, int64_t* f_nnz, int64_t* scan_tmp,
                unsigned long long* ctr, int num_sms, cudaStream_t s,
                const float* Ad = nullptr, const float* r_d = nullptr);

// Batched occlusion prune of explicit candidate lists.
int prune_lists(const VecLayout& L, const int32_t* owner, const int64_t* l_off,
                const int32_t* l_ids, int64_t nlists, float alpha2, int R, int32_t* out_ids,
                int32_t* out_cnt, unsigned long long* ctr, cudaStream_t s);

// The list prune on a fixed, file-scope device scratch array (no allocation).
int prune_lists_static(const VecLayout& L, const int32_t* owner, const int64_t* l_off,
                       const int32_t* l_ids, int64_t nlists, float alpha2, int R,
                       int32_t* out_ids, int32_t* out_cnt, cudaStream_t s);
int64_t prune_lists_static_max_lists();
int prune_lists_static_max_len();

// Harvest prune as its own kernel over the expanded lists the search wrote.
// With rows non-null the lists are the final graph's: list qidx belongs to
// point rows[qidx], its keys start at Eg + Eg_off[point], the list count is
// read from *nq_dev, and the kept keys go to K_out[qidx * R ...] with their
// count in cnt_out[qidx].
int harvest_prune_smem(int ecap, int nchunks);
int harvest_prune(const VecLayout& L, const uint64_t* Eg, const int32_t* Eg_cnt, int ecap,
                  int64_t nq, int64_t q_first, int64_t q_step, int R, float alpha2,
                  int32_t* A_out, int32_t* cnt_out, unsigned long long* prune_ctr, int num_sms,
                  cudaStream_t s, const int32_t* rows = nullptr, const int64_t* Eg_off = nullptr,
                  const uint32_t* nq_dev = nullptr, uint64_t* K_out = nullptr,
                  uint32_t* err = nullptr, int32_t* long_list = nullptr,
                  uint32_t* long_cnt = nullptr, const int32_t* qlist = nullptr,
                  float* D_out = nullptr);
// (qlist: work item w < nq is the list of qidx = qlist[w]; NULL: qidx = w.)
// Dominance bits of the prune on the tensor cores (1, the default, for the
// float32 metrics and lists of at most 128 when err is given) or on the lane
// groups (0).  The pruned lists are the same either way.
extern int g_prune_tc;
// The same for the SAT's closest-child assignment.
extern int g_sat_tc;
// Polls of the first bounded wait of a tensor-core CTA for its MMA products
// (default 2^22).  When it gives up, the CTA sets its error flag, waits for
// the products in flight with the full bound kDrainPolls, frees its tensor
// memory and returns; the host reports FGRAFT_ETIMEOUT.
extern int g_mma_wait_polls;
// Harvest launch settings chosen by the autotuner, by (metric, d, ef_h, R,
// ceil(log2 n)); hash_log2 0 keeps the occupancy rule for the visited sets.
struct TuneKey {
  int metric, d, ef, R, log2_n, T, B;
};
struct TuneVal {
  int wpc, hash_log2, overflow, gather, id_batch;
  float us_per_query;
};
bool tune_table_lookup(const TuneKey& k, TuneVal* v);
void tune_table_put(const TuneKey& k, const TuneVal& v);
int tune_table_size();
int tune_table_save(const char* path);
int tune_table_load(const char* path);

// Streaming multiprocessors of the current device (cached per device; 1 if
// the query fails).  Grid caps of the grid-stride kernels are multiples of it.
int device_sms();
constexpr int kDrainPolls = 1 << 22;

// Coherent harvest schedule (Section 5.5): pre[v] = the place of v in a
// preorder of the tree given by parent (-1 at its root; siblings in no fixed
// order), qorder = for blocks b = 0..nb-1 one after another, the query
// indices i of the points b + i * nb of block b in preorder.  Sets *ok =
// false and writes neither output when nb > 64, parent is not a forest, or
// it is deeper than max_depth (one launch per depth).
int coherent_schedule(int64_t n, const int32_t* parent, int nb, int max_depth, int32_t* pre,
                      int32_t* qorder, cudaStream_t s, bool* ok);
extern int g_coherent;

// Dense-block top-k with the BF16 or FP8 tensor-core filter and canonical
// rerank; stats (host, optional): rerank fraction, Gram ms, select ms, prep
// ms, and with err64 the float64 error maxima over the reranked pairs.
int dense_block_tc(const VecLayout& L, const int32_t* block_ids, int64_t nb, int bs, int k,
                   int fp8, bool err64, int32_t* out_ids, float* out_dist, double* stats,
                   cudaStream_t s);

// Gram and approximate distances of every pair of the blocks on the tensor
// cores, reduced to the smallest approximate distance per row (out_min,
// nb * bs floats; +inf for padding rows); *ms (optional) gets the kernel's
// time.  Measures the dense ceiling without any selection.
int dense_gram_tc(const VecLayout& L, const int32_t* block_ids, int64_t nb, int bs, int fp8,
                  float* out_min, double* ms, cudaStream_t s);
// Exact k nearest neighbours of points row0 .. row0 + nrows - 1 among all
// points (self excluded): BF16 tensor-core filter, canonical rerank.
int knn_tc(const VecLayout& L, int64_t row0, int64_t nrows, int k, int32_t* out_ids,
           float* out_dist, double* stats, cudaStream_t s);

// Dense-block top-k (canonical float32 distances of every pair of a block).
int dense_block(const VecLayout& L, const int32_t* block_ids, int64_t nb, int bs, int k,
                int32_t* out_ids, float* out_dist, cudaStream_t s);

}  // namespace fg
