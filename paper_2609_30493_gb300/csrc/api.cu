// C ABI of libfgraft: argument checks, the index object, and the host-side
// sequencing of the kernels (SAT levels, harvest blocks with their overflow
// re-run and reverse-list update, final graph, search, dense blocks).
#include <array>
#include <atomic>
#include <map>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/fgraft.h"
#include "beam.cuh"
#include "internal.h"

namespace fg {

static thread_local std::string g_err;
static thread_local int g_err_code = 0;

void set_error(int code, const std::string& msg) {
  g_err_code = code;
  g_err = msg;
}

static std::atomic<uint64_t> g_launches{0};
void note_launch(uint64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
uint64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }
void set_launch_count(uint64_t v) { g_launches.store(v, std::memory_order_relaxed); }

cudaError_t raise_smem_limit(const void* fn, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> limits;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  int& cur = limits[{dev, fn}];
  if (bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

int device_sms() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1)
    return 1;
  cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

int cuda_fail(cudaError_t e, const char* what) {
  set_error(FGRAFT_ECUDA, std::string(what) + ": " + cudaGetErrorName(e) + " (" +
                              cudaGetErrorString(e) + ")");
  return FGRAFT_ECUDA;
}

bool choose_shape(int metric, int d, int* G, int* K) {
  if (d < 1) return false;
  if (metric == L2_U8) {
    if (d > 256) return false;
    const int nch = (d + 15) / 16;
    *K = 1;
    *G = nch <= 4 ? 4 : (nch <= 8 ? 8 : 16);
    return true;
  }
  if (metric != L2_F32 && metric != ANGULAR_F32) return false;
  if (d > 1024) return false;
  const int nch = (d + 3) / 4;
  if (nch <= 32) {
    *K = 1;
    *G = nch <= 4 ? 4 : (nch <= 8 ? 8 : (nch <= 16 ? 16 : 32));
  } else {
    *G = 32;
    const int k = (nch + 31) / 32;
    *K = k <= 2 ? 2 : (k <= 4 ? 4 : 8);
  }
  return true;
}

// splitmix64 (Steele, Lea and Flood, OOPSLA 2014): first output of the
// generator started at state z.  Keys the tree roots.
static uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static void keyed_roots(uint64_t seed, int T, int64_t n, std::vector<int32_t>& roots) {
  roots.resize(T);
  for (int t = 0; t < T; ++t) {
    const uint64_t base = seed ^ (0x9E3779B97F4A7C15ULL * (uint64_t)(t + 1));
    for (uint64_t j = 0;; ++j) {
      const int32_t r = (int32_t)(splitmix64(base + j) % (uint64_t)n);
      bool dup = false;
      for (int s = 0; s < t; ++s) dup |= roots[s] == r;
      if (!dup) {
        roots[t] = r;
        break;
      }
    }
  }
}

}  // namespace fg

using namespace fg;

// Nodes of at least this many points are built by the multi-CTA SAT path.
int fg::g_mma_wait_polls = 1 << 22;
static int32_t g_sat_big_min = 16384;
static int32_t g_sat_finish_len = 512;
static int32_t g_scaffold_cap = 0;  // 0: no degree cap
static constexpr int kCoherentMaxDepth = 4096;

#define FGS(call)                                                      \
  do {                                                                 \
    cudaError_t e_ = (call);                                           \
    if (e_ != cudaSuccess) \
      return (fgraft_status)cuda_fail(e_, #call " at " __FILE__ ":" FG_STR(__LINE__)); \
  } while (0)

enum CtrSlot {
  C_HARVEST = 0,
  C_EXPANSIONS = 1,
  C_PRUNE = 2,
  C_SCANNED = 3,
  C_RERUNS = 4,
  C_SAT = 5,
  C_FINAL = 6,
  C_SEARCH = 8,  // search-side slots 8..12 (same layout as 0..4)
  C_VLOG = 16,   // visited-set logs, slots 16..20 (same layout)
  C_COUNT = 24
};

struct fgraft_index {
  VecLayout L;
  fgraft_params p;
  int32_t nb;
  int64_t ld;
  std::vector<int32_t> roots_h;
  int32_t* roots = nullptr;
  int32_t* parents = nullptr;
  int64_t* s_off = nullptr;
  int32_t* s_ids = nullptr;
  int64_t s_nnz = 0;
  int32_t* A = nullptr;
  float* Ad = nullptr;    // delta(p, A[p][i]) beside each harvested id
  float* r_d = nullptr;   // delta(u, r_ids[k]) beside each reverse id (final rebuild)
  int32_t* cnt = nullptr;
  int64_t* r_off = nullptr;
  int32_t* r_ids = nullptr;
  uint32_t* rcnt = nullptr;
  uint32_t* rcur = nullptr;
  int64_t* f_off = nullptr;
  int32_t* f_ids = nullptr;
  int64_t f_nnz = 0;
  bool final_done = false;  // the final graph is computed (it never changes after)
  int64_t* scan_tmp = nullptr;
  // [0] smem pass, [1] re-run pass, [2] ovf count, [3] err flag, [4] prune
  // timeout, [5] long prune lists, [6] gather timeout
  uint32_t* work = nullptr;
  int32_t* ovf_list = nullptr;
  int64_t ovf_cap = 0;
  char* gscratch = nullptr;
  int64_t gscratch_per_warp = 0;
  int32_t g_ecap = 0;
  int32_t g_warps = 0;
  unsigned long long* ctr = nullptr;
  int32_t blocks_done = 0;
  int32_t hash_log2 = 12;
  bool bitmap_ok = true;
  bool hash_auto = true;       // visited-set layout chosen by occupancy (no explicit hash size)
  int32_t overflow_mode = 1;   // 1: continue in a global bitmap, 2: abandon and re-run
  int32_t gather = 0;          // 1: candidate rows bulk-copied into shared memory
  int32_t id_batch = 2;        // chunks of 32 ids whose bitmap tests go together
  uint64_t* Eg = nullptr;      // expanded lists handed from the search to the prune kernel
  int32_t* Eg_cnt = nullptr;
  int32_t eg_ecap = 0;
  int32_t prune_ns = 0;        // candidates staged per warp by the prune kernel (0: prune in place)
  uint32_t* gvbits = nullptr;  // per-warp global bitmaps for visited sets that outgrow the hash
  int64_t gvbits_words = 0;
  int64_t gvbits_warps = 0;
  int32_t wpc = 4;
  int32_t num_sms = 0;
  cudaGraphExec_t graph_exec = nullptr;
  uint64_t graph_kernels = 0;
  bool profile = false;
  std::vector<cudaEvent_t> ev_beg, ev_end;  // around the harvest kernel of each block
  std::vector<cudaEvent_t> ev_pend;         // after the prune kernel of each block
  int32_t* pre = nullptr;     // place of each point in the preorder of tree 0 (coherent schedule)
  int32_t* qorder = nullptr;  // query indices of every block in that preorder, block after block
};

namespace {

int fail(int code, const std::string& msg) {
  set_error(code, msg);
  return code;
}

int check_vectors(const void* X, int64_t n, int32_t d, int64_t ld, int32_t metric,
                  VecLayout* L) {
  if (!X) return fail(FGRAFT_EINVAL, "X is NULL");
  if (n < 1 || n >= 2147483647LL) return fail(FGRAFT_EINVAL, "n must be in [1, 2^31-2]");
  int G, K;
  if (!choose_shape(metric, d, &G, &K))
    return fail(FGRAFT_EINVAL, "unsupported metric/d (float32: 1<=d<=1024, uint8: 1<=d<=256)");
  const int es = metric == L2_U8 ? 1 : 4;
  if (ld < d) return fail(FGRAFT_EINVAL, "ld < d");
  if ((ld * es) % 16 != 0) return fail(FGRAFT_EINVAL, "row stride must be a multiple of 16 bytes");
  if (reinterpret_cast<uintptr_t>(X) % 16 != 0)
    return fail(FGRAFT_EINVAL, "X must be 16-byte aligned");
  L->X = static_cast<const char*>(X);
  L->n = n;
  L->d = d;
  L->ld_bytes = ld * es;
  L->metric = metric;
  L->nchunks = (int32_t)((d * es + 15) / 16);
  L->G = G;
  L->K = K;
  return 0;
}

BeamKernelFn beam_kernel_for(int metric, int G, int K, int S, bool gather = false) {
  if (gather) {
    if (metric == 0) return beam_kernel_metric0_gather(G, K, S);
    if (metric == 1) return beam_kernel_metric1_gather(G, K, S);
    return beam_kernel_metric2_gather(G, K, S);
  }
  if (metric == 0) return beam_kernel_metric0(G, K, S);
  if (metric == 1) return beam_kernel_metric1(G, K, S);
  return beam_kernel_metric2(G, K, S);
}

int pool_slots(int ef) { return ef <= 32 ? 1 : (ef <= 64 ? 2 : 4); }

int ceil_log2(int64_t v) {
  int k = 0;
  while ((1ll << k) < v) ++k;
  return k;
}

// Inside a stream capture a plain event record only marks a dependency; the
// external flag makes it a timed event-record node of the graph.
cudaError_t record_event(cudaEvent_t e, cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  cudaError_t err = cudaStreamIsCapturing(s, &st);
  if (err != cudaSuccess) return err;
  if (st == cudaStreamCaptureStatusActive) return cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
  return cudaEventRecord(e, s);
}

// Visited-set layout, per-warp shared memory and CTAs per SM of the beam
// kernel for a pool of S slots.  With an explicit hash size the n-bit bitmap
// is used when it is no larger than the hash.  Otherwise the search prefers
// the bitmap (exact, never full) when it keeps the CTAs per SM that the
// smallest hash allows, else the largest hash of 2^7..2^12 slots that keeps
// them: a search whose visited set outgrows the hash goes on in a global
// bitmap, and the harvest is bound by the latency of its dependent loads, so
// searches in flight matter more than hash hits (at n = 1.18M, d = 100 the
// 2^12-slot hash allows 12 warps per SM and 2^11 the register limit of 16,
// 27 % faster).
struct BeamShape {
  bool bitmap = false;
  int nslots = 0, ecap = 0, vis_bytes = 0, wbytes = 0, per_sm = 0;
};

int beam_shape(fgraft_index* ix, BeamKernelFn kern, int S, BeamShape* out) {
  const int64_t bm_bytes = ((ix->L.n + 127) / 128) * 16;
  const int ecap = 1 << std::max(6, ceil_log2(2 * 32 * S));
  const int fixed = 8 * ecap + (ecap / 8 + 15) / 16 * 16 + 256 + 16 * ix->L.nchunks +
                    (ix->gather ? 32 * 16 * ix->L.nchunks + 16 : 0);
  int dev = 0, optin = 0;
  FG_CUDA(cudaGetDevice(&dev));
  FG_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  auto eval = [&](bool bitmap, int nslots, BeamShape* sh) -> int {
    sh->bitmap = bitmap;
    sh->nslots = nslots;
    sh->ecap = ecap;
    sh->vis_bytes = bitmap ? (int)bm_bytes : 4 * nslots;
    sh->wbytes = sh->vis_bytes + fixed;
    sh->per_sm = 0;
    if ((int64_t)sh->wbytes * ix->wpc > optin) return 0;
    FG_CUDA(raise_smem_limit(reinterpret_cast<const void*>(kern), sh->wbytes * ix->wpc));
    FG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&sh->per_sm, kern, ix->wpc * 32,
                                                          sh->wbytes * ix->wpc));
    return 0;
  };
  int rc = 0;
  if (!ix->hash_auto) {
    const int nslots = 1 << ix->hash_log2;
    return eval(ix->bitmap_ok && bm_bytes <= 4ll * nslots, nslots, out);
  }
  BeamShape best, c;
  if ((rc = eval(false, 1 << 7, &best))) return rc;
  if (bm_bytes <= optin) {
    if ((rc = eval(true, 0, &c))) return rc;
    if (c.per_sm >= best.per_sm && c.per_sm > 0) {
      *out = c;
      return 0;
    }
  }
  for (int k = 12; k > 7; --k) {
    if ((rc = eval(false, 1 << k, &c))) return rc;
    if (c.per_sm >= best.per_sm && c.per_sm > 0) {
      *out = c;
      return 0;
    }
  }
  *out = best;
  return 0;
}

int launch_rerun(fgraft_index* ix, BeamArgs a, unsigned long long* ctr, cudaStream_t s);

// Launch the beam over `nq` work items (shared-memory pass), then the
// overflow list on global scratch.  `a` carries everything but the scratch.
int launch_beam(fgraft_index* ix, BeamArgs a, unsigned long long* ctr, cudaStream_t s,
                cudaEvent_t e0 = nullptr, cudaEvent_t e1 = nullptr) {
  const int S = pool_slots(a.ef);
  BeamKernelFn kern = beam_kernel_for(ix->L.metric, ix->L.G, ix->L.K, S, ix->gather != 0);
  if (!kern) return fail(FGRAFT_EINVAL, "no beam kernel for this metric and dimension");
  BeamShape sh;
  int rc = beam_shape(ix, kern, S, &sh);
  if (rc) return rc;
  const int ecap = sh.ecap, nslots = sh.nslots, vis_bytes = sh.vis_bytes, wbytes = sh.wbytes;
  const bool bitmap = sh.bitmap;
  const int qbytes = 16 * ix->L.nchunks;  // staged query (then c* in the prune)
  const int smem = wbytes * ix->wpc;
  const int per_sm = sh.per_sm;
  if (per_sm < 1) return fail(FGRAFT_EINVAL, "harvest launch does not fit an SM");
  a.counters = ctr;
  a.work = ix->work;
  a.ovf_list = ix->ovf_list;
  a.ovf_count = ix->work + 2;
  a.ovf_cap = (uint32_t)ix->ovf_cap;
  a.err_flag = ix->work + 3;
  a.hash_log2 = ceil_log2(std::max(nslots, 1 << 7));
  a.bitmap = bitmap ? 1 : 0;
  a.vis_bytes = vis_bytes;
  a.vis_cap = bitmap ? INT32_MAX : (int32_t)(0.8 * nslots) - 32;
  a.ecap = ecap;
  // visited sets that outgrow the hash continue in per-warp global bitmaps
  // (sized for the largest harvest grid when the index is built or tuned)
  const int64_t grid_warps = (int64_t)per_sm * ix->num_sms * ix->wpc;
  const bool migrate = !bitmap && ix->overflow_mode == 1 && grid_warps <= ix->gvbits_warps;
  a.gvbits = migrate ? ix->gvbits : nullptr;
  a.gvbits_words = ix->gvbits_words;
  a.wbytes = wbytes;
  a.qbytes = qbytes;
  a.global_scratch = 0;
  a.gather = ix->gather;
  a.id_batch = ix->id_batch;
  a.wait_polls = g_mma_wait_polls;
  // the per-warp layout must be complete before any launch
  if (a.wbytes < a.vis_bytes + 8 * a.ecap + 256 + a.qbytes +
                     (a.gather ? 32 * a.qbytes + 16 : 0) ||
      a.qbytes < 16 * ix->L.nchunks)
    return fail(FGRAFT_EINVAL, "internal: harvest shared-memory layout incomplete");
  FG_CUDA(cudaMemsetAsync(ix->work, 0, 3 * sizeof(uint32_t), s));
  if (e0) FG_CUDA(record_event(e0, s));
  kern<<<per_sm * ix->num_sms, ix->wpc * 32, smem, s>>>(a);
  note_launch();
  FG_CUDA(cudaGetLastError());
  if (e1) FG_CUDA(record_event(e1, s));
  return launch_rerun(ix, a, ctr, s);
}

// Re-run of the work items a harvest or search launch of index ix abandoned
// (listed in ix->ovf_list, count ix->work[2]) with per-warp global scratch,
// pruned in place.  `a` is that launch's descriptor.
int launch_rerun(fgraft_index* ix, BeamArgs a, unsigned long long* ctr, cudaStream_t s) {
  const int S = pool_slots(a.ef);
  BeamKernelFn kern_rr = beam_kernel_for(ix->L.metric, ix->L.G, ix->L.K, S, false);
  if (!kern_rr) return fail(FGRAFT_EINVAL, "no beam kernel for this metric and dimension");
  const int qbytes = 16 * ix->L.nchunks;
  a.global_scratch = 1;
  a.Eg = nullptr;
  a.Eg_cnt = nullptr;
  a.qlist = ix->ovf_list;
  a.qlist_len = ix->work + 2;
  a.work = ix->work + 1;
  a.hash_log2 = 7;
  a.bitmap = 1;  // this warp's n-bit bitmap in gvbits: exact, never full
  a.vis_bytes = (int32_t)(4 * ix->gvbits_words);
  a.vis_cap = INT32_MAX;
  a.gvbits = ix->gvbits;
  a.gvbits_words = ix->gvbits_words;
  a.ecap = ix->g_ecap;
  a.wbytes = 256 + qbytes;
  a.gather = 0;
  if (ix->gvbits_warps < ix->g_warps || !ix->gvbits)
    return fail(FGRAFT_EINVAL, "internal: re-run bitmaps missing");
  a.gscratch = ix->gscratch;
  a.gscratch_per_warp = ix->gscratch_per_warp;
  a.counters = ctr;
  kern_rr<<<ix->g_warps / 4, 128, a.wbytes * 4, s>>>(a);
  note_launch();
  FG_CUDA(cudaGetLastError());
  return 0;
}

// Per-warp n-bit bitmaps for visited sets that outgrow the shared-memory
// hash: enough warps for the largest harvest or search grid at the current
// tuning (and for the re-run pass).  Not called during stream capture.
int size_visited_bitmaps(fgraft_index* ix) {
  int64_t need = ix->g_warps;
  for (int S = 1; S <= 4; S *= 2) {
    BeamKernelFn kern = beam_kernel_for(ix->L.metric, ix->L.G, ix->L.K, S, ix->gather != 0);
    if (!kern) continue;
    BeamShape sh;
    const int rc = beam_shape(ix, kern, S, &sh);
    if (rc) return rc;
    need = std::max<int64_t>(need, (int64_t)sh.per_sm * ix->num_sms * ix->wpc);
  }
  if (need <= ix->gvbits_warps) return 0;
  if (ix->gvbits) cudaFree(ix->gvbits);
  ix->gvbits = nullptr;
  ix->gvbits_warps = 0;
  ix->gvbits_words = (ix->L.n + 127) / 128 * 4;
  cudaError_t e = cudaMalloc(&ix->gvbits, sizeof(uint32_t) * ix->gvbits_words * need);
  if (e != cudaSuccess) {
    set_error(FGRAFT_ENOMEM, std::string("cudaMalloc(visited bitmaps): ") + cudaGetErrorString(e));
    return FGRAFT_ENOMEM;
  }
  ix->gvbits_warps = need;
  return 0;
}

int check_err_flag(fgraft_index* ix, cudaStream_t s) {
  uint32_t f[4] = {0, 0, 0, 0};
  FG_CUDA(cudaMemcpyAsync(f, ix->work + 3, sizeof(f), cudaMemcpyDeviceToHost, s));
  FG_CUDA(cudaStreamSynchronize(s));
  if (f[0]) return fail(FGRAFT_EOVERFLOW, "a search outgrew its global-memory scratch");
  if (f[1]) return fail(FGRAFT_ETIMEOUT, "a tensor-core prune timed out waiting for its products");
  if (f[3]) return fail(FGRAFT_ETIMEOUT, "a search's bulk copies of candidate rows timed out");
  return 0;
}

int read_counters(fgraft_index* ix, cudaStream_t s, fgraft_counters* c) {
  unsigned long long h[C_COUNT];
  FG_CUDA(cudaMemcpyAsync(h, ix->ctr, sizeof(h), cudaMemcpyDeviceToHost, s));
  FG_CUDA(cudaStreamSynchronize(s));
  c->sat_evals = h[C_SAT];
  c->harvest_evals = h[C_HARVEST];
  c->prune_evals = h[C_PRUNE];
  c->final_prune_evals = h[C_FINAL];
  c->expansions = h[C_EXPANSIONS];
  c->ids_scanned = h[C_SCANNED];
  c->reruns = h[C_RERUNS];
  return check_err_flag(ix, s);
}

template <typename T>
int dalloc(T** p, int64_t count) {
  cudaError_t e = cudaMalloc(p, sizeof(T) * (size_t)std::max<int64_t>(count, 1));
  if (e != cudaSuccess) {
    set_error(FGRAFT_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    return FGRAFT_ENOMEM;
  }
  return 0;
}

// Stream-ordered scratch: the device's default memory pool keeps what it has
// reserved (release threshold raised once per device), so the scratch of a
// repeated build or prune is served without new mappings or device syncs.
static void keep_pool_reserved() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  done[dev] = true;
}

template <typename T>
int dalloc_async(T** p, int64_t count, cudaStream_t s) {
  cudaError_t e = cudaMallocAsync(p, sizeof(T) * (size_t)std::max<int64_t>(count, 1), s);
  if (e != cudaSuccess) {
    *p = nullptr;
    set_error(FGRAFT_ENOMEM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
    return FGRAFT_ENOMEM;
  }
  return 0;
}

void free_index(fgraft_index* ix) {
  if (!ix) return;
  if (ix->graph_exec) cudaGraphExecDestroy(ix->graph_exec);
  for (cudaEvent_t e : ix->ev_beg) cudaEventDestroy(e);
  for (cudaEvent_t e : ix->ev_end) cudaEventDestroy(e);
  for (cudaEvent_t e : ix->ev_pend) cudaEventDestroy(e);
  void* ptrs[] = {ix->roots, ix->parents, ix->s_off, ix->s_ids, ix->A,   ix->cnt, ix->Ad, ix->r_d,
                  ix->r_off, ix->r_ids,   ix->rcnt,  ix->rcur,  ix->f_off, ix->f_ids,
                  ix->scan_tmp, ix->work, ix->ovf_list, ix->gscratch, ix->ctr, ix->gvbits,
                  ix->Eg, ix->Eg_cnt, ix->pre, ix->qorder};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  delete ix;
}

// Harvest launch settings of an index (visited-set layout, warps per CTA,
// overflow handling); hash_log2 0 selects the occupancy rule.
void apply_settings(fgraft_index* ix, int wpc, int hash_log2, int overflow, int gather,
                    int id_batch) {
  ix->wpc = wpc;
  ix->overflow_mode = overflow;
  ix->gather = ix->L.nchunks <= 64 ? gather : 0;  // the gather kernels take rows of <= 64 chunks
  ix->id_batch = id_batch;
  if (hash_log2 == 0) {
    ix->hash_auto = true;
    ix->bitmap_ok = true;
    ix->hash_log2 = 12;
  } else {
    ix->hash_auto = false;
    ix->bitmap_ok = false;
    ix->hash_log2 = hash_log2;
  }
  if (ix->graph_exec) {
    cudaGraphExecDestroy(ix->graph_exec);
    ix->graph_exec = nullptr;
  }
}

TuneKey tune_key(const fgraft_index* ix) {
  return TuneKey{ix->L.metric, ix->L.d, ix->p.ef_h, ix->p.R, ceil_log2(ix->L.n), ix->p.T, ix->nb};
}

// The harvest search arguments of block b of index ix (everything but the
// launch layout, which launch_beam or a many-builds launch fills in).
BeamArgs harvest_args(fgraft_index* ix, int32_t b) {
  BeamArgs a{};
  a.X = ix->L.X;
  a.ld_bytes = ix->L.ld_bytes;
  a.d = ix->L.d;
  a.nchunks = ix->L.nchunks;
  a.n = ix->L.n;
  a.s_off = ix->s_off;
  a.s_ids = ix->s_ids;
  a.A = ix->A;
  a.cnt = ix->cnt;
  a.R = ix->p.R;
  a.r_off = b > 0 ? ix->r_off : nullptr;
  a.r_ids = ix->r_ids;
  a.B = ix->nb;
  a.b = b;
  a.roots = ix->roots;
  a.T = ix->p.T;
  a.nq = (ix->L.n - b + ix->nb - 1) / ix->nb;
  a.q_first = b;
  a.q_step = ix->nb;
  if (ix->qorder) {  // block b's searches in tree-0 preorder; blocks before b hold b*q + min(b, r)
    const int64_t q = ix->L.n / ix->nb, r = ix->L.n % ix->nb;
    a.qlist = ix->qorder + (int64_t)b * q + std::min<int64_t>(b, r);
  }
  a.ef = ix->p.ef_h;
  a.mode = 0;
  a.alpha2 = ix->p.alpha * ix->p.alpha;
  a.A_out = ix->A;
  a.cnt_out = ix->cnt;
  a.Ad_out = ix->Ad;
  const bool sep = ix->prune_ns > 0;
  a.Eg = sep ? ix->Eg : nullptr;
  a.Eg_cnt = sep ? ix->Eg_cnt : nullptr;
  return a;
}

// After block b's searches: the occlusion prune (when it runs in its own
// kernels) and the reverse lists that make S_{b+1}.
int harvest_after(fgraft_index* ix, int32_t b, const BeamArgs& a, cudaStream_t s) {
  const bool prof = ix->profile && (int)ix->ev_beg.size() > b;
  if (ix->prune_ns > 0) {
    const int rc = harvest_prune(ix->L, ix->Eg, ix->Eg_cnt, ix->eg_ecap, a.nq, a.q_first,
                                 a.q_step, ix->p.R, a.alpha2, ix->A, ix->cnt, ix->ctr + C_PRUNE,
                                 ix->num_sms, s, nullptr, nullptr, nullptr, nullptr, ix->work + 4,
                                 ix->ovf_list, ix->work + 5, nullptr, ix->Ad);
    if (rc) return rc;
  }
  if (prof) FG_CUDA(record_event(ix->ev_pend[b], s));
  // the last rebuild also carries the distances the final graph reads
  const bool last = b == ix->nb - 1;
  const int rc = reverse_rows(ix->L.n, ix->p.R, ix->nb, b, ix->A, ix->cnt, ix->rcnt, ix->rcur,
                              ix->r_off, ix->r_ids, ix->scan_tmp, s, last ? ix->Ad : nullptr,
                              last ? ix->r_d : nullptr);
  if (rc) return rc;
  ix->blocks_done = b + 1;
  return 0;
}

int harvest_block_impl(fgraft_index* ix, int32_t b, cudaStream_t s) {
  BeamArgs a = harvest_args(ix, b);
  const bool prof = ix->profile && (int)ix->ev_beg.size() > b;
  int rc = launch_beam(ix, a, ix->ctr + C_HARVEST, s, prof ? ix->ev_beg[b] : nullptr,
                       prof ? ix->ev_end[b] : nullptr);
  if (rc) return rc;
  return harvest_after(ix, b, a, s);
}

// The searches of the next block b (the blocks harvested so far; block 0
// when all are) for its first `sample` work items in claim order (tree-0
// preorder when the index has the coherent schedule), each followed by its
// occlusion prune; counters go to tctr.  The rows written are those points'
// final rows (block b searches S_b, which holds rows of blocks < b only, and
// its own harvest writes the same rows again), and nothing else of the index
// changes: this is the autotuner's calibration workload.
int harvest_sample(fgraft_index* ix, int64_t sample, unsigned long long* tctr, cudaStream_t s) {
  const int32_t b = ix->blocks_done < ix->nb ? ix->blocks_done : 0;
  BeamArgs a = harvest_args(ix, b);
  a.nq = std::min<int64_t>(sample, a.nq);
  const bool sep = ix->prune_ns > 0;
  int rc = launch_beam(ix, a, tctr, s);
  if (rc || !sep) return rc;
  return harvest_prune(ix->L, ix->Eg, ix->Eg_cnt, ix->eg_ecap, a.nq, b, ix->nb, ix->p.R, a.alpha2,
                       ix->A, ix->cnt, tctr + 5, ix->num_sms, s, nullptr, nullptr, nullptr,
                       nullptr, ix->work + 4, ix->ovf_list, ix->work + 5, a.qlist, ix->Ad);
}

// Scratch of the many-builds launches on a device: the launch's claim
// counter and the per-warp global bitmaps of visited sets that outgrow the
// shared-memory hash, sized for the largest index of the launch; created on
// first use, grown when needed, kept for the process.  Not for use during
// stream capture.
struct MultiScratch {
  uint32_t* work = nullptr;
  uint32_t* gvbits = nullptr;
  int64_t gv_words = 0;  // allocated words
  std::mutex mu;
};

int multi_scratch(MultiScratch** out) {
  static std::mutex mu;
  static MultiScratch* per_dev[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return fail(FGRAFT_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lock(mu);
  if (!per_dev[dev]) {
    MultiScratch* m = new MultiScratch();
    if ((e = cudaMalloc(&m->work, 16)) != cudaSuccess) {
      delete m;
      return cuda_fail(e, "cudaMalloc(multi-build counter)");
    }
    per_dev[dev] = m;
  }
  *out = per_dev[dev];
  return 0;
}

// Block b of the indices g[0..cnt) -- same metric, lane groups, pool slots
// and row chunks -- in one search launch: every index's work items are one
// range of a single claim counter, each with its own descriptor.  The
// per-warp layout is common: a shared-memory hash sized by occupancy (the
// n-bit shared bitmap depends on n), warps per CTA 4, register gathers;
// searches whose visited set outgrows the hash go on in global bitmaps sized
// for the largest n.  Then, per index, the re-run pass, the prune and the
// reverse lists, as fgraft_harvest_block does.
int harvest_multi_launch(fgraft_index* const* g, int cnt, int32_t b, cudaStream_t s) {
  fgraft_index* ix0 = g[0];
  const int S = pool_slots(ix0->p.ef_h);
  BeamMultiFn kern = ix0->L.metric == 0 ? beam_multi_metric0(ix0->L.G, ix0->L.K, S)
                     : ix0->L.metric == 1 ? beam_multi_metric1(ix0->L.G, ix0->L.K, S)
                                          : beam_multi_metric2(ix0->L.G, ix0->L.K, S);
  if (!kern) return fail(FGRAFT_EINVAL, "no beam kernel for this metric and dimension");
  const int wpc = 4;
  const int ecap = 1 << std::max(6, ceil_log2(2 * 32 * S));
  const int qbytes = 16 * ix0->L.nchunks;
  const int fixed = 8 * ecap + (ecap / 8 + 15) / 16 * 16 + 256 + qbytes;
  int dev = 0, optin = 0;
  FG_CUDA(cudaGetDevice(&dev));
  FG_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  // the largest hash of 2^7..2^12 slots that keeps the CTAs per SM of 2^7
  int nslots = 0, per_sm = 0, base_per_sm = -1;
  for (int k = 7; k <= 12; ++k) {
    const int wb = 4 * (1 << k) + fixed;
    if (wb * wpc > optin) break;
    FG_CUDA(raise_smem_limit(reinterpret_cast<const void*>(kern), wb * wpc));
    int ps = 0;
    FG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, kern, wpc * 32, wb * wpc));
    if (base_per_sm < 0) base_per_sm = ps;
    if (ps >= base_per_sm && ps > 0) {
      nslots = 1 << k;
      per_sm = ps;
    }
  }
  if (per_sm < 1) return fail(FGRAFT_EINVAL, "many-builds launch does not fit an SM");
  const int wbytes = 4 * nslots + fixed;
  MultiScratch* ms = nullptr;
  int rc = multi_scratch(&ms);
  if (rc) return rc;
  std::lock_guard<std::mutex> lock(ms->mu);
  int64_t words = 0;
  for (int k = 0; k < cnt; ++k) words = std::max<int64_t>(words, (g[k]->L.n + 127) / 128 * 4);
  const int64_t grid_warps = (int64_t)per_sm * ix0->num_sms * wpc;
  if (words * grid_warps > ms->gv_words) {
    if (ms->gvbits) cudaFree(ms->gvbits);
    ms->gvbits = nullptr;
    ms->gv_words = 0;
    cudaError_t e = cudaMalloc(&ms->gvbits, sizeof(uint32_t) * words * grid_warps);
    if (e != cudaSuccess) {
      set_error(FGRAFT_ENOMEM, std::string("cudaMalloc(visited bitmaps): ") + cudaGetErrorString(e));
      return FGRAFT_ENOMEM;
    }
    ms->gv_words = words * grid_warps;
  }
  BeamMulti P{};
  P.nidx = cnt;
  P.work = ms->work;
  P.start[0] = 0;
  for (int k = 0; k < cnt; ++k) {
    fgraft_index* ix = g[k];
    BeamArgs a = harvest_args(ix, b);
    a.counters = ix->ctr + C_HARVEST;
    a.work = nullptr;  // the launch's counter
    a.ovf_list = ix->ovf_list;
    a.ovf_count = ix->work + 2;
    a.ovf_cap = (uint32_t)ix->ovf_cap;
    a.err_flag = ix->work + 3;
    a.hash_log2 = ceil_log2(nslots);
    a.bitmap = 0;
    a.vis_bytes = 4 * nslots;
    a.vis_cap = (int32_t)(0.8 * nslots) - 32;
    a.ecap = ecap;
    a.gvbits = ix->overflow_mode == 1 ? ms->gvbits : nullptr;
    a.gvbits_words = words;
    a.wbytes = wbytes;
    a.qbytes = qbytes;
    a.global_scratch = 0;
    a.gather = 0;
    a.id_batch = ix->id_batch;
    a.wait_polls = g_mma_wait_polls;
    P.d[k] = a;
    P.start[k + 1] = P.start[k] + a.nq;
    FG_CUDA(cudaMemsetAsync(ix->work, 0, 3 * sizeof(uint32_t), s));
  }
  FG_CUDA(cudaMemsetAsync(ms->work, 0, sizeof(uint32_t), s));
  for (int k = 0; k < cnt; ++k)  // profiled indices time the shared launch
    if (g[k]->profile && (int)g[k]->ev_beg.size() > b) FG_CUDA(record_event(g[k]->ev_beg[b], s));
  kern<<<per_sm * ix0->num_sms, wpc * 32, wbytes * wpc, s>>>(P);
  note_launch();
  FG_CUDA(cudaGetLastError());
  for (int k = 0; k < cnt; ++k)
    if (g[k]->profile && (int)g[k]->ev_end.size() > b) FG_CUDA(record_event(g[k]->ev_end[b], s));
  for (int k = 0; k < cnt && !rc; ++k) {
    fgraft_index* ix = g[k];
    rc = launch_rerun(ix, P.d[k], ix->ctr + C_HARVEST, s);
    if (!rc) rc = harvest_after(ix, b, P.d[k], s);
  }
  return rc;
}

}  // namespace

extern "C" {

const char* fgraft_last_error(void) { return g_err.c_str(); }

fgraft_status fgraft_build_scaffold(const void* X, int64_t n, int32_t d, int64_t ld,
                                    const fgraft_params* params, fgraft_stream stream,
                                    fgraft_index** out, fgraft_counters* counters) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!out) return (fgraft_status)fail(FGRAFT_EINVAL, "out is NULL");
  *out = nullptr;
  if (!params) return (fgraft_status)fail(FGRAFT_EINVAL, "params is NULL");
  const fgraft_params p = *params;
  VecLayout L;
  int rc = check_vectors(X, n, d, ld, p.metric, &L);
  if (rc) return (fgraft_status)rc;
  if (p.T < 1 || p.T > 64 || p.T > n) return (fgraft_status)fail(FGRAFT_EINVAL, "need 1 <= T <= min(64, n)");
  if (p.R < 1 || p.R > 1024) return (fgraft_status)fail(FGRAFT_EINVAL, "need 1 <= R <= 1024");
  if (p.ef_h < 1 || p.ef_h > 128) return (fgraft_status)fail(FGRAFT_EINVAL, "need 1 <= ef_h <= 128");
  if (p.B < 0) return (fgraft_status)fail(FGRAFT_EINVAL, "need B >= 0");
  if (!(p.alpha >= 0.0f) || !std::isfinite(p.alpha))
    return (fgraft_status)fail(FGRAFT_EINVAL, "alpha must be finite and >= 0");
  if (p.metric == L2_U8 && p.metric != L.metric) return (fgraft_status)fail(FGRAFT_EINVAL, "metric");

  fgraft_index* ix = new fgraft_index();
  ix->L = L;
  ix->p = p;
  ix->nb = p.B <= 1 ? 1 : p.B;
  ix->ld = ld;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&ix->num_sms, cudaDevAttrMultiProcessorCount, dev);
  {
    TuneVal tv;  // settings the autotuner chose earlier for this shape
    if (tune_table_lookup(tune_key(ix), &tv))
      apply_settings(ix, tv.wpc, tv.hash_log2, tv.overflow, tv.gather, tv.id_batch);
  }
  const int64_t T = p.T, tot = T * n;
  rc = 0;
  rc = rc ? rc : dalloc(&ix->roots, T);
  rc = rc ? rc : dalloc(&ix->parents, tot);
  rc = rc ? rc : dalloc(&ix->s_off, n + 1);
  rc = rc ? rc : dalloc(&ix->A, n * p.R);
  rc = rc ? rc : dalloc(&ix->Ad, n * p.R);
  rc = rc ? rc : dalloc(&ix->cnt, n);
  rc = rc ? rc : dalloc(&ix->r_off, n + 1);
  rc = rc ? rc : dalloc(&ix->r_ids, n * p.R);
  rc = rc ? rc : dalloc(&ix->r_d, n * p.R);
  rc = rc ? rc : dalloc(&ix->rcnt, n);
  rc = rc ? rc : dalloc(&ix->rcur, n);
  rc = rc ? rc : dalloc(&ix->f_off, n + 1);
  rc = rc ? rc : dalloc(&ix->scan_tmp, scan_tmp_elems(std::max<int64_t>(tot, 2 * n)) + 1);
  rc = rc ? rc : dalloc(&ix->work, 8);
  ix->ovf_cap = std::max<int64_t>(n, 1 << 16);
  rc = rc ? rc : dalloc(&ix->ovf_list, ix->ovf_cap);
  rc = rc ? rc : dalloc(&ix->ctr, C_COUNT);
  // re-run scratch: expanded list (up to 2^20 entries) and alive bits per warp;
  // the re-run's visited sets are the first g_warps bitmaps of gvbits
  ix->g_ecap = 1 << std::min(20, std::max(12, ceil_log2(std::min<int64_t>(n, 1 << 20))));
  ix->g_warps = 64;
  ix->gscratch_per_warp = (8ll * ix->g_ecap + ix->g_ecap / 8 + 255) / 256 * 256;
  rc = rc ? rc : dalloc(&ix->gscratch, ix->gscratch_per_warp * ix->g_warps);
  if (!rc) rc = size_visited_bitmaps(ix);
  // the prune kernel stages a point's whole candidate list in shared memory;
  // when that does not fit (large d or ef) the search prunes in place instead
  {
    const int S = pool_slots(p.ef_h);
    ix->eg_ecap = 1 << std::max(6, ceil_log2(2 * 32 * S));
    ix->prune_ns = harvest_prune_smem(ix->eg_ecap, L.nchunks) <= 112 * 1024 ? ix->eg_ecap : 0;
    if (ix->prune_ns) {
      const int64_t nq_max = (n + ix->nb - 1) / ix->nb;
      rc = rc ? rc : dalloc(&ix->Eg, nq_max * ix->eg_ecap);
      rc = rc ? rc : dalloc(&ix->Eg_cnt, nq_max);
    }
  }
  if (rc) {
    free_index(ix);
    return (fgraft_status)rc;
  }
  keyed_roots(p.seed, p.T, n, ix->roots_h);
#define FAILX(call)                                   \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) {                          \
      int c_ = cuda_fail(e_, #call);                  \
      free_index(ix);                                 \
      return (fgraft_status)c_;                       \
    }                                                 \
  } while (0)
  FAILX(cudaMemcpyAsync(ix->roots, ix->roots_h.data(), sizeof(int32_t) * T,
                        cudaMemcpyHostToDevice, s));
  FAILX(cudaMemsetAsync(ix->ctr, 0, sizeof(unsigned long long) * C_COUNT, s));
  FAILX(cudaMemsetAsync(ix->work, 0, 8 * sizeof(uint32_t), s));
  FAILX(cudaMemsetAsync(ix->cnt, 0, sizeof(int32_t) * n, s));
  FAILX(cudaMemsetAsync(ix->A, 0xFF, sizeof(int32_t) * n * p.R, s));

  // SAT forest (stream-ordered scratch)
  keep_pool_reserved();
  SatScratch S{};
  rc = 0;
  rc = rc ? rc : dalloc_async(&S.node_of, tot, s);
  rc = rc ? rc : dalloc_async(&S.kcnt, tot, s);
  rc = rc ? rc : dalloc_async(&S.kstart, tot + 1, s);
  rc = rc ? rc : dalloc_async(&S.item_pt, tot, s);
  rc = rc ? rc : dalloc_async(&S.lst, 2 * tot, s);
  rc = rc ? rc : dalloc_async(&S.best, tot, s);
  rc = rc ? rc : dalloc_async(&S.kid, tot, s);
  S.big_min = g_sat_big_min;
  const int64_t nbig_max = tot / S.big_min + 1;
  rc = rc ? rc : dalloc_async(&S.seg_start, tot + nbig_max, s);
  rc = rc ? rc : dalloc_async(&S.seg_len, tot + nbig_max, s);
  rc = rc ? rc : dalloc_async(&S.seg_node, tot + nbig_max, s);
  rc = rc ? rc : dalloc_async(&S.seg_tree, tot + nbig_max, s);
  rc = rc ? rc : dalloc_async(&S.seg_k, tot + nbig_max, s);
  rc = rc ? rc : dalloc_async(&S.nseg, 7, s);
  rc = rc ? rc : dalloc_async(&S.big_list, nbig_max, s);
  rc = rc ? rc : dalloc_async(&S.big_keys, 3 * nbig_max, s);
  rc = rc ? rc : dalloc_async(&S.big_kcount, nbig_max, s);
  rc = rc ? rc : dalloc_async(&S.big_lens, 3 * nbig_max, s);
  S.finish_len = g_sat_finish_len;
  S.scan_tmp = ix->scan_tmp;
  auto free_sat = [&]() {
    void* ps[] = {S.node_of, S.kcnt, S.kstart, S.item_pt, S.lst, S.best, S.kid,
                  S.seg_start, S.seg_len, S.seg_node, S.seg_tree, S.seg_k, S.nseg,
                  S.big_list, S.big_keys, S.big_kcount, S.big_lens};
    for (void* q : ps)
      if (q) cudaFreeAsync(q, s);
  };
  if (!rc) {
    cudaError_t e = cudaMemsetAsync(S.kcnt, 0, sizeof(uint32_t) * tot, s);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemsetAsync");
  }
  if (!rc) rc = sat_forest(L, p.T, ix->roots, ix->parents, S, ix->ctr + C_SAT, s);
  free_sat();
  if (rc) {
    free_index(ix);
    return (fgraft_status)rc;
  }
  // scaffold CSR
  uint32_t* deg = nullptr;
  int64_t* tmp_off = nullptr;
  int32_t* tmp_ids = nullptr;
  rc = 0;
  rc = rc ? rc : dalloc_async(&deg, n, s);
  rc = rc ? rc : dalloc_async(&tmp_off, n + 1, s);
  rc = rc ? rc : dalloc_async(&tmp_ids, 2 * tot, s);
  if (!rc)
    rc = scaffold_csr(n, p.T, ix->parents, ix->s_off, &ix->s_ids, &ix->s_nnz, deg, tmp_off,
                      tmp_ids, ix->scan_tmp, s, &ix->L, g_scaffold_cap);
  if (deg) cudaFreeAsync(deg, s);
  if (tmp_off) cudaFreeAsync(tmp_off, s);
  if (tmp_ids) cudaFreeAsync(tmp_ids, s);
  // coherent harvest schedule from tree 0 (the rows do not depend on it)
  bool coherent = g_coherent == 1;
  if (g_coherent == 2) {  // auto: only when the vectors do not fit in the L2 cache
    int l2 = 0;
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
    coherent = n * L.ld_bytes > (int64_t)l2;
  }
  if (!rc && coherent) {
    rc = rc ? rc : dalloc(&ix->pre, n);
    rc = rc ? rc : dalloc(&ix->qorder, n);
    bool ok = false;
    if (!rc)
      rc = coherent_schedule(n, ix->parents, ix->nb, kCoherentMaxDepth, ix->pre, ix->qorder, s,
                             &ok);
    if (!rc && !ok) {
      cudaFree(ix->pre);
      cudaFree(ix->qorder);
      ix->pre = ix->qorder = nullptr;
    }
  }
  cudaStreamSynchronize(s);
  if (rc) {
    free_index(ix);
    return (fgraft_status)rc;
  }
  if (counters) {
    rc = read_counters(ix, s, counters);
    if (rc) {
      free_index(ix);
      return (fgraft_status)rc;
    }
  }
  *out = ix;
  return FGRAFT_OK;
#undef FAILX
}

fgraft_status fgraft_harvest_block(fgraft_index* ix, int32_t b, fgraft_stream stream,
                                   fgraft_counters* counters) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!ix) return (fgraft_status)fail(FGRAFT_EINVAL, "index is NULL");
  if (b < 0 || b >= ix->nb) return (fgraft_status)fail(FGRAFT_EINVAL, "block index out of range");
  if (b != ix->blocks_done && b != 0)
    return (fgraft_status)fail(FGRAFT_EINVAL, "blocks must be harvested in order 0..B-1");
  int rc = harvest_block_impl(ix, b, s);
  if (rc) return (fgraft_status)rc;
  if (counters) return (fgraft_status)read_counters(ix, s, counters);
  return FGRAFT_OK;
}

fgraft_status fgraft_prune(fgraft_index* ix, fgraft_stream stream, fgraft_counters* counters,
                           int64_t* out_offsets, int32_t* out_ids, int64_t cap, int64_t* needed) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!ix) return (fgraft_status)fail(FGRAFT_EINVAL, "index is NULL");
  if (ix->blocks_done != ix->nb)
    return (fgraft_status)fail(FGRAFT_EINVAL, "every block must be harvested before the final prune");
  if ((out_offsets == nullptr) != (out_ids == nullptr))
    return (fgraft_status)fail(FGRAFT_EINVAL, "out_offsets and out_ids go together");
  int rc = check_err_flag(ix, s);
  if (rc) return (fgraft_status)rc;
  if (!ix->final_done) {
    FGS(cudaMemsetAsync(ix->ctr + C_FINAL, 0, sizeof(unsigned long long), s));
    keep_pool_reserved();
    rc = final_graph(ix->L, ix->p.R, ix->p.alpha * ix->p.alpha, ix->A, ix->cnt, ix->r_off,
                     ix->r_ids, ix->parents, ix->f_off, &ix->f_ids, &ix->f_nnz, ix->scan_tmp,
                     ix->ctr + C_FINAL, ix->num_sms, s, ix->Ad, ix->r_d);
    if (rc) return (fgraft_status)rc;
    ix->final_done = true;
  }
  if (needed) *needed = ix->f_nnz;
  if (out_offsets) {
    if (cap < ix->f_nnz) return (fgraft_status)fail(FGRAFT_EOVERFLOW, "out_ids capacity too small");
    FGS(cudaMemcpyAsync(out_offsets, ix->f_off, sizeof(int64_t) * (ix->L.n + 1),
                            cudaMemcpyDeviceToDevice, s));
    FGS(cudaMemcpyAsync(out_ids, ix->f_ids, sizeof(int32_t) * ix->f_nnz,
                            cudaMemcpyDeviceToDevice, s));
  }
  if (counters) return (fgraft_status)read_counters(ix, s, counters);
  return FGRAFT_OK;
}

fgraft_status fgraft_harvest_block_multi(fgraft_index* const* ixs, int32_t nix, int32_t b,
                                         fgraft_stream stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (nix < 0 || (nix > 0 && !ixs)) return (fgraft_status)fail(FGRAFT_EINVAL, "bad index list");
  for (int32_t i = 0; i < nix; ++i) {
    const fgraft_index* ix = ixs[i];
    if (!ix) return (fgraft_status)fail(FGRAFT_EINVAL, "index is NULL");
    if (b < 0 || b >= ix->nb) return (fgraft_status)fail(FGRAFT_EINVAL, "block index out of range");
    if (b != ix->blocks_done)
      return (fgraft_status)fail(FGRAFT_EINVAL, "blocks must be harvested in order 0..B-1");
    for (int32_t j = 0; j < i; ++j)
      if (ixs[j] == ix) return (fgraft_status)fail(FGRAFT_EINVAL, "an index is listed twice");
  }
  if (nix == 0) return FGRAFT_OK;
  // one search launch per group of indices sharing a kernel shape (metric,
  // lane groups, pool slots, row chunks), at most kMaxMulti per launch
  std::map<std::array<int, 5>, std::vector<fgraft_index*>> groups;
  for (int32_t i = 0; i < nix; ++i) {
    fgraft_index* ix = ixs[i];
    groups[{ix->L.metric, ix->L.G, ix->L.K, pool_slots(ix->p.ef_h), ix->L.nchunks}].push_back(ix);
  }
  int rc = 0;
  for (auto& kv : groups) {
    const std::vector<fgraft_index*>& g = kv.second;
    for (size_t i0 = 0; i0 < g.size() && !rc; i0 += kMaxMulti) {
      const size_t cnt = std::min<size_t>(kMaxMulti, g.size() - i0);
      rc = harvest_multi_launch(g.data() + i0, (int)cnt, b, s);
    }
    if (rc) break;
  }
  return (fgraft_status)rc;
}

fgraft_status fgraft_harvest_all(fgraft_index* ix, int32_t use_graph, fgraft_stream stream,
                                 fgraft_counters* counters) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!ix) return (fgraft_status)fail(FGRAFT_EINVAL, "index is NULL");
  int rc = 0;
  if (!use_graph) {
    for (int b = 0; b < ix->nb && !rc; ++b) rc = harvest_block_impl(ix, b, s);
    if (rc) return (fgraft_status)rc;
  } else {
    if (!ix->graph_exec) {
      cudaStream_t cs;
      FGS(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      cudaGraph_t graph = nullptr;
      const uint64_t before = launch_count();
      cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
      if (e == cudaSuccess) {
        for (int b = 0; b < ix->nb && !rc; ++b) rc = harvest_block_impl(ix, b, cs);
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (!rc && e2 != cudaSuccess) rc = cuda_fail(e2, "cudaStreamEndCapture");
        ix->graph_kernels = launch_count() - before;
        set_launch_count(before);
      } else {
        rc = cuda_fail(e, "cudaStreamBeginCapture");
      }
      if (!rc) {
        e = cudaGraphInstantiate(&ix->graph_exec, graph, 0);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaGraphInstantiate");
      }
      if (graph) cudaGraphDestroy(graph);
      cudaStreamDestroy(cs);
      if (rc) return (fgraft_status)rc;
    }
    FGS(cudaGraphLaunch(ix->graph_exec, s));
    note_launch(ix->graph_kernels);
    ix->blocks_done = ix->nb;
  }
  return fgraft_prune(ix, stream, counters, nullptr, nullptr, 0, nullptr);
}

fgraft_status fgraft_prune_lists(const void* X, int64_t n, int32_t d, int64_t ld, int32_t metric,
                                 const int32_t* owner, const int64_t* cand_off,
                                 const int32_t* cand_ids, int64_t nlists, float alpha, int32_t R,
                                 int32_t* out_ids, int32_t* out_cnt, fgraft_stream stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  VecLayout L;
  int rc = check_vectors(X, n, d, ld, metric, &L);
  if (rc) return (fgraft_status)rc;
  if (nlists < 0) return (fgraft_status)fail(FGRAFT_EINVAL, "nlists < 0");
  if (nlists == 0) return FGRAFT_OK;
  if (!owner || !cand_off || !cand_ids || !out_ids || !out_cnt)
    return (fgraft_status)fail(FGRAFT_EINVAL, "NULL list pointer");
  if (R < 1 || R > 1024) return (fgraft_status)fail(FGRAFT_EINVAL, "need 1 <= R <= 1024");
  if (!(alpha >= 0.0f) || !std::isfinite(alpha))
    return (fgraft_status)fail(FGRAFT_EINVAL, "alpha must be finite and >= 0");
  return (fgraft_status)prune_lists(L, owner, cand_off, cand_ids, nlists, alpha * alpha, R,
                                    out_ids, out_cnt, nullptr, s);
}

fgraft_status fgraft_prune_lists_noalloc(const void* X, int64_t n, int32_t d, int64_t ld,
                                         int32_t metric, const int32_t* owner,
                                         const int64_t* cand_off, const int32_t* cand_ids,
                                         int64_t nlists, float alpha, int32_t R, int32_t* out_ids,
                                         int32_t* out_cnt, fgraft_stream stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  VecLayout L;
  int rc = check_vectors(X, n, d, ld, metric, &L);
  if (rc) return (fgraft_status)rc;
  if (nlists < 0 || nlists > prune_lists_static_max_lists())
    return (fgraft_status)fail(FGRAFT_EINVAL, "nlists must be in [0, 65536]");
  if (nlists == 0) return FGRAFT_OK;
  if (!owner || !cand_off || !cand_ids || !out_ids || !out_cnt)
    return (fgraft_status)fail(FGRAFT_EINVAL, "NULL list pointer");
  if (R < 1 || R > 1024) return (fgraft_status)fail(FGRAFT_EINVAL, "need 1 <= R <= 1024");
  if (!(alpha >= 0.0f) || !std::isfinite(alpha))
    return (fgraft_status)fail(FGRAFT_EINVAL, "alpha must be finite and >= 0");
  return (fgraft_status)prune_lists_static(L, owner, cand_off, cand_ids, nlists, alpha * alpha, R,
                                           out_ids, out_cnt, s);
}

fgraft_status fgraft_search(fgraft_index* ix, const void* Q, int64_t nq, int64_t ldq, int32_t k,
                            int32_t ef_s, int32_t* out_ids, float* out_dist, uint32_t* out_evals,
                            fgraft_stream stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!ix) return (fgraft_status)fail(FGRAFT_EINVAL, "index is NULL");
  if (!ix->f_ids) return (fgraft_status)fail(FGRAFT_EINVAL, "search needs fgraft_prune first");
  if (nq < 0) return (fgraft_status)fail(FGRAFT_EINVAL, "nq < 0");
  if (nq == 0) return FGRAFT_OK;
  if (k < 1 || ef_s < k || ef_s > 128) return (fgraft_status)fail(FGRAFT_EINVAL, "need 1 <= k <= ef_s <= 128");
  if (!Q || !out_ids || !out_dist) return (fgraft_status)fail(FGRAFT_EINVAL, "NULL pointer");
  const int es = ix->L.metric == L2_U8 ? 1 : 4;
  if (ldq < ix->L.d || (ldq * es) % 16 || reinterpret_cast<uintptr_t>(Q) % 16)
    return (fgraft_status)fail(FGRAFT_EINVAL, "Q stride/alignment");
  BeamArgs a{};
  a.X = ix->L.X;
  a.ld_bytes = ix->L.ld_bytes;
  a.d = ix->L.d;
  a.nchunks = ix->L.nchunks;
  a.n = ix->L.n;
  a.s_off = ix->f_off;
  a.s_ids = ix->f_ids;
  a.B = 1;
  a.b = 0;
  a.roots = ix->roots;
  a.T = ix->p.T;
  a.nq = nq;
  a.Q = static_cast<const char*>(Q);
  a.ldq_bytes = ldq * es;
  a.ef = ef_s;
  a.mode = 1;
  a.k = k;
  a.top_ids = out_ids;
  a.top_d = out_dist;
  a.q_evals = out_evals;
  int rc = launch_beam(ix, a, ix->ctr + C_SEARCH, s);
  return (fgraft_status)rc;
}

fgraft_status fgraft_harvest_visited(fgraft_index* ix, const int32_t* points, int64_t np,
                                     int32_t cap, int32_t* out_ids, int32_t* out_cnt,
                                     fgraft_stream stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!ix) return (fgraft_status)fail(FGRAFT_EINVAL, "index is NULL");
  if (np < 0 || np > INT32_MAX) return (fgraft_status)fail(FGRAFT_EINVAL, "need 0 <= np < 2^31");
  if (cap < 1) return (fgraft_status)fail(FGRAFT_EINVAL, "need cap >= 1");
  if (np == 0) return FGRAFT_OK;
  if (!points || !out_ids || !out_cnt) return (fgraft_status)fail(FGRAFT_EINVAL, "NULL pointer");
  // the searches of the next block's harvest (substrate S_b, b = blocks
  // harvested so far), for the listed points, logging instead of pruning
  BeamArgs a = harvest_args(ix, ix->blocks_done);
  a.qlist = nullptr;
  a.nq = np;
  a.qpoints = points;
  a.Eg = nullptr;
  a.Eg_cnt = nullptr;
  a.A_out = nullptr;
  a.cnt_out = nullptr;
  a.Ad_out = nullptr;
  a.vlog = out_ids;
  a.vlog_cnt = out_cnt;
  a.vlog_cap = cap;
  int rc = launch_beam(ix, a, ix->ctr + C_VLOG, s);
  if (rc) return (fgraft_status)rc;
  return (fgraft_status)check_err_flag(ix, s);
}

fgraft_status fgraft_dense_block_dist(const void* X, int64_t n, int32_t d, int64_t ld,
                                      int32_t metric, const int32_t* block_ids, int64_t nb,
                                      int32_t bs, int32_t k, int32_t precision, int32_t* out_ids,
                                      float* out_dist, double* stats, fgraft_stream stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  VecLayout L;
  int rc = check_vectors(X, n, d, ld, metric, &L);
  if (rc) return (fgraft_status)rc;
  if (metric == L2_U8 && precision != 0)
    return (fgraft_status)fail(FGRAFT_EINVAL, "uint8 dense blocks take precision 0");
  if (precision < 0 || precision > 2)
    return (fgraft_status)fail(FGRAFT_EINVAL,
                               "precision must be 0 (float32), 1 (BF16 filter) or 2 (FP8 filter)");
  if (nb < 0 || nb > 65535 || bs < 1 || bs > 1024 || k < 1 || k > 64)
    return (fgraft_status)fail(FGRAFT_EINVAL, "need nb <= 65535, bs in [1,1024], k in [1,64]");
  const bool err64 = stats && stats[4] != 0.0;  // float64 error maxima requested
  if (stats)
    for (int i = 0; i < 6; ++i) stats[i] = 0.0;
  if (nb == 0) return FGRAFT_OK;
  if (!block_ids || !out_ids || !out_dist) return (fgraft_status)fail(FGRAFT_EINVAL, "NULL pointer");
  if (precision >= 1)
    return (fgraft_status)dense_block_tc(L, block_ids, nb, bs, k, precision == 2, err64,
                                         out_ids, out_dist, stats, s);
  rc = dense_block(L, block_ids, nb, bs, k, out_ids, out_dist, s);
  if (!rc && stats) FGS(cudaStreamSynchronize(s));
  return (fgraft_status)rc;
}

fgraft_status fgraft_knn_exact(const void* X, int64_t n, int32_t d, int64_t ld, int32_t metric,
                               int64_t row0, int64_t nrows, int32_t k, int32_t* out_ids,
                               float* out_dist, double* stats, fgraft_stream stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  VecLayout L;
  int rc = check_vectors(X, n, d, ld, metric, &L);
  if (rc) return (fgraft_status)rc;
  if (metric == L2_U8) return (fgraft_status)fail(FGRAFT_EINVAL, "exact k-NN takes float32 metrics");
  if (k < 1 || k > 32) return (fgraft_status)fail(FGRAFT_EINVAL, "need 1 <= k <= 32");
  if (row0 < 0 || nrows < 0 || row0 + nrows > n)
    return (fgraft_status)fail(FGRAFT_EINVAL, "need 0 <= row0 and row0 + nrows <= n");
  if (stats)
    for (int i = 0; i < 4; ++i) stats[i] = 0.0;
  if (nrows == 0) return FGRAFT_OK;
  if (!out_ids || !out_dist) return (fgraft_status)fail(FGRAFT_EINVAL, "NULL pointer");
  return (fgraft_status)knn_tc(L, row0, nrows, k, out_ids, out_dist, stats, s);
}

fgraft_status fgraft_dense_block_gram(const void* X, int64_t n, int32_t d, int64_t ld,
                                      int32_t metric, const int32_t* block_ids, int64_t nb,
                                      int32_t bs, int32_t precision, float* out_min, double* ms,
                                      fgraft_stream stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  VecLayout L;
  int rc = check_vectors(X, n, d, ld, metric, &L);
  if (rc) return (fgraft_status)rc;
  if (metric == L2_U8) return (fgraft_status)fail(FGRAFT_EINVAL, "the Gram path takes float32 metrics");
  if (precision != 1 && precision != 2)
    return (fgraft_status)fail(FGRAFT_EINVAL, "precision must be 1 (BF16) or 2 (FP8)");
  if (nb < 0 || nb > 65535 || bs < 1 || bs > 1024)
    return (fgraft_status)fail(FGRAFT_EINVAL, "need nb <= 65535, bs in [1,1024]");
  if (ms) *ms = 0.0;
  if (nb == 0) return FGRAFT_OK;
  if (!block_ids || !out_min) return (fgraft_status)fail(FGRAFT_EINVAL, "NULL pointer");
  return (fgraft_status)dense_gram_tc(L, block_ids, nb, bs, precision == 2, out_min, ms, s);
}

fgraft_status fgraft_index_copy(const fgraft_index* ix, int32_t* roots, int32_t* parents,
                                int64_t* s_offsets, int32_t* s_ids, int32_t* rows,
                                int32_t* counts, fgraft_stream stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!ix) return (fgraft_status)fail(FGRAFT_EINVAL, "index is NULL");
  const int64_t n = ix->L.n, T = ix->p.T;
  if (roots)
    FGS(cudaMemcpyAsync(roots, ix->roots, sizeof(int32_t) * T, cudaMemcpyDeviceToDevice, s));
  if (parents)
    FGS(cudaMemcpyAsync(parents, ix->parents, sizeof(int32_t) * T * n,
                            cudaMemcpyDeviceToDevice, s));
  if (s_offsets)
    FGS(cudaMemcpyAsync(s_offsets, ix->s_off, sizeof(int64_t) * (n + 1),
                            cudaMemcpyDeviceToDevice, s));
  if (s_ids)
    FGS(cudaMemcpyAsync(s_ids, ix->s_ids, sizeof(int32_t) * ix->s_nnz,
                            cudaMemcpyDeviceToDevice, s));
  if (rows)
    FGS(cudaMemcpyAsync(rows, ix->A, sizeof(int32_t) * n * ix->p.R, cudaMemcpyDeviceToDevice,
                            s));
  if (counts)
    FGS(cudaMemcpyAsync(counts, ix->cnt, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
  return FGRAFT_OK;
}

fgraft_status fgraft_index_sizes(const fgraft_index* ix, int64_t* n, int32_t* T, int32_t* R,
                                 int64_t* scaffold_nnz, int64_t* final_nnz,
                                 int32_t* blocks_done) {
  if (!ix) return (fgraft_status)fail(FGRAFT_EINVAL, "index is NULL");
  if (n) *n = ix->L.n;
  if (T) *T = ix->p.T;
  if (R) *R = ix->p.R;
  if (scaffold_nnz) *scaffold_nnz = ix->s_nnz;
  if (final_nnz) *final_nnz = ix->f_ids ? ix->f_nnz : 0;
  if (blocks_done) *blocks_done = ix->blocks_done;
  return FGRAFT_OK;
}

fgraft_status fgraft_index_counters(fgraft_index* ix, fgraft_stream stream,
                                    fgraft_counters* counters) {
  if (!ix || !counters) return (fgraft_status)fail(FGRAFT_EINVAL, "NULL argument");
  return (fgraft_status)read_counters(ix, reinterpret_cast<cudaStream_t>(stream), counters);
}

fgraft_status fgraft_index_tune(fgraft_index* ix, int32_t hash_log2, int32_t warps_per_cta,
                                int32_t overflow_mode) {
  if (!ix) return (fgraft_status)fail(FGRAFT_EINVAL, "index is NULL");
  if (overflow_mode < 0 || overflow_mode > 2)
    return (fgraft_status)fail(FGRAFT_EINVAL, "overflow_mode must be 0, 1 or 2");
  if (overflow_mode) ix->overflow_mode = overflow_mode;
  if (hash_log2 && (hash_log2 < 7 || hash_log2 > 14))
    return (fgraft_status)fail(FGRAFT_EINVAL, "hash_log2 must be in [7, 14]");
  if (warps_per_cta && (warps_per_cta < 1 || warps_per_cta > 4))
    return (fgraft_status)fail(FGRAFT_EINVAL, "warps_per_cta must be in [1, 4]");
  if (hash_log2) {
    ix->hash_log2 = hash_log2;
    ix->bitmap_ok = false;  // an explicit hash size selects the hash
    ix->hash_auto = false;
  }
  if (warps_per_cta) ix->wpc = warps_per_cta;
  if (ix->gather && ix->L.nchunks > 64) ix->gather = 0;
  const int rc = size_visited_bitmaps(ix);
  if (rc) return (fgraft_status)rc;
  if (ix->graph_exec) {
    cudaGraphExecDestroy(ix->graph_exec);
    ix->graph_exec = nullptr;
  }
  return FGRAFT_OK;
}

fgraft_status fgraft_index_autotune(fgraft_index* ix, int32_t sample, fgraft_stream stream,
                                    fgraft_tuning* chosen) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!ix) return (fgraft_status)fail(FGRAFT_EINVAL, "index is NULL");
  if (sample < 1) return (fgraft_status)fail(FGRAFT_EINVAL, "sample must be >= 1");
  int rc = check_err_flag(ix, s);
  if (rc) return (fgraft_status)rc;
  // a candidate: warps per CTA, hash_log2 (0: occupancy rule), overflow mode,
  // gather, id batch
  using Cfg = std::array<int, 5>;
  const Cfg start{ix->wpc, ix->hash_auto ? 0 : ix->hash_log2, ix->overflow_mode, ix->gather,
                  ix->id_batch};
  const Cfg defaults{4, 0, 1, 0, 2};
  unsigned long long* tctr = nullptr;
  if ((rc = dalloc(&tctr, 8))) return (fgraft_status)rc;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // one calibration run of the given settings: the fastest of three timed runs
  auto time_one = [&](const Cfg& c, float* ms) -> int {
    apply_settings(ix, c[0], c[1], c[2], c[3], c[4]);
    int r = size_visited_bitmaps(ix);
    if (r) return r;
    *ms = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0, s);
      r = harvest_sample(ix, sample, tctr, s);
      if (r) return r;
      cudaEventRecord(e1, s);
      cudaError_t e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) return cuda_fail(e, "autotune");
      float t = 0.0f;
      cudaEventElapsedTime(&t, e0, e1);
      *ms = std::min(*ms, t);
    }
    return check_err_flag(ix, s);
  };
  // options per setting; the shared-memory gather only for rows of at most
  // 64 chunks (32 rows of 1 KB per warp)
  const std::vector<std::vector<int>> opts = {
      {4, 2, 1}, {0, 9, 10, 11, 12}, {1, 2},
      ix->L.nchunks <= 64 ? std::vector<int>{0, 1} : std::vector<int>{0}, {1, 2}};
  float base_ms = 0.0f, best_ms = 0.0f;
  Cfg best = defaults;
  rc = time_one(defaults, &base_ms);  // warm-up, then the defaults' time
  if (!rc) rc = time_one(defaults, &base_ms);
  best_ms = base_ms;
  // coordinate descent: each setting in turn over its options, the others
  // held at the best so far; two rounds
  for (int round = 0; round < 2 && !rc; ++round)
    for (int dim = 0; dim < 5 && !rc; ++dim)
      for (int v : opts[dim]) {
        Cfg c = best;
        c[dim] = v;
        if (c == best) continue;
        float ms = 0.0f;
        if ((rc = time_one(c, &ms))) break;
        if (ms < best_ms) {
          best_ms = ms;
          best = c;
        }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(tctr);
  if (rc) {
    apply_settings(ix, start[0], start[1], start[2], start[3], start[4]);
    size_visited_bitmaps(ix);
    return (fgraft_status)rc;
  }
  apply_settings(ix, best[0], best[1], best[2], best[3], best[4]);
  rc = size_visited_bitmaps(ix);
  if (rc) return (fgraft_status)rc;
  const int64_t nsamp = std::min<int64_t>(sample, (ix->L.n + ix->nb - 1) / ix->nb);
  const float us = 1e3f * best_ms / (float)nsamp;
  tune_table_put(tune_key(ix), TuneVal{best[0], best[1], best[2], best[3], best[4], us});
  if (chosen) {
    chosen->warps_per_cta = best[0];
    chosen->hash_log2 = best[1];
    chosen->overflow_mode = best[2];
    chosen->gather = best[3];
    chosen->id_batch = best[4];
    chosen->us_per_query = us;
    chosen->default_us_per_query = 1e3f * base_ms / (float)nsamp;
  }
  return FGRAFT_OK;
}

fgraft_status fgraft_index_set_tuning(fgraft_index* ix, const fgraft_tuning* t) {
  if (!ix || !t) return (fgraft_status)fail(FGRAFT_EINVAL, "NULL argument");
  if (t->warps_per_cta < 1 || t->warps_per_cta > 4 ||
      (t->hash_log2 != 0 && (t->hash_log2 < 7 || t->hash_log2 > 14)) || t->overflow_mode < 1 ||
      t->overflow_mode > 2 || t->gather < 0 || t->gather > 1 || t->id_batch < 1 ||
      t->id_batch > 2 || (t->gather && ix->L.nchunks > 64))
    return (fgraft_status)fail(FGRAFT_EINVAL, "tuning setting out of range");
  apply_settings(ix, t->warps_per_cta, t->hash_log2, t->overflow_mode, t->gather, t->id_batch);
  return (fgraft_status)size_visited_bitmaps(ix);
}

fgraft_status fgraft_tuning_table_save(const char* path) {
  if (!path) return (fgraft_status)fail(FGRAFT_EINVAL, "path is NULL");
  return (fgraft_status)tune_table_save(path);
}

fgraft_status fgraft_tuning_table_load(const char* path) {
  if (!path) return (fgraft_status)fail(FGRAFT_EINVAL, "path is NULL");
  return (fgraft_status)tune_table_load(path);
}

fgraft_status fgraft_index_profile(fgraft_index* ix, int32_t enable) {
  if (!ix) return (fgraft_status)fail(FGRAFT_EINVAL, "index is NULL");
  if (enable && ix->ev_beg.empty()) {
    ix->ev_beg.resize(ix->nb);
    ix->ev_end.resize(ix->nb);
    ix->ev_pend.resize(ix->nb);
    for (int b = 0; b < ix->nb; ++b) {
      FGS(cudaEventCreate(&ix->ev_beg[b]));
      FGS(cudaEventCreate(&ix->ev_end[b]));
      FGS(cudaEventCreate(&ix->ev_pend[b]));
    }
  }
  if ((enable != 0) != ix->profile && ix->graph_exec) {
    cudaGraphExecDestroy(ix->graph_exec);
    ix->graph_exec = nullptr;
  }
  ix->profile = enable != 0;
  return FGRAFT_OK;
}

fgraft_status fgraft_index_harvest_ms(fgraft_index* ix, fgraft_stream stream, double* ms,
                                      int32_t* launches, double* prune_ms) {
  if (!ix || !ms) return (fgraft_status)fail(FGRAFT_EINVAL, "NULL argument");
  if (!ix->profile) return (fgraft_status)fail(FGRAFT_EINVAL, "profiling is off");
  FGS(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)));
  double tot = 0.0, ptot = 0.0;
  for (int b = 0; b < ix->blocks_done && b < (int)ix->ev_beg.size(); ++b) {
    float t = 0.0f, t2 = 0.0f;
    FGS(cudaEventElapsedTime(&t, ix->ev_beg[b], ix->ev_end[b]));
    FGS(cudaEventElapsedTime(&t2, ix->ev_end[b], ix->ev_pend[b]));
    tot += t;
    ptot += t2;
  }
  *ms = tot;
  if (launches) *launches = ix->blocks_done;
  if (prune_ms) *prune_ms = ptot;
  return FGRAFT_OK;
}

uint64_t fgraft_kernel_launches(void) { return launch_count(); }

fgraft_status fgraft_tune_prune(int32_t tensor_cores) {
  if (tensor_cores != 0 && tensor_cores != 1)
    return (fgraft_status)fail(FGRAFT_EINVAL, "tensor_cores must be 0 or 1");
  g_prune_tc = tensor_cores;
  g_sat_tc = tensor_cores;
  return FGRAFT_OK;
}

fgraft_status fgraft_tune_mma_wait(int32_t polls) {
  if (polls < -1) return (fgraft_status)fail(FGRAFT_EINVAL, "polls must be >= -1");
  g_mma_wait_polls = polls == -1 ? (1 << 22) : polls;
  return FGRAFT_OK;
}

fgraft_status fgraft_tune_scaffold_cap(int32_t cap) {
  if (cap < 0) return (fgraft_status)fail(FGRAFT_EINVAL, "cap must be >= 0");
  g_scaffold_cap = cap;
  return FGRAFT_OK;
}

fgraft_status fgraft_tune_schedule(int32_t coherent) {
  if (coherent < 0 || coherent > 2) return (fgraft_status)fail(FGRAFT_EINVAL, "coherent must be 0, 1 or 2");
  g_coherent = coherent;
  return FGRAFT_OK;
}

fgraft_status fgraft_index_schedule(const fgraft_index* ix, int32_t* pre, int32_t* qorder,
                                    int32_t* coherent, fgraft_stream stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!ix) return (fgraft_status)fail(FGRAFT_EINVAL, "index is NULL");
  if (coherent) *coherent = ix->qorder ? 1 : 0;
  const int64_t n = ix->L.n;
  if (pre && ix->pre)
    FGS(cudaMemcpyAsync(pre, ix->pre, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
  if (qorder && ix->qorder)
    FGS(cudaMemcpyAsync(qorder, ix->qorder, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
  return FGRAFT_OK;
}

fgraft_status fgraft_tune_sat(int32_t big_node_min, int32_t finish_len) {
  if (big_node_min == 1 || big_node_min < 0)
    return (fgraft_status)fail(FGRAFT_EINVAL, "big_node_min must be >= 2");
  if (finish_len < 0) return (fgraft_status)fail(FGRAFT_EINVAL, "finish_len must be >= 1");
  if (big_node_min) g_sat_big_min = big_node_min;
  if (finish_len) g_sat_finish_len = finish_len;
  return FGRAFT_OK;
}

void fgraft_index_destroy(fgraft_index* ix) { free_index(ix); }

}  // extern "C"
