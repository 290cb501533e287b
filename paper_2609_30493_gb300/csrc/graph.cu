// Graph bookkeeping kernels: device-wide scan, the scaffold CSR (Section 3:
// union of the trees' edges, symmetrised), the reverse lists that turn the
// rows of finished blocks into S_{b+1}, the final graph (rows symmetrised,
// re-pruned when over R, tree-0 spine added) and the stand-alone list prune.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "rowops.cuh"

namespace fg {

// ---------------------------------------------------------------------------
// Exclusive scan, uint32 -> int64, three passes over tiles of 2048.
// ---------------------------------------------------------------------------
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_PER = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_PER;

int64_t scan_tmp_elems(int64_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE + 1; }

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t* total) {
  __shared__ int64_t warp_sums[SCAN_THREADS / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    int64_t y = __shfl_up_sync(FULL, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  int64_t wpre = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < SCAN_THREADS / 32; ++w) {
    int64_t s = warp_sums[w];
    if (w < warp) wpre += s;
    tot += s;
  }
  __syncthreads();
  *total = tot;
  return wpre + x - v;
}

__global__ void scan_tiles_kernel(const uint32_t* in, int64_t n, int64_t* tile_sums) {
  const int64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t base = tile * SCAN_TILE + (int64_t)threadIdx.x * SCAN_PER;
    int64_t s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_PER; ++j)
      if (base + j < n) s += in[base + j];
    int64_t tot;
    block_exclusive_scan(s, &tot);
    if (threadIdx.x == 0) tile_sums[tile] = tot;
  }
}

__global__ void scan_prefix_kernel(int64_t* tile_sums, int64_t ntiles) {
  int64_t carry = 0;
  for (int64_t base = 0; base < ntiles; base += SCAN_THREADS) {
    const int64_t i = base + threadIdx.x;
    const int64_t v = i < ntiles ? tile_sums[i] : 0;
    int64_t tot;
    const int64_t ex = block_exclusive_scan(v, &tot);
    if (i < ntiles) tile_sums[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) tile_sums[ntiles] = carry;
}

__global__ void scan_apply_kernel(const uint32_t* in, int64_t* out, int64_t n,
                                  const int64_t* tile_pre) {
  const int64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t base = tile * SCAN_TILE + (int64_t)threadIdx.x * SCAN_PER;
    uint32_t v[SCAN_PER];
    int64_t s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_PER; ++j) {
      v[j] = base + j < n ? in[base + j] : 0u;
      s += v[j];
    }
    int64_t tot;
    int64_t run = tile_pre[tile] + block_exclusive_scan(s, &tot);
#pragma unroll
    for (int j = 0; j < SCAN_PER; ++j) {
      if (base + j < n) out[base + j] = run;
      run += v[j];
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = tile_pre[ntiles];
}

int scan_u32(const uint32_t* in, int64_t* out, int64_t n, int64_t* tmp, cudaStream_t s) {
  const int64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)device_sms() * 8));
  scan_tiles_kernel<<<grid, SCAN_THREADS, 0, s>>>(in, n, tmp);
  note_launch();
  scan_prefix_kernel<<<1, SCAN_THREADS, 0, s>>>(tmp, ntiles);
  note_launch();
  scan_apply_kernel<<<grid, SCAN_THREADS, 0, s>>>(in, out, n, tmp);
  note_launch();
  FG_CUDA(cudaGetLastError());
  return 0;
}

static int grid1d(int64_t tot, int threads = 256) {
  int64_t g = (tot + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)device_sms() * 32));
}

// ---------------------------------------------------------------------------
// Scaffold CSR.
// ---------------------------------------------------------------------------
__global__ void edge_count_kernel(int64_t n, int64_t tot, const int32_t* parents, uint32_t* deg) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = parents[i];
    if (p >= 0) {
      atomicAdd(&deg[i % n], 1u);
      atomicAdd(&deg[p], 1u);
    }
  }
}

__global__ void edge_fill_kernel(int64_t n, int64_t tot, const int32_t* parents, uint32_t* cur,
                                 const int64_t* off, int32_t* ids) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = parents[i];
    if (p >= 0) {
      const int32_t x = (int32_t)(i % n);
      ids[off[x] + atomicSub(&cur[x], 1u) - 1u] = p;
      ids[off[p] + atomicSub(&cur[p], 1u) - 1u] = x;
    }
  }
}

constexpr int ROW_WARPS = 4;
constexpr int ROW_CAP = 1024;  // keys per warp in shared memory

// Sort each row's ids ascending and drop repeats; ucnt[r] = distinct count,
// the distinct ids at the front of the row.  Rows longer than the buffer
// (cap) are appended to long_rows and left for the global-scratch pass.
__global__ void __launch_bounds__(ROW_WARPS * 32)
    sort_unique_rows_kernel(int64_t nrows, const int32_t* rowlist, const uint32_t* rowlist_len,
                            const int64_t* off, int32_t* ids, uint32_t* ucnt, int32_t* long_rows,
                            uint32_t* nlong, uint64_t* gbuf, int32_t gcap) {
  __shared__ uint64_t sbuf[ROW_WARPS][ROW_CAP];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t* keys = gbuf ? gbuf + ((int64_t)blockIdx.x * ROW_WARPS + warp) * gcap : sbuf[warp];
  const int cap = gbuf ? gcap : ROW_CAP;
  const int64_t total = rowlist_len ? (int64_t)*rowlist_len : nrows;
  for (int64_t w = (int64_t)blockIdx.x * ROW_WARPS + warp; w < total;
       w += (int64_t)gridDim.x * ROW_WARPS) {
    const int64_t r = rowlist ? rowlist[w] : w;
    const int64_t o = off[r];
    const int len = (int)(off[r + 1] - o);
    int N2 = 32;
    while (N2 < len) N2 <<= 1;
    if (N2 > cap) {
      if (lane == 0) long_rows[atomicAdd(nlong, 1u)] = (int32_t)r;
      continue;
    }
    for (int i = lane; i < len; i += 32) keys[i] = (uint64_t)(uint32_t)ids[o + i];
    __syncwarp();
    const int u = sort_unique(keys, len, lane);
    for (int i = lane; i < u; i += 32) ids[o + i] = (int32_t)keys[i];
    if (lane == 0) ucnt[r] = (uint32_t)u;
    __syncwarp();
  }
}

__global__ void compact_rows_kernel(int64_t n, const int64_t* src_off, const int32_t* src,
                                    const int64_t* dst_off, int32_t* dst) {
  const int lane = threadIdx.x & 31;
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; r < n;
       r += ((int64_t)gridDim.x * blockDim.x) / 32) {
    const int64_t len = dst_off[r + 1] - dst_off[r];
    for (int64_t i = lane; i < len; i += 32) dst[dst_off[r] + i] = src[src_off[r] + i];
  }
}

__global__ void max_row_kernel(int64_t n, const int64_t* off, const int32_t* rows,
                               const uint32_t* nrows, uint32_t* mx) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)*nrows;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = rows[i];
    atomicMax(mx, (uint32_t)(off[r + 1] - off[r]));
  }
}

static int pow2_at_least(int64_t v) {
  int p = 32;
  while (p < v) p <<= 1;
  return p;
}

// Runs the sort-unique pass, then the long rows with global scratch.
static int sort_unique_all(int64_t n, const int64_t* off, int32_t* ids, uint32_t* ucnt,
                           cudaStream_t s) {
  int32_t* long_rows = nullptr;
  uint32_t* small = nullptr;  // [0] nlong, [1] max length
  FG_CUDA(cudaMallocAsync(&long_rows, sizeof(int32_t) * std::max<int64_t>(n, 1), s));
  FG_CUDA(cudaMallocAsync(&small, 2 * sizeof(uint32_t), s));
  FG_CUDA(cudaMemsetAsync(small, 0, 2 * sizeof(uint32_t), s));
  sort_unique_rows_kernel<<<grid1d(n * 32, ROW_WARPS * 32), ROW_WARPS * 32, 0, s>>>(
      n, nullptr, nullptr, off, ids, ucnt, long_rows, small, nullptr, 0);
  note_launch();
  max_row_kernel<<<64, 256, 0, s>>>(n, off, long_rows, small, small + 1);
  note_launch();
  FG_CUDA(cudaGetLastError());
  uint32_t h[2];
  FG_CUDA(cudaMemcpyAsync(h, small, sizeof(h), cudaMemcpyDeviceToHost, s));
  FG_CUDA(cudaStreamSynchronize(s));
  int rc = 0;
  if (h[0] > 0) {
    const int gcap = pow2_at_least(h[1]);
    const int ctas = (int)std::min<uint32_t>((h[0] + ROW_WARPS - 1) / ROW_WARPS, 64);
    uint64_t* gbuf = nullptr;
    cudaError_t e = cudaMallocAsync(&gbuf, sizeof(uint64_t) * (int64_t)gcap * ctas * ROW_WARPS, s);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "cudaMallocAsync(long-row scratch)");
    } else {
      sort_unique_rows_kernel<<<ctas, ROW_WARPS * 32, 0, s>>>(n, long_rows, small, off, ids, ucnt,
                                                             long_rows, small, gbuf, gcap);
      note_launch();
      e = cudaGetLastError();
      if (e != cudaSuccess) rc = cuda_fail(e, "sort_unique_rows_kernel(long)");
      cudaFreeAsync(gbuf, s);
    }
  }
  cudaFreeAsync(long_rows, s);
  cudaFreeAsync(small, s);
  return rc;
}

// ---------------------------------------------------------------------------
// Scaffold degree cap (Section 6, an ablation the paper reports as negative):
// one warp per row longer than cap computes its keys (delta(u, v), v), finds
// the cap-th smallest key by a 64-step bit search and keeps the entries at or
// below it, in the row's id order.
// ---------------------------------------------------------------------------
constexpr int CAP_WARPS = 4;

template <int METRIC, int G, int K>
__global__ void __launch_bounds__(CAP_WARPS * 32)
    cap_rows_kernel(const RowVec V, int64_t n, int cap, const int64_t* off, int32_t* ids,
                    uint32_t* deg, uint64_t* kbuf) {
  extern __shared__ __align__(16) uint4 cap_us[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint4* us = cap_us + (int64_t)warp * V.nchunks;
  for (int64_t u = (int64_t)blockIdx.x * CAP_WARPS + warp; u < n;
       u += (int64_t)gridDim.x * CAP_WARPS) {
    const int len = (int)deg[u];
    if (len <= cap) continue;  // uniform over the warp
    const int64_t o = off[u];
    uint64_t* kb = kbuf + o;
    for (int i = lane; i < len; i += 32) kb[i] = (uint64_t)(uint32_t)ids[o + i] << 1;
    __syncwarp();
    stage_row(us, V.X + u * V.ld_bytes, V.nchunks, lane);
    eval_keys_inplace<METRIC, G, K>(V, us, kb, len, lane);
    uint64_t t = 0;  // the largest key value with fewer than cap keys below it
    for (int bit = 63; bit >= 0; --bit) {
      const uint64_t tt = t | (1ull << bit);
      int below = 0;
      for (int i = lane; i < len; i += 32) below += kb[i] < tt ? 1 : 0;
      if (__reduce_add_sync(FULL, below) < cap) t = tt;
    }
    int pos = 0;
    for (int i0 = 0; i0 < len; i0 += 32) {
      const int i = i0 + lane;
      const bool keep = i < len && kb[i] <= t;
      const int32_t v = keep ? ids[o + i] : 0;
      const unsigned bal = __ballot_sync(FULL, keep);
      if (keep) ids[o + pos + __popc(bal & ((1u << lane) - 1u))] = v;
      pos += __popc(bal);
      __syncwarp();
    }
    if (lane == 0) deg[u] = (uint32_t)pos;
  }
}

using CapKernelFn = void (*)(const RowVec, int64_t, int, const int64_t*, int32_t*, uint32_t*,
                             uint64_t*);

static CapKernelFn cap_kernel_for(int metric, int G, int K) {
#define CX(M, GG, KK) \
  if (metric == M && G == GG && K == KK) return cap_rows_kernel<M, GG, KK>;
#define CF(M) CX(M, 4, 1) CX(M, 8, 1) CX(M, 16, 1) CX(M, 32, 1) CX(M, 32, 2) CX(M, 32, 4) \
  CX(M, 32, 8)
  CF(0)
  CF(1)
  CX(2, 4, 1) CX(2, 8, 1) CX(2, 16, 1)
#undef CF
#undef CX
  return nullptr;
}

int scaffold_csr(int64_t n, int T, const int32_t* parents, int64_t* s_off, int32_t** s_ids,
                 int64_t* nnz_out, uint32_t* deg, int64_t* tmp_off, int32_t* tmp_ids,
                 int64_t* scan_tmp, cudaStream_t s, const VecLayout* L, int cap) {
  const int64_t tot = (int64_t)T * n;
  FG_CUDA(cudaMemsetAsync(deg, 0, sizeof(uint32_t) * n, s));
  edge_count_kernel<<<grid1d(tot), 256, 0, s>>>(n, tot, parents, deg);
  note_launch();
  int rc = scan_u32(deg, tmp_off, n, scan_tmp, s);
  if (rc) return rc;
  edge_fill_kernel<<<grid1d(tot), 256, 0, s>>>(n, tot, parents, deg, tmp_off, tmp_ids);
  note_launch();
  FG_CUDA(cudaGetLastError());
  rc = sort_unique_all(n, tmp_off, tmp_ids, deg, s);
  if (rc) return rc;
  if (cap > 0) {
    CapKernelFn ck = cap_kernel_for(L->metric, L->G, L->K);
    if (!ck) {
      set_error(1, "no scaffold cap kernel for this metric and dimension");
      return 1;
    }
    uint64_t* kbuf = nullptr;
    FG_CUDA(cudaMallocAsync(&kbuf, sizeof(uint64_t) * std::max<int64_t>(2 * tot, 1), s));
    const int smem = CAP_WARPS * 16 * L->nchunks;
    FG_CUDA(raise_smem_limit(reinterpret_cast<const void*>(ck), smem));
    ck<<<grid1d(n * 32, CAP_WARPS * 32), CAP_WARPS * 32, smem, s>>>(
        RowVec{L->X, L->ld_bytes, L->d, L->nchunks}, n, cap, tmp_off, tmp_ids, deg, kbuf);
    note_launch();
    FG_CUDA(cudaGetLastError());
    FG_CUDA(cudaFreeAsync(kbuf, s));
  }
  rc = scan_u32(deg, s_off, n, scan_tmp, s);
  if (rc) return rc;
  int64_t nnz = 0;
  FG_CUDA(cudaMemcpyAsync(&nnz, s_off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  FG_CUDA(cudaStreamSynchronize(s));
  FG_CUDA(cudaMalloc(s_ids, sizeof(int32_t) * std::max<int64_t>(nnz, 1)));
  compact_rows_kernel<<<grid1d(n * 32), 256, 0, s>>>(n, tmp_off, tmp_ids, s_off, *s_ids);
  note_launch();
  FG_CUDA(cudaGetLastError());
  *nnz_out = nnz;
  return 0;
}

// ---------------------------------------------------------------------------
// Reverse lists of the rows of blocks 0..b.
// ---------------------------------------------------------------------------
__global__ void rev_count_kernel(int64_t n, int R, int nb, int b, const int32_t* A,
                                 const int32_t* cnt, uint32_t* rcnt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n * R;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = i / R;
    const int j = (int)(i - p * R);
    if ((int)(p % nb) <= b && j < cnt[p]) atomicAdd(&rcnt[A[i]], 1u);
  }
}

__global__ void rev_fill_kernel(int64_t n, int R, int nb, int b, const int32_t* A,
                                const int32_t* cnt, uint32_t* rcur, const int64_t* r_off,
                                int32_t* r_ids, const float* Ad, float* r_d) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n * R;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = i / R;
    const int j = (int)(i - p * R);
    if ((int)(p % nb) <= b && j < cnt[p]) {
      const int32_t u = A[i];
      const int64_t k = r_off[u] + atomicAdd(&rcur[u], 1u);
      r_ids[k] = (int32_t)p;
      if (r_d) r_d[k] = Ad[i];
    }
  }
}

int reverse_rows(int64_t n, int R, int nb, int b, const int32_t* A, const int32_t* cnt,
                 uint32_t* rcnt, uint32_t* rcur, int64_t* r_off, int32_t* r_ids,
                 int64_t* scan_tmp, cudaStream_t s, const float* Ad, float* r_d) {
  FG_CUDA(cudaMemsetAsync(rcnt, 0, sizeof(uint32_t) * n, s));
  FG_CUDA(cudaMemsetAsync(rcur, 0, sizeof(uint32_t) * n, s));
  rev_count_kernel<<<grid1d(n * R), 256, 0, s>>>(n, R, nb, b, A, cnt, rcnt);
  note_launch();
  int rc = scan_u32(rcnt, r_off, n, scan_tmp, s);
  if (rc) return rc;
  rev_fill_kernel<<<grid1d(n * R), 256, 0, s>>>(n, R, nb, b, A, cnt, rcur, r_off, r_ids,
                                                Ad, Ad ? r_d : nullptr);
  note_launch();
  FG_CUDA(cudaGetLastError());
  return 0;
}

// ---------------------------------------------------------------------------
// Final graph and list prune: one warp per row.
// ---------------------------------------------------------------------------
struct FinalArgs {
  RowVec V;
  int64_t n;
  int32_t R;
  float alpha2;
  // final graph: candidate sources
  const int32_t* A;
  const int32_t* cnt;
  const int64_t* r_off;
  const int32_t* r_ids;
  const int32_t* parent0;
  const int64_t* c0_off;
  const int32_t* c0_ids;
  // list prune: candidate lists and owners
  const int32_t* owner;
  const int64_t* l_off;
  const int32_t* l_ids;
  // outputs: final rows into out_ids at out_cap_off[u] with out_cnt[u];
  // list prune rows into out_ids[i*R] with out_cnt[i]
  const int64_t* out_cap_off;
  int32_t* out_ids;
  int32_t* out_cnt;
  // work list (NULL: all rows) and long-row spill
  const int32_t* rowlist;
  const uint32_t* rowlist_len;
  int64_t nrows;
  int32_t* long_rows;
  uint32_t* nlong;
  uint64_t* gbuf;
  int32_t gcap;
  int32_t mode;  // 0 final graph, 1 list prune, 2 final rows after the CTA prune
  int32_t qbytes;  // bytes of one staged vector (16 * nchunks)
  unsigned long long* ctr;
  // final graph rows handed to the CTA prune (def_keys null: none): rows
  // with R < m <= def_cap write their sorted keys to def_keys + def_koff[u]
  // and join the list def_rows / def_m (length *def_count); mode 2 then
  // takes the kept keys (def_kept, R per listed row, def_kcnt of them)
  uint64_t* def_keys;
  const int64_t* def_koff;
  int32_t* def_rows;
  int32_t* def_m;
  uint32_t* def_count;
  int32_t* def_long;
  int32_t def_cap;
  const uint64_t* def_kept;
  const int32_t* def_kcnt;
  // non-null: warps claim the entries of the work list one at a time from
  // this counter (a persistent grid), instead of a fixed stride
  uint32_t* claim;
  // keys per warp in shared memory when gbuf is null (0: FIN_CAP)
  int32_t scap;
  // final graph (optional, both or neither): the distance beside each id of
  // A and of the reverse lists; the candidate keys are then read, not evaluated
  const float* Ad;
  const float* r_d;
  // the CTA-wide kernel's rows (hlist null: none): rows with more than
  // fh_raw raw candidates whose keys fit FH_CAP are listed beforehand and
  // skipped here; rows with more than heavy_thr distinct candidates are
  // appended to hlist (count *hcount) here, once their keys are known
  int32_t* hlist;
  uint32_t* hcount;
  int32_t fh_raw;
  int32_t heavy_thr;
};

// Final row of u from its kept keys (sorted, kk of them, owner's vector
// staged in us): the tree-0 spine members not yet in it are evaluated and
// added, the row is sorted by (delta, id) and written out.
template <int METRIC, int G, int K>
__device__ void final_spine_out(const FinalArgs& a, int32_t u, const uint4* us, uint64_t* keys,
                                int kk, int lane) {
  const int32_t p0 = a.parent0[u];
  const int32_t* ch = a.c0_ids + a.c0_off[u];
  const int sdeg = (p0 >= 0 ? 1 : 0) + (int)(a.c0_off[u + 1] - a.c0_off[u]);
  int add = 0;
  for (int j = 0; j < sdeg; ++j) {
    const int32_t v = (p0 >= 0) ? (j == 0 ? p0 : ch[j - 1]) : ch[j];
    if (keys_contain(keys, kk, v, lane)) continue;
    // evaluate delta(u, v) and append
    eval_keys<METRIC, G, K>(a.V, us, &v, 1, nullptr, 0, keys, kk + add, lane);
    ++add;
  }
  kk = sort_unique(keys, kk + add, lane);
  int32_t* out = a.out_ids + a.out_cap_off[u];
  for (int i = lane; i < kk; i += 32) out[i] = key_id(keys[i]);
  if (lane == 0) a.out_cnt[u] = kk;
}

constexpr int FIN_WARPS = 4;
constexpr int FIN_CAP = 1024;
constexpr int FIN_DEF_CAP = 256;  // longest final row list the CTA prune takes

// The CTA-wide kernel for final rows with many candidates (below).
constexpr int FH_WARPS = 8;
constexpr int FH_CAP = 4096;  // keys of one row (a power of two)

__host__ __device__ inline int fh_smem_bytes(int qbytes) {
  return 8 * FH_CAP + 2 * (FH_CAP / 8) + 2 * qbytes + 64;
}

// Whether the CTA-wide kernel takes a row: more raw candidates than the
// threshold, and its keys, with the kept ones and the spine after the
// prune, fit the shared buffer.
__device__ __forceinline__ bool fh_takes(int mraw, int sdeg, int R, int thr) {
  if (thr <= 0 || mraw <= thr) return false;
  const int need = max(pow2_dev(mraw), pow2_dev(min(mraw, R) + sdeg));
  return need <= FH_CAP;
}


// Shared memory per warp: key buffer and bit words of scap keys (unless the
// row works in global scratch), then two staged vectors (the row's owner,
// the kept c*).
__host__ __device__ inline int fin_warp_bytes(bool global_keys, int qbytes, int scap = 0) {
  const int c = scap > 0 ? scap : FIN_CAP;
  return (global_keys ? 0 : 8 * c + c / 4) + 2 * qbytes;
}

template <int METRIC, int G, int K>
__global__ void __launch_bounds__(FIN_WARPS * 32) final_rows_kernel(const FinalArgs a) {
  extern __shared__ __align__(16) unsigned char fsm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * FIN_WARPS + warp;
  unsigned char* wsm = fsm + (int64_t)warp * fin_warp_bytes(a.gbuf != nullptr, a.qbytes, a.scap);
  uint64_t* keys;
  uint32_t* bits;
  int cap;
  if (a.gbuf) {
    keys = a.gbuf + gw * ((int64_t)a.gcap + a.gcap / 32);
    bits = reinterpret_cast<uint32_t*>(keys + a.gcap);
    cap = a.gcap;
  } else {
    cap = a.scap > 0 ? a.scap : FIN_CAP;
    keys = reinterpret_cast<uint64_t*>(wsm);
    bits = reinterpret_cast<uint32_t*>(wsm + 8 * cap);
    wsm += 8 * cap + cap / 4;
  }
  uint4* us = reinterpret_cast<uint4*>(wsm);
  uint4* cs = reinterpret_cast<uint4*>(wsm + a.qbytes);
  const int64_t total = a.rowlist_len ? (int64_t)*a.rowlist_len : a.nrows;
  unsigned long long ev = 0;
  auto next_item = [&](int64_t cur) -> int64_t {
    if (!a.claim) return cur + (int64_t)gridDim.x * FIN_WARPS;
    uint32_t v = 0;
    if (lane == 0) v = atomicAdd(a.claim, 1u);
    return (int64_t)__shfl_sync(FULL, v, 0);
  };
  for (int64_t w = a.claim ? next_item(0) : gw; w < total; w = next_item(w)) {
    const int64_t r = a.rowlist ? a.rowlist[w] : w;
    if (a.mode == 2) {
      const int32_t u2 = a.def_rows[r];
      const int kk2 = a.def_kcnt[r];
      for (int i = lane; i < kk2; i += 32) keys[i] = a.def_kept[r * a.R + i];
      stage_row(us, a.V.X + (int64_t)u2 * a.V.ld_bytes, a.V.nchunks, lane);
      final_spine_out<METRIC, G, K>(a, u2, us, keys, kk2, lane);
      __syncwarp();
      continue;
    }
    int32_t u;
    const int32_t *seg0, *seg1;
    int len0, len1;
    int sdeg = 0;
    if (a.mode == 0) {
      u = (int32_t)r;
      seg0 = a.A + (int64_t)u * a.R;
      len0 = a.cnt[u];
      seg1 = a.r_ids + a.r_off[u];
      len1 = (int)(a.r_off[u + 1] - a.r_off[u]);
      sdeg = (a.parent0[u] >= 0 ? 1 : 0) + (int)(a.c0_off[u + 1] - a.c0_off[u]);
    } else {
      u = a.owner[r];
      seg0 = a.l_ids + a.l_off[r];
      len0 = (int)(a.l_off[r + 1] - a.l_off[r]);
      seg1 = nullptr;
      len1 = 0;
    }
    const int mraw = len0 + len1;
    if (a.mode == 0 && a.hlist && fh_takes(mraw, sdeg, a.R, a.fh_raw)) continue;  // listed already
    const int need = max(pow2_dev(mraw), pow2_dev(min(mraw, a.R) + sdeg));
    if (need > cap) {
      if (lane == 0) a.long_rows[atomicAdd(a.nlong, 1u)] = (int32_t)r;
      continue;
    }
    // the distinct candidate ids first, then their keys
    int m;
    if (a.mode == 0) {
      // C(u) = A[u] u rev(u): neither list repeats an id or holds u, so only
      // the reverse ids that also sit in A[u] are dropped
      // (with the distances at hand the keys are complete already)
      const float* dseg0 = a.Ad ? a.Ad + (int64_t)u * a.R : nullptr;
      const float* dseg1 = a.Ad ? a.r_d + a.r_off[u] : nullptr;
      for (int i = lane; i < len0; i += 32)
        keys[i] = dseg0 ? make_key(dseg0[i], seg0[i]) : (uint64_t)(uint32_t)seg0[i] << 1;
      __syncwarp();
      m = len0;
      for (int base = 0; base < len1; base += 32) {
        const int i = base + lane;
        const int32_t v = i < len1 ? seg1[i] : -1;
        bool dup = v < 0;
        for (int x = 0; x < len0; ++x) dup |= key_id(keys[x]) == v;
        const unsigned keep = __ballot_sync(FULL, !dup);
        if (!dup)
          keys[m + __popc(keep & ((1u << lane) - 1u))] =
              dseg1 ? make_key(dseg1[i], v) : (uint64_t)(uint32_t)v << 1;
        m += __popc(keep);
      }
      __syncwarp();
    } else {
      // a list may repeat ids and hold its owner
      for (int i = lane; i < mraw; i += 32) {
        const int32_t v = seg0[i];
        keys[i] = v == u ? PAD : ((uint64_t)(uint32_t)v << 1);
      }
      __syncwarp();
      m = sort_unique(keys, mraw, lane);
      if (m > 0 && __shfl_sync(FULL, keys[m - 1] == PAD ? 1 : 0, 0)) --m;  // dropped owner
    }
    if (a.mode == 0 && a.hlist && m > a.heavy_thr) {
      // more distinct candidates than the tensor-core prune takes: the
      // CTA-wide kernel prunes the row (and counts it)
      if (lane == 0) a.hlist[atomicAdd(a.hcount, 1u)] = u;
      __syncwarp();
      continue;
    }
    stage_row(us, a.V.X + (int64_t)u * a.V.ld_bytes, a.V.nchunks, lane);
    if (m > 0 && !(a.mode == 0 && a.Ad)) eval_keys_inplace<METRIC, G, K>(a.V, us, keys, m, lane);
    ev += (unsigned long long)m;  // the evaluations C(u) takes, whether done here or earlier
    // rows the CTA prune takes stay unsorted (that kernel orders them)
    const bool defer =
        a.mode == 0 && a.def_keys && !a.gbuf && m > a.R && m <= a.def_cap;
    if (!defer) {
      int N2 = 32;
      while (N2 < m) N2 <<= 1;
      for (int i = m + lane; i < N2; i += 32) keys[i] = PAD;
      __syncwarp();
      warp_sort_mem(keys, N2, lane);
    }
    if (a.mode == 0) {
      // spine members not already candidates cost one evaluation each
      const int32_t p0 = a.parent0[u];
      const int32_t* ch = a.c0_ids + a.c0_off[u];
      for (int j = 0; j < sdeg; ++j) {
        const int32_t v = (p0 >= 0) ? (j == 0 ? p0 : ch[j - 1]) : ch[j];
        if (!keys_contain(keys, m, v, lane)) ++ev;
      }
      if (defer) {
        // the prune of this row runs in the CTA prune kernel
        uint32_t slot = 0;
        if (lane == 0) slot = atomicAdd(a.def_count, 1u);
        slot = __shfl_sync(FULL, slot, 0);
        uint64_t* dst = a.def_keys + a.def_koff[u];
        for (int i = lane; i < m; i += 32) dst[i] = keys[i];
        if (lane == 0) {
          a.def_rows[slot] = u;
          a.def_m[slot] = m;
        }
        __syncwarp();
        continue;
      }
    }
    int kk = m;
    if (m > a.R || a.mode == 1)
      kk = prune_sorted<METRIC, G, K>(a.V, keys, m, a.alpha2, a.R, bits, cs, &ev, lane);
    if (a.mode == 0) {
      final_spine_out<METRIC, G, K>(a, u, us, keys, kk, lane);
    } else {
      int32_t* out = a.out_ids + r * a.R;
      for (int i = lane; i < a.R; i += 32) out[i] = i < kk ? key_id(keys[i]) : -1;
      if (lane == 0) a.out_cnt[r] = kk;
    }
    __syncwarp();
  }
  if (lane == 0 && ev && a.ctr) atomicAdd(a.ctr, ev);
}

using FinalKernelFn = void (*)(const FinalArgs);

// ---------------------------------------------------------------------------
// Final graph rows with many candidates: one CTA of 8 warps per row.  The
// keys come from the stored distances (A[u] and the reverse list of u);
// the CTA sorts them in shared memory (a repeated key -- a candidate both in
// A[u] and in the reverse list -- stays out of the alive set), and each
// removal pass of the prune is spread over the warps, a word of 32
// candidates at a time: every candidate of a pass is tested against the same
// c*, so the words are independent.  Then warp 0 adds the tree-0 spine and
// writes the row, as the one-warp kernel does.
// ---------------------------------------------------------------------------
template <int METRIC, int G, int K>
__global__ void __launch_bounds__(FH_WARPS * 32) final_heavy_kernel(const FinalArgs a,
                                                                     const int32_t* hrows,
                                                                     const uint32_t* hcount,
                                                                     uint32_t* claim) {
  using L = Lanes<G, K>;
  extern __shared__ __align__(16) unsigned char hsm[];
  uint64_t* keys = reinterpret_cast<uint64_t*>(hsm);
  uint32_t* alive = reinterpret_cast<uint32_t*>(hsm + 8 * FH_CAP);
  uint32_t* keptm = alive + FH_CAP / 32;
  uint4* cs = reinterpret_cast<uint4*>(hsm + 8 * FH_CAP + 2 * (FH_CAP / 8));
  uint4* us = reinterpret_cast<uint4*>(hsm + 8 * FH_CAP + 2 * (FH_CAP / 8) + a.qbytes);
  int* sh = reinterpret_cast<int*>(hsm + 8 * FH_CAP + 2 * (FH_CAP / 8) + 2 * a.qbytes);
  // sh[0]: claimed row, sh[1]: cur (c*), sh[2]: kept, sh[3]: done, sh[4]: distinct count
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane / L::P, j = lane % L::P;
  const int64_t total = (int64_t)*hcount;
  unsigned long long ev = 0;
  for (;;) {
    if (tid == 0) sh[0] = (int)atomicAdd(claim, 1u);
    __syncthreads();
    const int64_t r = sh[0];
    if (r >= total) break;
    const int32_t u = hrows[r];
    const int len0 = a.cnt[u];
    const int64_t r0 = a.r_off[u];
    const int len1 = (int)(a.r_off[u + 1] - r0);
    const int N = len0 + len1;
    int N2 = 32;
    while (N2 < N) N2 <<= 1;
    for (int i = tid; i < N2; i += FH_WARPS * 32) {
      uint64_t k = PAD;
      if (i < len0)
        k = make_key(a.Ad[(int64_t)u * a.R + i], a.A[(int64_t)u * a.R + i]);
      else if (i < N)
        k = make_key(a.r_d[r0 + i - len0], a.r_ids[r0 + i - len0]);
      keys[i] = k;
    }
    if (warp == 1) stage_row(us, a.V.X + (int64_t)u * a.V.ld_bytes, a.V.nchunks, lane);
    __syncthreads();
    // bitonic sort of the N2 keys
    for (int kk = 2; kk <= N2; kk <<= 1) {
      for (int jj = kk >> 1; jj > 0; jj >>= 1) {
        for (int i = tid; i < N2; i += FH_WARPS * 32) {
          const int l = i ^ jj;
          if (l > i) {
            const uint64_t x = keys[i], y = keys[l];
            const bool up = (i & kk) == 0;
            if ((x > y) == up) {
              keys[i] = y;
              keys[l] = x;
            }
          }
        }
        __syncthreads();
      }
    }
    // the distinct candidates are alive; the kept mask starts empty
    const int nw = N2 / 32;
    if (tid == 0) sh[4] = 0;
    __syncthreads();
    for (int w = tid; w < nw; w += FH_WARPS * 32) {
      uint32_t bits = 0;
      for (int t = 0; t < 32; ++t) {
        const int i = 32 * w + t;
        const uint64_t k = keys[i];
        if (k != PAD && (i == 0 || keys[i - 1] != k)) bits |= 1u << t;
      }
      alive[w] = bits;
      keptm[w] = 0u;
      atomicAdd(&sh[4], __popc(bits));
    }
    __syncthreads();
    const int m = sh[4];
    ev += (unsigned long long)(tid == 0 ? m : 0);
    // spine members outside C(u) cost one evaluation each (warp 0)
    const int32_t p0 = a.parent0[u];
    const int32_t* ch = a.c0_ids + a.c0_off[u];
    const int sdeg = (p0 >= 0 ? 1 : 0) + (int)(a.c0_off[u + 1] - a.c0_off[u]);
    if (warp == 0) {
      for (int q = 0; q < sdeg; ++q) {
        const int32_t v = (p0 >= 0) ? (q == 0 ? p0 : ch[q - 1]) : ch[q];
        if (!keys_contain(keys, N2, v, lane) && lane == 0) ++ev;
      }
    }
    if (m > a.R) {
      if (tid == 0) {
        sh[1] = -1;
        sh[2] = 0;
        sh[3] = 0;
      }
      __syncthreads();
      for (;;) {
        if (warp == 0) {
          // the next alive candidate after c*
          const int cur = sh[1];
          int nxt = -1;
          for (int w0 = (cur + 1) / 32; w0 < nw && nxt < 0; w0 += 32) {
            const int w = w0 + lane;
            uint32_t bits = w < nw ? alive[w] : 0u;
            if (w == (cur + 1) / 32) bits &= ~((1u << ((cur + 1) % 32)) - 1u);
            if (w < (cur + 1) / 32) bits = 0u;
            const unsigned nz = __ballot_sync(FULL, bits != 0u);
            if (nz) {
              const int wl = __ffs(nz) - 1;
              const uint32_t b = __shfl_sync(FULL, bits, wl);
              nxt = (w0 + wl) * 32 + __ffs(b) - 1;
            }
          }
          if (lane == 0) {
            if (nxt < 0) {
              sh[3] = 1;
            } else {
              alive[nxt / 32] &= ~(1u << (nxt % 32));
              keptm[nxt / 32] |= 1u << (nxt % 32);
              sh[1] = nxt;
              sh[2] += 1;
              if (sh[2] == a.R) sh[3] = 1;
            }
          }
        }
        __syncthreads();
        if (sh[3]) break;
        const int cur = sh[1];
        for (int c = tid; c < a.V.nchunks; c += FH_WARPS * 32)
          cs[c] = __ldg(reinterpret_cast<const uint4*>(a.V.X + (int64_t)key_id(keys[cur]) *
                                                                   a.V.ld_bytes) + c);
        __syncthreads();
        // the removal pass: each warp its words of candidates after c*
        for (int w = cur / 32 + warp; w < nw; w += FH_WARPS) {
          uint32_t bits = alive[w];
          if (w == cur / 32) bits &= ~((2u << (cur % 32)) - 1u);
          if (lane == 0) ev += (unsigned long long)__popc(bits);
          uint32_t kill = 0;
          while (bits) {
            const int nb = __popc(bits);
            uint4 y[L::UW][L::VL][K];
            int jx[L::UW];
#pragma unroll
            for (int uu = 0; uu < L::UW; ++uu) {
              const int rr = uu * L::CPW + g;
              jx[uu] = rr < nb ? nth_set_bit(bits, rr) : -1;
              const int e = w * 32 + (jx[uu] >= 0 ? jx[uu] : 0);
              load_slots<G, K>(a.V.X + (int64_t)key_id(keys[e]) * a.V.ld_bytes, a.V.nchunks, j,
                               y[uu]);
            }
#pragma unroll
            for (int uu = 0; uu < L::UW; ++uu) {
              const float dd = slots_dist<METRIC, G, K>(cs, y[uu], a.V.nchunks, a.V.d, j);
              if (jx[uu] >= 0 && j == 0) {
                const float dp = key_dist(keys[w * 32 + jx[uu]]);
                if (__fmul_rn(a.alpha2, dd) <= dp) kill |= 1u << jx[uu];
              }
            }
            const int consumed = nb < L::CPW * L::UW ? nb : L::CPW * L::UW;
            if (consumed >= nb)
              bits = 0;
            else
              bits &= ~((1u << nth_set_bit(bits, consumed)) - 1u);
          }
          kill = __reduce_or_sync(FULL, kill);
          if (lane == 0) alive[w] &= ~kill;
        }
        __syncthreads();
      }
    } else {
      // every distinct candidate is kept
      for (int w = tid; w < nw; w += FH_WARPS * 32) keptm[w] = alive[w];
      __syncthreads();
    }
    // the kept keys to the front, in order, then the spine and the row (warp 0)
    if (warp == 0) {
      int outn = 0;
      for (int base = 0; base < N2; base += 32) {
        const int i = base + lane;
        const bool keep = (keptm[i / 32] >> (i % 32)) & 1u;
        const uint64_t k = keep ? keys[i] : PAD;
        const unsigned msk = __ballot_sync(FULL, keep);
        __syncwarp();
        if (keep) keys[outn + __popc(msk & ((1u << lane) - 1u))] = k;
        outn += __popc(msk);
        __syncwarp();
      }
      final_spine_out<METRIC, G, K>(a, u, us, keys, outn, lane);
    }
    __syncthreads();
  }
  if (ev && a.ctr) atomicAdd(a.ctr, ev);
}

using FinalHeavyFn = void (*)(const FinalArgs, const int32_t*, const uint32_t*, uint32_t*);

static FinalHeavyFn final_heavy_for(int metric, int G, int K) {
#define HX(M, GG, KK) \
  if (metric == M && G == GG && K == KK) return final_heavy_kernel<M, GG, KK>;
#define HF(M) HX(M, 4, 1) HX(M, 8, 1) HX(M, 16, 1) HX(M, 32, 1) HX(M, 32, 2) HX(M, 32, 4) \
  HX(M, 32, 8)
  HF(0)
  HF(1)
  HX(2, 4, 1) HX(2, 8, 1) HX(2, 16, 1)
#undef HF
#undef HX
  return nullptr;
}

static FinalKernelFn final_kernel_for(int metric, int G, int K) {
#define FX(M, GG, KK) \
  if (metric == M && G == GG && K == KK) return final_rows_kernel<M, GG, KK>;
#define FF(M) FX(M, 4, 1) FX(M, 8, 1) FX(M, 16, 1) FX(M, 32, 1) FX(M, 32, 2) FX(M, 32, 4) \
  FX(M, 32, 8)
  FF(0)
  FF(1)
  FX(2, 4, 1) FX(2, 8, 1) FX(2, 16, 1)
#undef FF
#undef FX
  return nullptr;
}

__global__ void child_count_kernel(int64_t n, const int32_t* parent0, uint32_t* c) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (parent0[i] >= 0) atomicAdd(&c[parent0[i]], 1u);
}
__global__ void child_fill_kernel(int64_t n, const int32_t* parent0, uint32_t* cur,
                                  const int64_t* off, int32_t* ids) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = parent0[i];
    if (p >= 0) ids[off[p] + atomicAdd(&cur[p], 1u)] = (int32_t)i;
  }
}
__global__ void final_cap_kernel(int64_t n, int R, const int32_t* parent0, const int64_t* c0_off,
                                 uint32_t* cap) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    cap[i] = (uint32_t)(R + (parent0[i] >= 0 ? 1 : 0) + (c0_off[i + 1] - c0_off[i]));
}
__global__ void max_final_need_kernel(int64_t n, const int32_t* rows, const uint32_t* nrows,
                                      int mode, int R, const int32_t* cnt, const int64_t* r_off,
                                      const int32_t* parent0, const int64_t* c0_off,
                                      const int64_t* l_off, uint32_t* mx) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)*nrows;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = rows[i];
    int64_t mraw, sdeg = 0;
    if (mode == 0) {
      mraw = cnt[r] + (r_off[r + 1] - r_off[r]);
      sdeg = (parent0[r] >= 0 ? 1 : 0) + (c0_off[r + 1] - c0_off[r]);
    } else {
      mraw = l_off[r + 1] - l_off[r];
    }
    int64_t need = max(mraw, min(mraw, (int64_t)R) + sdeg);
    atomicMax(mx, (uint32_t)need);
  }
}

// Dynamic shared memory of the two final_rows_kernel launches (shared-memory
// keys, global-scratch keys); the function's maximum is set to the larger.
static int fin_smem(FinalKernelFn kern, int qbytes, int* sm_shared, int* sm_global) {
  *sm_shared = FIN_WARPS * fin_warp_bytes(false, qbytes);
  *sm_global = FIN_WARPS * fin_warp_bytes(true, qbytes);
  FG_CUDA(raise_smem_limit(reinterpret_cast<const void*>(kern), std::max(*sm_shared, *sm_global)));
  return 0;
}

// The final graph's rows in the order the candidate kernel claims them: the
// rows it prunes itself (more raw candidates than the CTA prune takes, or
// than R when nothing is deferred) first, then the rest, so that the long
// in-warp prunes start early instead of trailing the launch.  With hlist,
// the rows whose keys the one-warp kernel cannot hold (more than fh_raw raw
// candidates) and the CTA-wide kernel can (fh_takes) are listed there; the
// one-warp kernel skips them by the same test and lists the others with
// many distinct candidates itself.
__global__ void final_order_kernel(int64_t n, int heavy, const int32_t* cnt, const int64_t* r_off,
                                   int32_t* order, uint32_t* ctr2, int R, const int32_t* parent0,
                                   const int64_t* c0_off, int32_t* hlist, uint32_t* hcount,
                                   int fh_raw) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t mraw = cnt[i] + (r_off[i + 1] - r_off[i]);
    if (mraw > heavy)
      order[atomicAdd(&ctr2[0], 1u)] = (int32_t)i;
    else
      order[n - 1 - atomicAdd(&ctr2[1], 1u)] = (int32_t)i;
    if (hlist) {
      const int sdeg = (parent0[i] >= 0 ? 1 : 0) + (int)(c0_off[i + 1] - c0_off[i]);
      if (fh_takes((int)mraw, sdeg, R, fh_raw)) hlist[atomicAdd(hcount, 1u)] = (int32_t)i;
    }
  }
}

static int run_final_rows(FinalArgs a, const VecLayout& L, int64_t nrows, int num_sms,
                          cudaStream_t s) {
  FinalKernelFn kern = final_kernel_for(L.metric, L.G, L.K);
  if (!kern) {
    set_error(1, "no row kernel for this metric and dimension");
    return 1;
  }
  a.qbytes = 16 * L.nchunks;
  int sm0 = 0, sm1 = 0;
  const int rc0 = fin_smem(kern, a.qbytes, &sm0, &sm1);
  if (rc0) return rc0;
  int32_t* long_rows = nullptr;
  uint32_t* small = nullptr;
  int32_t* order = nullptr;
  int32_t* hlist = nullptr;
  // small: [0] long rows, [1] their largest need, [2..3] order counters,
  // [4] main claim, [5] CTA-wide rows, [6] their claim
  FG_CUDA(cudaMallocAsync(&long_rows, sizeof(int32_t) * std::max<int64_t>(nrows, 1), s));
  FG_CUDA(cudaMallocAsync(&small, 8 * sizeof(uint32_t), s));
  FG_CUDA(cudaMemsetAsync(small, 0, 8 * sizeof(uint32_t), s));
  a.rowlist = nullptr;
  a.rowlist_len = nullptr;
  a.nrows = nrows;
  a.long_rows = long_rows;
  a.nlong = small;
  a.gbuf = nullptr;
  a.gcap = 0;
  a.claim = nullptr;
  int per_sm = 0;
  if (a.mode == 0 && num_sms > 0)
    FG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, FIN_WARPS * 32, sm0));
  // rows above the CTA prune's tile (or above R when nothing is deferred)
  // go to the CTA-wide kernel when their keys are stored
  const int heavy = a.def_keys ? a.def_cap : a.R;
  FinalHeavyFn hkern = a.Ad ? final_heavy_for(L.metric, L.G, L.K) : nullptr;
  int per_sm_h = 0;
  const int hsm_bytes = fh_smem_bytes(a.qbytes);
  if (per_sm > 0 && hkern) {
    FG_CUDA(raise_smem_limit(reinterpret_cast<const void*>(hkern), hsm_bytes));
    FG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_h, hkern, FH_WARPS * 32,
                                                          hsm_bytes));
  }
  if (per_sm > 0) {
    // final graph: heavy rows first, claimed one by one by a persistent grid
    FG_CUDA(cudaMallocAsync(&order, sizeof(int32_t) * std::max<int64_t>(nrows, 1), s));
    if (per_sm_h > 0)
      FG_CUDA(cudaMallocAsync(&hlist, sizeof(int32_t) * std::max<int64_t>(nrows, 1), s));
    final_order_kernel<<<grid1d(nrows, 256), 256, 0, s>>>(
        nrows, heavy, a.cnt, a.r_off, order, small + 2, a.R, a.parent0, a.c0_off, hlist,
        small + 5, FIN_CAP);
    note_launch();
    FinalArgs m = a;
    m.rowlist = order;
    m.claim = small + 4;
    if (per_sm_h > 0) {
      m.hlist = hlist;
      m.hcount = small + 5;
      m.fh_raw = FIN_CAP;
      m.heavy_thr = heavy;
    }
    kern<<<per_sm * num_sms, FIN_WARPS * 32, sm0, s>>>(m);
    note_launch();
    if (per_sm_h > 0) {
      hkern<<<per_sm_h * num_sms, FH_WARPS * 32, hsm_bytes, s>>>(m, hlist, small + 5, small + 6);
      note_launch();
    }
  } else {
    kern<<<grid1d(nrows * 32, FIN_WARPS * 32), FIN_WARPS * 32, sm0, s>>>(a);
    note_launch();
  }
  max_final_need_kernel<<<64, 256, 0, s>>>(nrows, long_rows, small, a.mode, a.R, a.cnt, a.r_off,
                                           a.parent0, a.c0_off, a.l_off, small + 1);
  note_launch();
  FG_CUDA(cudaGetLastError());
  uint32_t h[2];
  FG_CUDA(cudaMemcpyAsync(h, small, sizeof(h), cudaMemcpyDeviceToHost, s));
  FG_CUDA(cudaStreamSynchronize(s));
  int rc = 0;
  int optin = 0;
  {
    int dev = 0;
    FG_CUDA(cudaGetDevice(&dev));
    FG_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  }
  const int lcap = h[0] > 0 ? pow2_at_least(h[1]) : 0;
  const int lsm = FIN_WARPS * fin_warp_bytes(false, a.qbytes, lcap);
  if (h[0] > 0 && lsm <= optin) {
    // long rows whose keys fit shared memory: sorted and pruned there, one
    // warp per row, as many CTAs as rows need
    cudaError_t e = raise_smem_limit(reinterpret_cast<const void*>(kern), std::max(lsm, sm0));
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "cudaFuncSetAttribute(final_rows_kernel)");
    } else {
      FinalArgs l = a;
      l.rowlist = long_rows;
      l.rowlist_len = small;
      l.scap = lcap;
      kern<<<(int)((h[0] + FIN_WARPS - 1) / FIN_WARPS), FIN_WARPS * 32, lsm, s>>>(l);
      note_launch();
      e = cudaGetLastError();
      if (e != cudaSuccess) rc = cuda_fail(e, "final_rows_kernel(long)");
    }
  } else if (h[0] > 0) {
    const int gcap = lcap;
    const int ctas = (int)std::min<uint32_t>((h[0] + FIN_WARPS - 1) / FIN_WARPS, 64);
    uint64_t* gbuf = nullptr;
    cudaError_t e = cudaMallocAsync(
        &gbuf, sizeof(uint64_t) * ((int64_t)gcap + gcap / 32) * ctas * FIN_WARPS, s);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "cudaMallocAsync(long-row scratch)");
    } else {
      a.rowlist = long_rows;
      a.rowlist_len = small;
      a.gbuf = gbuf;
      a.gcap = gcap;
      kern<<<ctas, FIN_WARPS * 32, sm1, s>>>(a);
      note_launch();
      e = cudaGetLastError();
      if (e != cudaSuccess) rc = cuda_fail(e, "final_rows_kernel(long)");
      cudaFreeAsync(gbuf, s);
    }
  }
  if (!rc && a.def_keys) {
    // rows deferred to the CTA prune, then their spine merge
    rc = harvest_prune(L, a.def_keys, a.def_m, a.def_cap, 0, 0, 0, a.R, a.alpha2, nullptr,
                       const_cast<int32_t*>(a.def_kcnt), a.ctr, num_sms, s, a.def_rows,
                       a.def_koff, a.def_count, const_cast<uint64_t*>(a.def_kept),
                       a.def_count + 1, a.def_long, a.def_count + 2);
    if (!rc) {
      FinalArgs b = a;
      b.mode = 2;
      b.rowlist = nullptr;
      b.rowlist_len = a.def_count;
      b.gbuf = nullptr;
      b.gcap = 0;
      kern<<<grid1d(nrows * 32, FIN_WARPS * 32), FIN_WARPS * 32, sm0, s>>>(b);
      note_launch();
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) rc = cuda_fail(e, "final_rows_kernel(merge)");
    }
  }
  cudaFreeAsync(long_rows, s);
  cudaFreeAsync(small, s);
  cudaFreeAsync(order, s);
  cudaFreeAsync(hlist, s);
  return rc;
}

// Key space of a final row that may go to the CTA prune: its raw candidate
// count (row plus reverse list) when above R, capped at def_cap.
__global__ void final_defcap_kernel(int64_t n, int R, int def_cap, const int32_t* cnt,
                                    const int64_t* r_off, uint32_t* capd) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t mraw = cnt[i] + (r_off[i + 1] - r_off[i]);
    capd[i] = mraw > R ? (uint32_t)std::min<int64_t>(mraw, def_cap) : 0u;
  }
}

int final_graph(const VecLayout& L, int R, float alpha2, const int32_t* A, const int32_t* cnt,
                const int64_t* r_off, const int32_t* r_ids, const int32_t* parent0,
                int64_t* f_off, int32_t** f_ids, int64_t* f_nnz, int64_t* scan_tmp,
                unsigned long long* ctr, int num_sms, cudaStream_t s, const float* Ad,
                const float* r_d) {
  const int64_t n = L.n;
  uint32_t *c0cnt = nullptr, *capc = nullptr;
  int64_t *c0_off = nullptr, *cap_off = nullptr;
  int32_t *c0_ids = nullptr, *tmp_ids = nullptr, *rowcnt = nullptr;
  // rows pruned by the CTA prune kernel
  int64_t* def_koff = nullptr;
  uint64_t *def_keys = nullptr, *def_kept = nullptr;
  int32_t *def_rows = nullptr, *def_m = nullptr, *def_kcnt = nullptr;
  uint32_t* def_count = nullptr;
  int32_t* def_long = nullptr;
  int rc = 0;
  auto cleanup = [&]() {
    cudaFreeAsync(c0cnt, s);
    cudaFreeAsync(capc, s);
    cudaFreeAsync(c0_off, s);
    cudaFreeAsync(cap_off, s);
    cudaFreeAsync(c0_ids, s);
    cudaFreeAsync(tmp_ids, s);
    cudaFreeAsync(rowcnt, s);
    cudaFreeAsync(def_koff, s);
    cudaFreeAsync(def_keys, s);
    cudaFreeAsync(def_kept, s);
    cudaFreeAsync(def_rows, s);
    cudaFreeAsync(def_m, s);
    cudaFreeAsync(def_kcnt, s);
    cudaFreeAsync(def_count, s);
    cudaFreeAsync(def_long, s);
  };
#define FG_TRY(call)                                \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) {                        \
      rc = cuda_fail(e_, #call);                    \
      cleanup();                                    \
      return rc;                                    \
    }                                               \
  } while (0)
  FG_TRY(cudaMallocAsync(&c0cnt, sizeof(uint32_t) * n, s));
  FG_TRY(cudaMallocAsync(&capc, sizeof(uint32_t) * n, s));
  FG_TRY(cudaMallocAsync(&c0_off, sizeof(int64_t) * (n + 1), s));
  FG_TRY(cudaMallocAsync(&cap_off, sizeof(int64_t) * (n + 1), s));
  FG_TRY(cudaMallocAsync(&c0_ids, sizeof(int32_t) * std::max<int64_t>(n, 1), s));
  FG_TRY(cudaMallocAsync(&rowcnt, sizeof(int32_t) * n, s));
  FG_TRY(cudaMemsetAsync(c0cnt, 0, sizeof(uint32_t) * n, s));
  child_count_kernel<<<grid1d(n), 256, 0, s>>>(n, parent0, c0cnt);
  note_launch();
  rc = scan_u32(c0cnt, c0_off, n, scan_tmp, s);
  if (rc) return cleanup(), rc;
  FG_TRY(cudaMemsetAsync(c0cnt, 0, sizeof(uint32_t) * n, s));
  child_fill_kernel<<<grid1d(n), 256, 0, s>>>(n, parent0, c0cnt, c0_off, c0_ids);
  note_launch();
  final_cap_kernel<<<grid1d(n), 256, 0, s>>>(n, R, parent0, c0_off, capc);
  note_launch();
  rc = scan_u32(capc, cap_off, n, scan_tmp, s);
  if (rc) return cleanup(), rc;
  int64_t capn = 0;
  FG_TRY(cudaMemcpyAsync(&capn, cap_off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  FG_TRY(cudaStreamSynchronize(s));
  FG_TRY(cudaMallocAsync(&tmp_ids, sizeof(int32_t) * std::max<int64_t>(capn, 1), s));
  // rows of at most def_cap candidates go to the CTA prune, which stages
  // them all in shared memory: def_cap is the largest power of two in
  // [64, FIN_DEF_CAP] that fits an SM, or 0 (no such rows) for long vectors
  int def_cap = 0;
  {
    int dev = 0, optin = 0;
    FG_TRY(cudaGetDevice(&dev));
    FG_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    for (int c = FIN_DEF_CAP; c >= 64 && !def_cap; c >>= 1)
      if (harvest_prune_smem(c, L.nchunks) <= optin) def_cap = c;
  }
  // key space of the rows that may go to the CTA prune (capc is reused)
  final_defcap_kernel<<<grid1d(n), 256, 0, s>>>(n, R, def_cap, cnt, r_off, capc);
  note_launch();
  FG_TRY(cudaMallocAsync(&def_koff, sizeof(int64_t) * (n + 1), s));
  rc = scan_u32(capc, def_koff, n, scan_tmp, s);
  if (rc) return cleanup(), rc;
  int64_t defn = 0;
  FG_TRY(cudaMemcpyAsync(&defn, def_koff + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  FG_TRY(cudaStreamSynchronize(s));
  FG_TRY(cudaMallocAsync(&def_keys, sizeof(uint64_t) * std::max<int64_t>(defn, 1), s));
  FG_TRY(cudaMallocAsync(&def_kept, sizeof(uint64_t) * std::max<int64_t>(n * R, 1), s));
  FG_TRY(cudaMallocAsync(&def_rows, sizeof(int32_t) * std::max<int64_t>(n, 1), s));
  FG_TRY(cudaMallocAsync(&def_m, sizeof(int32_t) * std::max<int64_t>(n, 1), s));
  FG_TRY(cudaMallocAsync(&def_kcnt, sizeof(int32_t) * std::max<int64_t>(n, 1), s));
  // count, timeout flag, rows longer than the 128-candidate tile
  FG_TRY(cudaMallocAsync(&def_count, 4 * sizeof(uint32_t), s));
  FG_TRY(cudaMemsetAsync(def_count, 0, 4 * sizeof(uint32_t), s));
  FG_TRY(cudaMallocAsync(&def_long, sizeof(int32_t) * std::max<int64_t>(n, 1), s));
  FinalArgs a{};
  a.Ad = Ad;
  a.r_d = Ad ? r_d : nullptr;
  a.def_keys = def_cap ? def_keys : nullptr;
  a.def_koff = def_koff;
  a.def_rows = def_rows;
  a.def_m = def_m;
  a.def_count = def_count;
  a.def_long = def_long;
  a.def_cap = def_cap;
  a.def_kept = def_kept;
  a.def_kcnt = def_kcnt;
  a.V = RowVec{L.X, L.ld_bytes, L.d, L.nchunks};
  a.n = n;
  a.R = R;
  a.alpha2 = alpha2;
  a.A = A;
  a.cnt = cnt;
  a.r_off = r_off;
  a.r_ids = r_ids;
  a.parent0 = parent0;
  a.c0_off = c0_off;
  a.c0_ids = c0_ids;
  a.out_cap_off = cap_off;
  a.out_ids = tmp_ids;
  a.out_cnt = rowcnt;
  a.mode = 0;
  a.ctr = ctr;
  rc = run_final_rows(a, L, n, num_sms, s);
  if (rc) return cleanup(), rc;
  // final CSR
  rc = scan_u32(reinterpret_cast<const uint32_t*>(rowcnt), f_off, n, scan_tmp, s);
  if (rc) return cleanup(), rc;
  int64_t nnz = 0;
  uint32_t tc_err = 0;
  FG_TRY(cudaMemcpyAsync(&nnz, f_off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  FG_TRY(cudaMemcpyAsync(&tc_err, def_count + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  FG_TRY(cudaStreamSynchronize(s));
  if (tc_err) {
    set_error(5, "a tensor-core prune timed out waiting for its products");
    cleanup();
    return 5;
  }
  if (*f_ids) {
    cudaFree(*f_ids);
    *f_ids = nullptr;
  }
  FG_TRY(cudaMalloc(f_ids, sizeof(int32_t) * std::max<int64_t>(nnz, 1)));
  compact_rows_kernel<<<grid1d(n * 32), 256, 0, s>>>(n, cap_off, tmp_ids, f_off, *f_ids);
  note_launch();
  FG_TRY(cudaGetLastError());
  *f_nnz = nnz;
  cleanup();
  return 0;
#undef FG_TRY
}

int prune_lists(const VecLayout& L, const int32_t* owner, const int64_t* l_off,
                const int32_t* l_ids, int64_t nlists, float alpha2, int R, int32_t* out_ids,
                int32_t* out_cnt, unsigned long long* ctr, cudaStream_t s) {
  FinalArgs a{};
  a.V = RowVec{L.X, L.ld_bytes, L.d, L.nchunks};
  a.n = L.n;
  a.R = R;
  a.alpha2 = alpha2;
  a.owner = owner;
  a.l_off = l_off;
  a.l_ids = l_ids;
  a.out_ids = out_ids;
  a.out_cnt = out_cnt;
  a.mode = 1;
  a.ctr = ctr;
  return run_final_rows(a, L, nlists, 0, s);
}

// ---------------------------------------------------------------------------
// List prune that allocates nothing.
//
// Some callers cannot call cudaMalloc at the moment they need a prune:
// serving loops that must never enter the allocator because an allocation
// can stall or fail under memory pressure, and hosts that have already handed
// all device memory to their own pool allocator.
// For them the scratch of the list prune lives in one file-scope device
// array, reserved when the library is loaded on a device and kept until the
// process exits.  Its size fixes the limits: at most NA_MAX_LISTS lists per
// call and at most NA_MAX_LEN candidates per list.
// ---------------------------------------------------------------------------
constexpr int64_t NA_MAX_LISTS = 1 << 16;
constexpr int NA_MAX_LEN = 4096;
constexpr int NA_CTAS = 16;  // CTAs of the pass over lists too long for shared memory
constexpr int64_t NA_WARP_WORDS = NA_MAX_LEN + NA_MAX_LEN / 32;  // keys + bit words, in uint64
constexpr size_t NA_COUNTERS = 256;
constexpr size_t NA_SCRATCH_BYTES = NA_COUNTERS + 2 * 4 * NA_MAX_LISTS +
                                    8 * NA_WARP_WORDS * NA_CTAS * FIN_WARPS;
static __device__ __align__(256) unsigned char g_prune_scratch[NA_SCRATCH_BYTES];

// Device address of g_prune_scratch for each device, looked up once.
static unsigned char* prune_scratch_address(int* rc) {
  static std::mutex mu;
  static unsigned char* addr[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    *rc = cuda_fail(e, "cudaGetDevice");
    return nullptr;
  }
  if (dev < 0 || dev >= 64) {
    set_error(1, "device index out of range");
    *rc = 1;
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_prune_scratch);
    if (e != cudaSuccess) {
      *rc = cuda_fail(e, "cudaGetSymbolAddress(g_prune_scratch)");
      return nullptr;
    }
    addr[dev] = static_cast<unsigned char*>(ptr);
  }
  *rc = 0;
  return addr[dev];
}

int64_t prune_lists_static_max_lists() { return NA_MAX_LISTS; }
int prune_lists_static_max_len() { return NA_MAX_LEN; }

int prune_lists_static(const VecLayout& L, const int32_t* owner, const int64_t* l_off,
                       const int32_t* l_ids, int64_t nlists, float alpha2, int R,
                       int32_t* out_ids, int32_t* out_cnt, cudaStream_t s) {
  FinalKernelFn kern = final_kernel_for(L.metric, L.G, L.K);
  if (!kern) {
    set_error(1, "no row kernel for this metric and dimension");
    return 1;
  }
  if (nlists > NA_MAX_LISTS) {
    set_error(1, "at most 65536 lists per call");
    return 1;
  }
  int rc = 0;
  unsigned char* base = prune_scratch_address(&rc);
  if (rc) return rc;
  const int qbytes = 16 * L.nchunks;
  int sm0 = 0, sm1 = 0;
  rc = fin_smem(kern, qbytes, &sm0, &sm1);
  if (rc) return rc;
  uint32_t* counters = reinterpret_cast<uint32_t*>(base);  // [0] long lists, [1] too long
  int32_t* long_rows = reinterpret_cast<int32_t*>(base + NA_COUNTERS);
  int32_t* too_long = long_rows + NA_MAX_LISTS;
  uint64_t* keys = reinterpret_cast<uint64_t*>(base + NA_COUNTERS + 8 * NA_MAX_LISTS);
  // the array keeps the previous call's contents: the counters start at zero
  FG_CUDA(cudaMemsetAsync(counters, 0, 2 * sizeof(uint32_t), s));
  FinalArgs a{};
  a.V = RowVec{L.X, L.ld_bytes, L.d, L.nchunks};
  a.n = L.n;
  a.R = R;
  a.alpha2 = alpha2;
  a.owner = owner;
  a.l_off = l_off;
  a.l_ids = l_ids;
  a.out_ids = out_ids;
  a.out_cnt = out_cnt;
  a.mode = 1;
  a.qbytes = qbytes;
  a.ctr = nullptr;
  a.rowlist = nullptr;
  a.rowlist_len = nullptr;
  a.nrows = nlists;
  a.long_rows = long_rows;
  a.nlong = counters;
  a.gbuf = nullptr;
  a.gcap = 0;
  kern<<<grid1d(nlists * 32, FIN_WARPS * 32), FIN_WARPS * 32, sm0, s>>>(a);
  note_launch();
  // lists longer than shared memory holds: fixed-size key buffers in the array
  a.rowlist = long_rows;
  a.rowlist_len = counters;
  a.long_rows = too_long;
  a.nlong = counters + 1;
  a.gbuf = keys;
  a.gcap = NA_MAX_LEN;
  kern<<<NA_CTAS, FIN_WARPS * 32, sm1, s>>>(a);
  note_launch();
  FG_CUDA(cudaGetLastError());
  uint32_t over = 0;
  FG_CUDA(cudaMemcpyAsync(&over, counters + 1, sizeof(over), cudaMemcpyDeviceToHost, s));
  FG_CUDA(cudaStreamSynchronize(s));
  if (over) {
    set_error(1, "a list holds more than 4096 candidates");
    return 1;
  }
  return 0;
}

}  // namespace fg
