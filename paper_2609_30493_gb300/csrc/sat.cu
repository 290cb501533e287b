// Spatial-approximation forest on the GPU (the scaffold of Section 1 and
// Section 3, after Navarro 2002), built level by level for all T trees at
// once.
//
// A node a holding the point set P picks its children by the sorted greedy
// scan: in (delta(x,a), id) order, x joins iff delta(x,a) < delta(x,b) for
// every child b already chosen.  Here the scan is run without a sort, as a
// sequence of minimum selections: the next child is the smallest key among
// the points no child has rejected yet (every smaller key is a child or
// rejected, so this is exactly the point the scan would accept next), and the
// new child then rejects every remaining point y with
// delta(y,b) <= delta(y,a).  The same pass keeps, for every point, its
// closest child by (delta, id), which is the assignment of the non-children.
// One CTA owns one node; the points of all nodes of a level are grouped by a
// counting sort keyed on (tree, node).
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace fg {

struct SatSegArgs {
  const char* X;
  int64_t ld_bytes;
  int32_t d;
  int32_t nchunks;
  int64_t n;
  const int32_t* item_pt;
  const int64_t* seg_start;
  const int32_t* seg_len;
  const int32_t* seg_node;
  const int32_t* seg_tree;
  float* kd;
  uint64_t* best;
  uint8_t* flag;  // 0 candidate, 1 rejected, 2 child
  int32_t* node_of;
  int32_t* parent;
  unsigned long long* ctr;
};

template <int NW>
__device__ __forceinline__ void block_argmin(uint64_t& key, int& idx, uint64_t (*rk)[NW],
                                             int (*ri)[NW], int parity) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    uint64_t ok = __shfl_xor_sync(FULL, key, off);
    int oi = __shfl_xor_sync(FULL, idx, off);
    if (ok < key) {
      key = ok;
      idx = oi;
    }
  }
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    rk[parity][warp] = key;
    ri[parity][warp] = idx;
  }
  __syncthreads();
  key = PAD;
  idx = -1;
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    uint64_t kk = rk[parity][w];
    if (kk < key) {
      key = kk;
      idx = ri[parity][w];
    }
  }
}

// Stage a row in shared memory with the whole CTA.
__device__ __forceinline__ void stage_row_cta(uint4* dst, const char* __restrict__ row,
                                              int nchunks) {
  for (int c = threadIdx.x; c < nchunks; c += blockDim.x)
    dst[c] = __ldg(reinterpret_cast<const uint4*>(row) + c);
}

template <int METRIC, int G, int K, int NW>
__global__ void __launch_bounds__(NW * 32) sat_segment_kernel(const SatSegArgs a) {
  using L = Lanes<G, K>;
  constexpr int STEP = L::CPW * L::U;
  __shared__ uint64_t rk[2][NW];
  __shared__ int ri[2][NW];
  __shared__ __align__(16) uint4 cvec[256];  // the node's point, then each new child
  const int s = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane / L::P, j = lane % L::P;
  const int64_t start = a.seg_start[s];
  const int m = a.seg_len[s];
  const int32_t anode = a.seg_node[s];
  const int64_t tbase = (int64_t)a.seg_tree[s] * a.n;

  stage_row_cta(cvec, a.X + (int64_t)anode * a.ld_bytes, a.nchunks);
  __syncthreads();
  uint64_t bk = PAD;
  int bi = -1;
  for (int base = warp * STEP; base < m; base += NW * STEP) {
    uint4 y[L::U][L::VL][K];
#pragma unroll
    for (int u = 0; u < L::U; ++u) {
      const int idx = min(base + u * L::CPW + g, m - 1);
      load_slots<G, K>(a.X + (int64_t)a.item_pt[start + idx] * a.ld_bytes, a.nchunks, j, y[u]);
    }
#pragma unroll
    for (int u = 0; u < L::U; ++u) {
      const float dd = slots_dist<METRIC, G, K>(cvec, y[u], a.nchunks, a.d, j);
      const int idx = base + u * L::CPW + g;
      if (idx < m && j == 0) {
        a.kd[start + idx] = dd;
        a.best[start + idx] = PAD;
        a.flag[start + idx] = 0;
        const uint64_t key = make_key(dd, a.item_pt[start + idx]);
        if (key < bk) {
          bk = key;
          bi = idx;
        }
      }
    }
  }
  int parity = 0;
  block_argmin<NW>(bk, bi, rk, ri, parity);
  long long k = 0;
  while (bk != PAD) {
    const int32_t bpt = key_id(bk);
    if (threadIdx.x == 0) {
      a.flag[start + bi] = 2;
      a.parent[tbase + bpt] = anode;
    }
    ++k;
    stage_row_cta(cvec, a.X + (int64_t)bpt * a.ld_bytes, a.nchunks);
    __syncthreads();
    bk = PAD;
    bi = -1;
    for (int base = warp * STEP; base < m; base += NW * STEP) {
      uint4 y[L::U][L::VL][K];
#pragma unroll
      for (int u = 0; u < L::U; ++u) {
        const int idx = min(base + u * L::CPW + g, m - 1);
        load_slots<G, K>(a.X + (int64_t)a.item_pt[start + idx] * a.ld_bytes, a.nchunks, j, y[u]);
      }
#pragma unroll
      for (int u = 0; u < L::U; ++u) {
        const float dd = slots_dist<METRIC, G, K>(cvec, y[u], a.nchunks, a.d, j);
        const int idx = base + u * L::CPW + g;
        if (idx < m && j == 0) {
          const int64_t it = start + idx;
          const uint8_t f = a.flag[it];
          if (f != 2) {
            const uint64_t ck = make_key(dd, bpt);
            if (ck < a.best[it]) a.best[it] = ck;
            if (f == 0) {
              const float kdv = a.kd[it];
              if (dd <= kdv) {
                a.flag[it] = 1;
              } else {
                const uint64_t key = make_key(kdv, a.item_pt[it]);
                if (key < bk) {
                  bk = key;
                  bi = idx;
                }
              }
            }
          }
        }
      }
    }
    parity ^= 1;
    block_argmin<NW>(bk, bi, rk, ri, parity);
  }
  for (int i = threadIdx.x; i < m; i += NW * 32) {
    const int64_t it = start + i;
    const int32_t pt = a.item_pt[it];
    a.node_of[tbase + pt] = a.flag[it] == 2 ? -1 : key_id(a.best[it]);
  }
  if (threadIdx.x == 0) {
    const long long mm = m;
    atomicAdd(a.ctr, (unsigned long long)(mm + k * (k - 1) / 2 + (mm - k) * k));
  }
}

// ---------------------------------------------------------------------------
// Nodes with many points: every CTA of a launch owns a tile of one node's
// points, and one launch performs one child selection for all such nodes.
// The minimum over a node's points is reduced with a 64-bit atomicMin into
// one of three rotating per-node key buffers (read, write, clear), so no CTA
// ever waits for another.
// ---------------------------------------------------------------------------
constexpr int BIG_TILE = 2048;  // points per CTA
constexpr int BIG_NW = 8;

struct SatBigArgs {
  SatSegArgs s;
  const int32_t* big;  // segment index of each big node
  uint64_t* cur;       // current minimum key per big node (the next child)
  uint64_t* nxt;       // receives the minimum of this pass
  uint64_t* clr;       // reset to PAD for the pass after
  uint32_t* kcount;    // children chosen so far per big node
  int32_t y_off;       // first big node of this launch (grid.y is limited to 65535)
};

template <int METRIC, int G, int K>
__device__ __forceinline__ uint64_t warp_min64(uint64_t v) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) v = umin64(v, __shfl_xor_sync(FULL, v, off));
  return v;
}

// mode 0: distances to the node's own point (kd), state reset, first minimum.
// mode 1: one child selection.  mode 2: write the assignment and the count.
template <int METRIC, int G, int K>
__global__ void __launch_bounds__(BIG_NW * 32) sat_big_kernel(const SatBigArgs A, int mode) {
  using L = Lanes<G, K>;
  constexpr int STEP = L::CPW * L::U;
  __shared__ __align__(16) uint4 cvec[256];
  const SatSegArgs& a = A.s;
  const int y = blockIdx.y + A.y_off;
  const int sidx = A.big[y];
  const int64_t start = a.seg_start[sidx];
  const int m = a.seg_len[sidx];
  const int32_t anode = a.seg_node[sidx];
  const int64_t tbase = (int64_t)a.seg_tree[sidx] * a.n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane / L::P, j = lane % L::P;
  const int t0 = blockIdx.x * BIG_TILE;
  if (t0 >= m) return;
  const int t1 = min(m, t0 + BIG_TILE);
  if (mode == 2) {
    for (int i = t0 + threadIdx.x; i < t1; i += BIG_NW * 32) {
      const int64_t it = start + i;
      a.node_of[tbase + a.item_pt[it]] = a.flag[it] == 2 ? -1 : key_id(a.best[it]);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      const long long mm = m, k = A.kcount[y];
      atomicAdd(a.ctr, (unsigned long long)(mm + k * (k - 1) / 2 + (mm - k) * k));
    }
    return;
  }
  int32_t bpt = anode;
  if (mode == 1) {
    if (blockIdx.x == 0 && threadIdx.x == 0) A.clr[y] = PAD;
    const uint64_t bk = A.cur[y];
    if (bk == PAD) return;
    bpt = key_id(bk);
  }
  stage_row_cta(cvec, a.X + (int64_t)bpt * a.ld_bytes, a.nchunks);
  __syncthreads();
  uint64_t lmin = PAD;
  for (int base = t0 + warp * STEP; base < t1; base += BIG_NW * STEP) {
    uint4 yv[L::U][L::VL][K];
#pragma unroll
    for (int u = 0; u < L::U; ++u) {
      const int idx = min(base + u * L::CPW + g, t1 - 1);
      load_slots<G, K>(a.X + (int64_t)a.item_pt[start + idx] * a.ld_bytes, a.nchunks, j, yv[u]);
    }
#pragma unroll
    for (int u = 0; u < L::U; ++u) {
      const float dd = slots_dist<METRIC, G, K>(cvec, yv[u], a.nchunks, a.d, j);
      const int idx = base + u * L::CPW + g;
      if (idx < t1 && j == 0) {
        const int64_t it = start + idx;
        const int32_t pt = a.item_pt[it];
        if (mode == 0) {
          a.kd[it] = dd;
          a.best[it] = PAD;
          a.flag[it] = 0;
          lmin = umin64(lmin, make_key(dd, pt));
        } else if (pt == bpt) {
          a.flag[it] = 2;
          a.parent[tbase + bpt] = anode;
          atomicAdd(&A.kcount[y], 1u);
        } else {
          const uint8_t f = a.flag[it];
          if (f != 2) {
            const uint64_t ck = make_key(dd, bpt);
            if (ck < a.best[it]) a.best[it] = ck;
            if (f == 0) {
              const float kdv = a.kd[it];
              if (dd <= kdv) {
                a.flag[it] = 1;
              } else {
                lmin = umin64(lmin, make_key(kdv, pt));
              }
            }
          }
        }
      }
    }
  }
  lmin = warp_min64<METRIC, G, K>(lmin);
  if (lane == 0 && lmin != PAD)
    atomicMin(reinterpret_cast<unsigned long long*>((mode == 0 ? A.cur : A.nxt) + y),
              (unsigned long long)lmin);
}

using SatBigFn = void (*)(const SatBigArgs, int);

using SatKernelFn = void (*)(const SatSegArgs);
constexpr int SAT_NW = 8;

static SatKernelFn sat_kernel_for(int metric, int G, int K) {
#define SATX(M, GG, KK) \
  if (metric == M && G == GG && K == KK) return sat_segment_kernel<M, GG, KK, SAT_NW>;
#define SATF(M) SATX(M, 4, 1) SATX(M, 8, 1) SATX(M, 16, 1) SATX(M, 32, 1) SATX(M, 32, 2) \
  SATX(M, 32, 4) SATX(M, 32, 8)
  SATF(0)
  SATF(1)
  SATX(2, 4, 1) SATX(2, 8, 1) SATX(2, 16, 1)
#undef SATF
#undef SATX
  return nullptr;
}

static SatBigFn sat_big_for(int metric, int G, int K) {
#define SATX(M, GG, KK) \
  if (metric == M && G == GG && K == KK) return sat_big_kernel<M, GG, KK>;
#define SATF(M) SATX(M, 4, 1) SATX(M, 8, 1) SATX(M, 16, 1) SATX(M, 32, 1) SATX(M, 32, 2) \
  SATX(M, 32, 4) SATX(M, 32, 8)
  SATF(0)
  SATF(1)
  SATX(2, 4, 1) SATX(2, 8, 1) SATX(2, 16, 1)
#undef SATF
#undef SATX
  return nullptr;
}

__global__ void sat_init_kernel(int64_t n, int T, const int32_t* roots, int32_t* node_of,
                                int32_t* parent) {
  const int64_t tot = (int64_t)T * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(i / n);
    const int32_t x = (int32_t)(i - (int64_t)t * n);
    node_of[i] = (x == roots[t]) ? -1 : roots[t];
    parent[i] = -1;
  }
}

__global__ void sat_count_kernel(int64_t n, int64_t tot, const int32_t* node_of, uint32_t* kcnt,
                                 uint32_t* err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = node_of[i];
    if (a >= n) {
      atomicOr(err, 1u);  // an invalid node id: recorded, never used as an index
      continue;
    }
    if (a >= 0) {
      const int64_t t = i / n;
      atomicAdd(&kcnt[t * n + a], 1u);
    }
  }
}

__global__ void sat_segments_kernel(int64_t n, int64_t tot, const uint32_t* kcnt,
                                    const int64_t* kstart, int64_t* seg_start, int32_t* seg_len,
                                    int32_t* seg_node, int32_t* seg_tree, uint32_t* nseg,
                                    int32_t big_min, int32_t* big_list, int64_t big_base) {
  for (int64_t key = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; key < tot;
       key += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t c = kcnt[key];
    if (c) {
      // small nodes fill the list from the front, big ones from big_base on
      uint32_t s;
      if ((int32_t)c >= big_min) {
        const uint32_t j = atomicAdd(nseg + 1, 1u);
        s = (uint32_t)(big_base + j);
        big_list[j] = (int32_t)s;
      } else {
        s = atomicAdd(nseg, 1u);
      }
      seg_start[s] = kstart[key];
      seg_len[s] = (int32_t)c;
      seg_node[s] = (int32_t)(key % n);
      seg_tree[s] = (int32_t)(key / n);
    }
  }
}

__global__ void sat_scatter_kernel(int64_t n, int64_t tot, const int32_t* node_of,
                                   uint32_t* kcnt, const int64_t* kstart, int32_t* item_pt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = node_of[i];
    if (a >= 0 && a < n) {
      const int64_t t = i / n;
      const int64_t key = t * n + a;
      const uint32_t r = atomicSub(&kcnt[key], 1u) - 1u;
      item_pt[kstart[key] + r] = (int32_t)(i - t * n);
    }
  }
}

static int grid_for(int64_t tot) {
  int64_t g = (tot + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 32));
}

int sat_forest(const VecLayout& L, int T, const int32_t* roots_d, int32_t* parents,
               SatScratch& S, unsigned long long* ctr_sat, cudaStream_t s) {
  SatKernelFn kern = sat_kernel_for(L.metric, L.G, L.K);
  SatBigFn bigk = sat_big_for(L.metric, L.G, L.K);
  if (!kern || !bigk) {
    set_error(1, "no SAT kernel for this metric and dimension");
    return 1;
  }
  const int64_t n = L.n, tot = (int64_t)T * n;
  sat_init_kernel<<<grid_for(tot), 256, 0, s>>>(n, T, roots_d, S.node_of, parents);
  note_launch();
  FG_CUDA(cudaGetLastError());
  SatSegArgs a;
  a.X = L.X;
  a.ld_bytes = L.ld_bytes;
  a.d = L.d;
  a.nchunks = L.nchunks;
  a.n = n;
  a.item_pt = S.item_pt;
  a.seg_start = S.seg_start;
  a.seg_len = S.seg_len;
  a.seg_node = S.seg_node;
  a.seg_tree = S.seg_tree;
  a.kd = S.kd;
  a.best = S.best;
  a.flag = S.flag;
  a.node_of = S.node_of;
  a.parent = parents;
  a.ctr = ctr_sat;
  std::vector<uint64_t> hkeys;
  for (int64_t level = 0; level <= n; ++level) {
    FG_CUDA(cudaMemsetAsync(S.nseg, 0, 3 * sizeof(uint32_t), s));
    sat_count_kernel<<<grid_for(tot), 256, 0, s>>>(n, tot, S.node_of, S.kcnt, S.nseg + 2);
    note_launch();
    int rc = scan_u32(S.kcnt, S.kstart, tot, S.scan_tmp, s);
    if (rc) return rc;
    sat_segments_kernel<<<grid_for(tot), 256, 0, s>>>(n, tot, S.kcnt, S.kstart, S.seg_start,
                                                      S.seg_len, S.seg_node, S.seg_tree, S.nseg,
                                                      S.big_min, S.big_list, tot);
    note_launch();
    sat_scatter_kernel<<<grid_for(tot), 256, 0, s>>>(n, tot, S.node_of, S.kcnt, S.kstart,
                                                     S.item_pt);
    note_launch();
    FG_CUDA(cudaGetLastError());
    uint32_t cnts[3] = {0, 0, 0};
    FG_CUDA(cudaMemcpyAsync(cnts, S.nseg, sizeof(cnts), cudaMemcpyDeviceToHost, s));
    FG_CUDA(cudaStreamSynchronize(s));
    if (cnts[2]) {
      set_error(3, "SAT: a point was assigned to an invalid node");
      return 3;
    }
    const uint32_t nsmall = cnts[0], nbig = cnts[1];
    if (nsmall == 0 && nbig == 0) return 0;
    if (nsmall) {
      kern<<<nsmall, SAT_NW * 32, 0, s>>>(a);
      note_launch();
      FG_CUDA(cudaGetLastError());
    }
    if (nbig) {
      SatBigArgs B;
      B.s = a;
      B.big = S.big_list;
      uint64_t* buf[3] = {S.big_keys, S.big_keys + nbig, S.big_keys + 2 * nbig};
      B.kcount = S.big_kcount;
      FG_CUDA(cudaMemsetAsync(S.big_keys, 0xFF, 3 * nbig * sizeof(uint64_t), s));
      FG_CUDA(cudaMemsetAsync(S.big_kcount, 0, nbig * sizeof(uint32_t), s));
      const unsigned gx = (unsigned)((n + BIG_TILE - 1) / BIG_TILE);
      // grid.y is limited to 65535: big nodes are covered in chunks
      auto launch_all = [&](int mode) {
        for (uint32_t y0 = 0; y0 < nbig; y0 += 65535u) {
          B.y_off = (int32_t)y0;
          const dim3 grid(gx, std::min<uint32_t>(65535u, nbig - y0));
          bigk<<<grid, BIG_NW * 32, 0, s>>>(B, mode);
          note_launch();
        }
      };
      B.cur = buf[0];
      B.nxt = buf[1];
      B.clr = buf[2];
      launch_all(0);
      FG_CUDA(cudaGetLastError());
      hkeys.resize(nbig);
      int r = 0;  // buf[r] holds the next child of every big node
      bool done = false;
      for (int64_t it = 0; it <= n && !done;) {
        for (int j = 0; j < 8; ++j, ++it) {
          B.cur = buf[r];
          B.nxt = buf[(r + 1) % 3];
          B.clr = buf[(r + 2) % 3];
          launch_all(1);
          r = (r + 1) % 3;
        }
        FG_CUDA(cudaGetLastError());
        FG_CUDA(cudaMemcpyAsync(hkeys.data(), buf[r], nbig * sizeof(uint64_t),
                                cudaMemcpyDeviceToHost, s));
        FG_CUDA(cudaStreamSynchronize(s));
        done = true;
        for (uint64_t k : hkeys) done &= (k == PAD);
      }
      if (!done) {
        set_error(1, "SAT child selection did not terminate");
        return 1;
      }
      launch_all(2);
      FG_CUDA(cudaGetLastError());
    }
  }
  set_error(1, "SAT construction did not terminate");
  return 1;
}

}  // namespace fg
