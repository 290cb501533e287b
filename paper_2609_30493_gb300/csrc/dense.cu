// Dense-block ceiling (Section 5.3, the blocked side of the two-ceiling model):
// a pair set fixed in advance -- every
// ordered pair of distinct members of a block -- evaluated in the canonical
// float32 order, with the k smallest (delta, id) kept per row.  One warp owns
// one row; the row's own vector sits in registers and the block's vectors
// stream through L1/L2 in 16-byte chunks.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace fg {

struct DenseArgs {
  const char* X;
  int64_t ld_bytes;
  int32_t d;
  int32_t nchunks;
  const int32_t* block_ids;
  int64_t nb;
  int32_t bs;
  int32_t k;
  int32_t* out_ids;
  float* out_dist;
};

template <int METRIC, int G, int K, int S>
__global__ void __launch_bounds__(256) dense_rows_kernel(const DenseArgs a) {
  constexpr int GPW = 32 / G;
  constexpr int U = Unroll<G, K>::value;
  const int lane = threadIdx.x & 31;
  const int g = lane / G, gl = lane % G;
  const int64_t rows = a.nb * a.bs;
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; r < rows;
       r += ((int64_t)gridDim.x * blockDim.x) / 32) {
    const int64_t blk = r / a.bs;
    const int i = (int)(r - blk * a.bs);
    const int32_t* ids = a.block_ids + blk * a.bs;
    const int32_t xi = ids[i];
    uint64_t pool[S];
#pragma unroll
    for (int s = 0; s < S; ++s) pool[s] = PAD;
    if (xi >= 0) {
      uint4 q[K];
      load_chunks<METRIC, G, K>(a.X + (int64_t)xi * a.ld_bytes, a.nchunks, gl, q);
      for (int base = 0; base < a.bs; base += 32) {
        uint64_t mykey = PAD;
        for (int sub = 0; sub < 32 && base + sub < a.bs; sub += GPW * U) {
          uint4 v[U][K];
          int32_t jd[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int j = base + sub + u * GPW + g;
            jd[u] = (j < a.bs && j != i) ? ids[j] : -1;
            if (jd[u] >= 0) {
              load_chunks<METRIC, G, K>(a.X + (int64_t)jd[u] * a.ld_bytes, a.nchunks, gl, v[u]);
            } else {
#pragma unroll
              for (int kk = 0; kk < K; ++kk) v[u][kk] = make_uint4(0u, 0u, 0u, 0u);
            }
          }
#pragma unroll
          for (int u = 0; u < U; ++u) {
            float dd = group_reduce<METRIC, G>(partial<METRIC, G, K>(q, v[u], a.d, gl));
            const int rel = lane - sub - u * GPW;
            float got = __shfl_sync(FULL, dd, (rel & (GPW - 1)) * G);
            const int32_t jid = __shfl_sync(FULL, jd[u], (rel & (GPW - 1)) * G);
            if (rel >= 0 && rel < GPW && jid >= 0) mykey = make_key(got, jid);
          }
        }
        merge_into_pool<S>(pool, mykey, a.k, lane);
      }
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const int t = s * 32 + lane;
      if (t < a.k) {
        a.out_ids[r * a.k + t] = pool[s] == PAD ? -1 : key_id(pool[s]);
        a.out_dist[r * a.k + t] = pool[s] == PAD ? __int_as_float(0x7f800000) : key_dist(pool[s]);
      }
    }
  }
}

using DenseKernelFn = void (*)(const DenseArgs);

static DenseKernelFn dense_kernel_for(int metric, int G, int K, int S) {
#define DX(M, GG, KK)                                                   \
  if (metric == M && G == GG && K == KK) {                              \
    if (S == 1) return dense_rows_kernel<M, GG, KK, 1>;                 \
    if (S == 2) return dense_rows_kernel<M, GG, KK, 2>;                 \
  }
#define DF(M) DX(M, 4, 1) DX(M, 8, 1) DX(M, 16, 1) DX(M, 32, 1) DX(M, 32, 2) DX(M, 32, 4) \
  DX(M, 32, 8)
  DF(0)
  DF(1)
#undef DF
#undef DX
  return nullptr;
}

int dense_block(const VecLayout& L, const int32_t* block_ids, int64_t nb, int bs, int k,
                int32_t* out_ids, float* out_dist, cudaStream_t s) {
  const int S = k <= 32 ? 1 : 2;
  DenseKernelFn kern = dense_kernel_for(L.metric, L.G, L.K, S);
  if (!kern) {
    set_error(1, "no dense kernel for this metric and dimension");
    return 1;
  }
  DenseArgs a{L.X, L.ld_bytes, L.d, L.nchunks, block_ids, nb, bs, k, out_ids, out_dist};
  const int64_t rows = nb * bs;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((rows + 7) / 8, 152 * 16));
  kern<<<grid, 256, 0, s>>>(a);
  note_launch();
  FG_CUDA(cudaGetLastError());
  return 0;
}

}  // namespace fg
