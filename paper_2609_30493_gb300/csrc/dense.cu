// Dense-block ceiling (Section 5.3, the blocked side of the two-ceiling model):
// a pair set fixed in advance -- every
// ordered pair of distinct members of a block -- evaluated in the canonical
// float32 order (exact integers for uint8 rows), with the k smallest
// (delta, id) kept per row.  One warp owns
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
  using L = Lanes<G, K>;
  __shared__ __align__(16) uint4 srow[8][256];  // the row's vector, per warp
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane / L::P, j = lane % L::P;
  uint4* qs = srow[warp];
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
      __syncwarp();
      stage_row(qs, a.X + (int64_t)xi * a.ld_bytes, a.nchunks, lane);
      for (int base = 0; base < a.bs; base += 32) {
        uint64_t mykey = PAD;
        for (int sub = 0; sub < 32 && base + sub < a.bs; sub += L::CPW * L::UW) {
          uint4 y[L::UW][L::VL][K];
          int32_t jd[L::UW];
#pragma unroll
          for (int u = 0; u < L::UW; ++u) {
            const int jj = base + sub + u * L::CPW + g;
            jd[u] = (jj < a.bs && jj != i) ? ids[jj] : -1;
            load_slots<G, K>(a.X + (int64_t)(jd[u] >= 0 ? jd[u] : xi) * a.ld_bytes, a.nchunks, j,
                             y[u]);
          }
#pragma unroll
          for (int u = 0; u < L::UW; ++u) {
            const float dd = slots_dist<METRIC, G, K>(qs, y[u], a.nchunks, a.d, j);
            const int rel = lane - sub - u * L::CPW;
            const float got = __shfl_sync(FULL, dd, (rel & (L::CPW - 1)) * L::P);
            const int32_t jid = __shfl_sync(FULL, jd[u], (rel & (L::CPW - 1)) * L::P);
            if (rel >= 0 && rel < L::CPW && jid >= 0) mykey = make_key(got, jid);
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
  DX(2, 4, 1) DX(2, 8, 1) DX(2, 16, 1)
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
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((rows + 7) / 8, (int64_t)device_sms() * 16));
  kern<<<grid, 256, 0, s>>>(a);
  note_launch();
  FG_CUDA(cudaGetLastError());
  return 0;
}

}  // namespace fg
