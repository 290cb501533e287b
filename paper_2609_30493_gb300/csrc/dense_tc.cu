// Dense-block ceiling on the 5th-generation tensor cores (Section 5.3: a pair
// set fixed before evaluation is a dense product and runs at arithmetic rate).
//
// Each block of up to 1024 points is centred on its float32 mean and rounded
// to BF16; its Gram matrix is computed by tcgen05.mma (kind::f16, BF16 in,
// FP32 accumulated in tensor memory), one 128 x 256 tile per CTA, and turned
// into approximate distances.  They are only a filter: per row, every pair
// whose approximate distance is within 2*eps of the k-th smallest is
// recomputed in the canonical float32 order and the k smallest (delta, id) are
// selected from those, where eps bounds |approximate - canonical| for the row
// (BF16 input rounding, FP32 accumulation in any order, the canonical sum's
// own rounding; times 2).  For every pair of the exact top-k,
// approx <= canonical + eps <= k-th canonical + eps <= k-th approx + 2 eps, so
// the result equals the canonical float32 top-k.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "internal.h"
#include "rowops.cuh"
#include "tc.cuh"

namespace fg {

constexpr int TC_ROWS = 1024;  // rows of a block after padding
constexpr int TC_M = 128;      // rows per CTA (one per TMEM lane)
constexpr int TC_N = 256;      // columns per CTA (TMEM columns)
constexpr int TC_KB = 128;     // K bytes per staged slice (8 core matrices of 16 bytes)
constexpr int TC_THREADS = 128;
constexpr uint32_t TC_TMEM_COLS = 256;

// Byte offset of the 16-byte unit (row r, byte kb) of a staged K-slice: core
// matrix (r/8, kb/16) at (r/8)*1024 + (kb/16)*128, row r%8 at +16*(r%8).
// A slice is 64 BF16 or 128 E4M3 elements per row.
__host__ __device__ constexpr uint32_t tile_off(int r, int kb) {
  return (uint32_t)((r >> 3) * 1024 + (kb >> 4) * 128 + (r & 7) * 16);
}

// --------------------------------------------------------------------------
// 1. Centre, round to BF16, norms
// --------------------------------------------------------------------------
struct TcArgs {
  const char* X;
  int64_t ld_bytes;
  int32_t d;
  int32_t dpad;  // d rounded up to a whole slice (64 BF16 or 128 E4M3 elements)
  int32_t rowb;  // bytes of a rounded row (2 dpad or dpad)
  int32_t fp8;   // 0: BF16, 1: E4M3 with a scale per row
  float u_in;    // unit roundoff of the input rounding (with the E4M3 subnormal term)
  int32_t metric;
  const int32_t* block_ids;
  int64_t nb;
  int32_t bs;
  unsigned char* Xb;  // [nb][1024][rowb]
  float* sc;          // [nb][1024] E4M3 row scale (the row is sc * its codes)
  float* nrm;         // [nb][1024] squared norm of the centred float32 row
  float* cc;          // [nb][1024] angular: (1 - |x|^2) / 2
  float* Mx;          // [nb] largest centred norm
  float* LP;          // [nb][1024][1024] approximate distances
  uint32_t* err;  // [0] timeout flag, [8] and [9] error maxima (float bits)
  unsigned long long* pairs;  // valid ordered pairs over all blocks
  int32_t errstat;  // measure the filter's error against float64 on the reranked pairs
  int32_t wait_polls;  // first bounded wait for a slice's products
};

__global__ void __launch_bounds__(256) dense_prep_kernel(const TcArgs a) {
  __shared__ float mu[1024];
  __shared__ int nvalid;
  const int64_t blk = blockIdx.x;
  const int32_t* ids = a.block_ids + blk * a.bs;
  if (threadIdx.x == 0) nvalid = 0;
  __syncthreads();
  int cnt = 0;
  for (int r = threadIdx.x; r < a.bs; r += blockDim.x) cnt += ids[r] >= 0;
  atomicAdd(&nvalid, cnt);
  __syncthreads();
  const float inv = nvalid > 0 ? 1.0f / (float)nvalid : 0.0f;
  if (threadIdx.x == 0 && nvalid > 1)
    atomicAdd(a.pairs, (unsigned long long)nvalid * (unsigned long long)(nvalid - 1));
  for (int j = threadIdx.x; j < a.d; j += blockDim.x) {
    float s = 0.0f;
    for (int r = 0; r < a.bs; ++r) {
      const int32_t id = ids[r];
      if (id >= 0) s += reinterpret_cast<const float*>(a.X + (int64_t)id * a.ld_bytes)[j];
    }
    mu[j] = s * inv;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int r = warp; r < TC_ROWS; r += 8) {
    const int32_t id = r < a.bs ? ids[r] : -1;
    unsigned char* dst = a.Xb + (blk * TC_ROWS + r) * (int64_t)a.rowb;
    float s2 = 0.0f, x2 = 0.0f;
    const float* xr = id >= 0 ? reinterpret_cast<const float*>(a.X + (int64_t)id * a.ld_bytes)
                              : nullptr;
    // E4M3: the row's largest centred magnitude maps to 448, the largest
    // finite E4M3 value
    float scale = 1.0f;
    if (a.fp8) {
      float mx = 0.0f;
      for (int j = lane; j < a.d; j += 32)
        if (id >= 0) mx = fmaxf(mx, fabsf(xr[j] - mu[j]));
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, off));
      scale = mx > 0.0f ? mx / 448.0f : 1.0f;
    }
    const float rs = 1.0f / scale;
    for (int j = lane; j < a.dpad; j += 32) {
      float v = 0.0f;
      if (id >= 0 && j < a.d) {
        const float x = xr[j];
        v = x - mu[j];
        x2 = __fmaf_rn(x, x, x2);
      }
      s2 = __fmaf_rn(v, v, s2);
      if (a.fp8)
        dst[j] = (unsigned char)__nv_cvt_float_to_fp8(v * rs, __NV_SATFINITE, __NV_E4M3);
      else
        reinterpret_cast<__nv_bfloat16*>(dst)[j] = __float2bfloat16_rn(v);
    }
    if (lane == 0) a.sc[blk * TC_ROWS + r] = scale;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
      s2 += __shfl_xor_sync(FULL, s2, off);
      x2 += __shfl_xor_sync(FULL, x2, off);
    }
    if (lane == 0) {
      a.nrm[blk * TC_ROWS + r] = s2;
      a.cc[blk * TC_ROWS + r] = id >= 0 ? 0.5f * (1.0f - x2) : 0.0f;
      if (id >= 0) atomicMax(reinterpret_cast<unsigned int*>(a.Mx + blk), __float_as_uint(sqrtf(s2)));
    }
  }
}

// --------------------------------------------------------------------------
// 2. Gram tile on the tensor cores and approximate distances
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(TC_THREADS) dense_gram_kernel(const TcArgs a) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  unsigned char* As = tsm;                      // 128 rows x 128 bytes = 16 KB
  unsigned char* Bs = tsm + TC_M * TC_KB;       // 256 rows x 128 bytes = 32 KB
  uint64_t* bar = reinterpret_cast<uint64_t*>(Bs + TC_N * TC_KB);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 1);
  const int rt = blockIdx.x, ct = blockIdx.y;
  const int64_t blk = blockIdx.z;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  if (warp == 0) {
    tmem_alloc(tmem_slot, TC_TMEM_COLS);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const unsigned char* Ag = a.Xb + (blk * TC_ROWS + rt * TC_M) * (int64_t)a.rowb;
  const unsigned char* Bg = a.Xb + (blk * TC_ROWS + ct * TC_N) * (int64_t)a.rowb;
  const uint32_t idesc = a.fp8 ? idesc_e4m3(TC_M, TC_N) : idesc_bf16(TC_M, TC_N);
  bool ok = true;
  const int nslices = a.rowb / TC_KB;
  for (int sl = 0; sl < nslices; ++sl) {
    const int k0 = sl * TC_KB;
    // stage the slices: 16-byte units (row, 16 K bytes), 8 per row
    for (int u = tid; u < TC_M * 8; u += TC_THREADS) {
      const int r = u >> 3, kc = u & 7;
      *reinterpret_cast<uint4*>(As + tile_off(r, kc * 16)) =
          *reinterpret_cast<const uint4*>(Ag + (int64_t)r * a.rowb + k0 + kc * 16);
    }
    for (int u = tid; u < TC_N * 8; u += TC_THREADS) {
      const int r = u >> 3, kc = u & 7;
      *reinterpret_cast<uint4*>(Bs + tile_off(r, kc * 16)) =
          *reinterpret_cast<const uint4*>(Bg + (int64_t)r * a.rowb + k0 + kc * 16);
    }
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        // one MMA takes 32 K bytes (16 BF16 or 32 E4M3 elements): two core
        // matrices along K (2 x 128 bytes of shared memory)
        const uint64_t ad = smem_desc(a0 + kk * 256, 128, 1024);
        const uint64_t bd = smem_desc(b0 + kk * 256, 128, 1024);
        if (a.fp8)
          mma_e4m3(tmem, ad, bd, idesc, (sl > 0 || kk > 0) ? 1u : 0u);
        else
          mma_bf16(tmem, ad, bd, idesc, (sl > 0 || kk > 0) ? 1u : 0u);
      }
      mma_commit(bar);
    }
    // wait (bounded) for the slice's products before its buffers are reused;
    // every thread takes the same decision
    bool done = false;
    for (int it = 0; it < a.wait_polls && !done; ++it) done = mbar_try_wait(bar, sl & 1);
    done = __syncthreads_and(done);
    if (!done) {
      ok = false;
      if (tid == 0) atomicOr(a.err, 1u);
      // let the slice's products land before the tensor memory is released
      for (int it = 0; it < kDrainPolls; ++it)
        if (mbar_try_wait(bar, sl & 1)) break;
      break;
    }
    tc_fence_after();
  }

  if (ok) {
    // epilogue: warp w reads TMEM lanes 32w..32w+31 (rows), 32 columns at a time
    const int i = rt * TC_M + warp * 32 + lane;
    const int64_t rowbase = blk * TC_ROWS;
    const float ni = a.nrm[rowbase + i];
    const float ci = a.cc[rowbase + i];
    const float si = a.fp8 ? a.sc[rowbase + i] : 1.0f;
    // each warp passes its 32 x 32 blocks through shared memory (the staging
    // buffers are free now) so that every store writes one 128-byte row piece
    float* stg = reinterpret_cast<float*>(tsm) + warp * 32 * 33;
    float* out0 = a.LP + (rowbase + rt * TC_M + warp * 32) * (int64_t)TC_ROWS + ct * TC_N;
    for (int c0 = 0; c0 < TC_N; c0 += 32) {
      uint32_t v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
      for (int t = 0; t < 32; ++t) {
        const int j = ct * TC_N + c0 + t;
        const float g = a.fp8 ? __uint_as_float(v[t]) * (si * a.sc[rowbase + j])
                              : __uint_as_float(v[t]);
        const float s = a.nrm[rowbase + j] + ni - 2.0f * g;
        stg[lane * 33 + t] = a.metric == ANGULAR_F32 ? 0.5f * s + ci + a.cc[rowbase + j] : s;
      }
      __syncwarp();
      for (int rr = 0; rr < 32; ++rr) out0[(int64_t)rr * TC_ROWS + c0 + lane] = stg[rr * 33 + lane];
      __syncwarp();
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, TC_TMEM_COLS);
}

// --------------------------------------------------------------------------
// 3. Per row: filter threshold, canonical rerank of the candidates, top-k
// --------------------------------------------------------------------------
constexpr int SEL_WARPS = 4;

template <int METRIC, int G, int K>
__global__ void __launch_bounds__(SEL_WARPS * 32)
    dense_select_kernel(const TcArgs a, int k, int32_t* out_ids, float* out_dist,
                        unsigned long long* reranked) {
  using L = Lanes<G, K>;
  extern __shared__ __align__(16) unsigned char ssm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane / L::P, j = lane % L::P;
  const int nch = (a.d * 4 + 15) / 16;
  const int wbytes = 8 * TC_ROWS + 16 * nch;
  uint64_t* keys = reinterpret_cast<uint64_t*>(ssm + warp * wbytes);
  uint4* qs = reinterpret_cast<uint4*>(ssm + warp * wbytes + 8 * TC_ROWS);
  const int64_t rows = a.nb * a.bs;
  const float u_b = a.u_in, gam = 1.0f / 16777216.0f;
  const float dk = (float)(a.d + 8);
  unsigned long long nre = 0;
  for (int64_t r = (int64_t)blockIdx.x * SEL_WARPS + warp; r < rows;
       r += (int64_t)gridDim.x * SEL_WARPS) {
    const int64_t blk = r / a.bs;
    const int i = (int)(r - blk * a.bs);
    const int32_t* ids = a.block_ids + blk * a.bs;
    const int32_t xi = ids[i];
    int kk = 0;
    if (xi >= 0) {
      const float* lp = a.LP + (blk * TC_ROWS + i) * (int64_t)TC_ROWS;
      // lane holds columns lane + 32 t; invalid columns get the largest key
      uint32_t u[TC_ROWS / 32];
      int nv = 0;
#pragma unroll
      for (int t = 0; t < TC_ROWS / 32; ++t) {
        const int c = lane + 32 * t;
        const bool valid = c < a.bs && c != i && ids[c] >= 0;
        u[t] = valid ? fkey(lp[c]) : 0xFFFFFFFFu;
        nv += valid ? 1 : 0;
      }
      nv = __reduce_add_sync(FULL, nv);
      // eps for this row (see the file header)
      const float Ai = sqrtf(a.nrm[blk * TC_ROWS + i]), M = a.Mx[blk];
      float eps = 2.0f * ((4.0f * u_b + 6.0f * dk * gam) * Ai * M +
                          6.0f * dk * gam * (Ai * Ai + M * M));
      if (a.metric == ANGULAR_F32) eps = 0.5f * eps + 2.0f * (3.0f * dk * gam + 2.0f * gam);
      // candidates: every valid column when there are at most k, else those
      // with approx <= tau + 2 eps, tau the k-th smallest approximate value,
      // found bit by bit (the largest t with fewer than k keys below t)
      uint32_t lim = 0xFFFFFFFEu;
      if (nv > k) {
        uint32_t t = 0;
        for (int bit = 31; bit >= 0; --bit) {
          const uint32_t tt = t | (1u << bit);
          int below = 0;
#pragma unroll
          for (int q = 0; q < TC_ROWS / 32; ++q) below += u[q] < tt ? 1 : 0;
          if (__reduce_add_sync(FULL, below) < k) t = tt;
        }
        lim = fkey(fkey_inv(t) + 2.0f * eps);
      }
      int cand = 0;
#pragma unroll
      for (int q = 0; q < TC_ROWS / 32; ++q) {
        const bool in = u[q] <= lim;
        const unsigned m = __ballot_sync(FULL, in);
        if (in) keys[cand + __popc(m & ((1u << lane) - 1u))] = (uint64_t)(lane + 32 * q);
        cand += __popc(m);
      }
      __syncwarp();
      nre += (unsigned long long)cand;
      // canonical distances of the candidates, in place
      stage_row(qs, a.X + (int64_t)xi * a.ld_bytes, nch, lane);
      for (int base = 0; base < cand; base += L::CPW) {
        const int c = base + g;
        // groups past the candidates load the row's own vector (keys[0..base)
        // already hold (distance, id) keys, not column indices)
        const int32_t cid = c < cand ? ids[(int)(uint32_t)keys[c]] : xi;
        uint4 y[L::VL][K];
        load_slots<G, K>(a.X + (int64_t)cid * a.ld_bytes, nch, j, y);
        const float dd = slots_dist<METRIC, G, K>(qs, y, nch, a.d, j);
        __syncwarp();
        if (c < cand && j == 0) {
          if (a.errstat) {
            // the same pair in float64 (plain order): the filter's error
            // relative to the bound used, the canonical value's absolute error
            const float* xa = reinterpret_cast<const float*>(a.X + (int64_t)xi * a.ld_bytes);
            const float* xb = reinterpret_cast<const float*>(a.X + (int64_t)cid * a.ld_bytes);
            double acc = 0.0;
            for (int e = 0; e < a.d; ++e) {
              if (METRIC == ANGULAR_F32) {
                acc += (double)xa[e] * (double)xb[e];
              } else {
                const double t = (double)xa[e] - (double)xb[e];
                acc += t * t;
              }
            }
            const double d64 = METRIC == ANGULAR_F32 ? 1.0 - acc : acc;
            const int col = (int)(uint32_t)keys[c];
            const float e1 = (float)(fabs((double)lp[col] - d64) / (double)eps);
            const float e2 = (float)fabs((double)dd - d64);
            atomicMax(a.err + 8, __float_as_uint(e1));
            atomicMax(a.err + 9, __float_as_uint(e2));
          }
          keys[c] = make_key(dd, cid);
        }
        __syncwarp();
      }
      kk = sort_unique(keys, cand, lane);
      kk = kk < k ? kk : k;
    }
    for (int t = lane; t < k; t += 32) {
      out_ids[r * k + t] = t < kk ? key_id(keys[t]) : -1;
      out_dist[r * k + t] = t < kk ? key_dist(keys[t]) : __int_as_float(0x7f800000);
    }
    __syncwarp();
  }
  if (lane == 0 && nre) atomicAdd(reranked, nre);
}

using SelectFn = void (*)(const TcArgs, int, int32_t*, float*, unsigned long long*);

static SelectFn select_kernel_for(int metric, int G, int K) {
#define SX(M, GG, KK) \
  if (metric == M && G == GG && K == KK) return dense_select_kernel<M, GG, KK>;
#define SF(M) SX(M, 4, 1) SX(M, 8, 1) SX(M, 16, 1) SX(M, 32, 1) SX(M, 32, 2) SX(M, 32, 4) \
  SX(M, 32, 8)
  SF(0)
  SF(1)
#undef SF
#undef SX
  return nullptr;
}

int dense_block_tc(const VecLayout& L, const int32_t* block_ids, int64_t nb, int bs, int k,
                   int fp8, bool err64, int32_t* out_ids, float* out_dist, double* stats,
                   cudaStream_t s) {
  SelectFn sel = select_kernel_for(L.metric, L.G, L.K);
  if (!sel || L.metric == L2_U8) {
    set_error(1, "tensor-core dense blocks take float32 metrics");
    return 1;
  }
  if (bs > TC_ROWS || nb > 65535) {
    set_error(1, "tensor-core dense blocks: bs <= 1024 and nb <= 65535");
    return 1;
  }
  TcArgs a{};
  a.X = L.X;
  a.ld_bytes = L.ld_bytes;
  a.d = L.d;
  a.fp8 = fp8 ? 1 : 0;
  a.errstat = stats && err64 ? 1 : 0;
  a.wait_polls = g_mma_wait_polls;
  const int slice = a.fp8 ? TC_KB : TC_KB / 2;  // elements per slice
  a.dpad = (L.d + slice - 1) / slice * slice;
  a.rowb = a.fp8 ? a.dpad : 2 * a.dpad;
  // input rounding: BF16 2^-8; E4M3 2^-4 plus its subnormal spacing, at most
  // 2^-10 of a code, summed over d elements of a row scaled to 448
  a.u_in = a.fp8 ? 0.0625f + sqrtf((float)L.d) * (1.0f / 1024.0f) / 448.0f : 1.0f / 256.0f;
  a.metric = L.metric;
  a.block_ids = block_ids;
  a.nb = nb;
  a.bs = bs;
  char* scratch = nullptr;
  const size_t xb = (size_t)nb * TC_ROWS * (size_t)a.rowb;
  const size_t vec = sizeof(float) * nb * TC_ROWS;
  const size_t lp = sizeof(float) * nb * (size_t)TC_ROWS * TC_ROWS;
  const size_t total = xb + 3 * vec + 256 * ((nb * 4 + 255) / 256 + 1) + lp + 512;
  FG_CUDA(cudaMallocAsync(&scratch, total, s));
  size_t off = 0;
  a.Xb = reinterpret_cast<unsigned char*>(scratch + off);
  off += (xb + 255) / 256 * 256;
  a.sc = reinterpret_cast<float*>(scratch + off);
  off += (vec + 255) / 256 * 256;
  a.nrm = reinterpret_cast<float*>(scratch + off);
  off += (vec + 255) / 256 * 256;
  a.cc = reinterpret_cast<float*>(scratch + off);
  off += (vec + 255) / 256 * 256;
  a.Mx = reinterpret_cast<float*>(scratch + off);
  off += (nb * 4 + 255) / 256 * 256;
  a.err = reinterpret_cast<uint32_t*>(scratch + off);
  a.pairs = reinterpret_cast<unsigned long long*>(scratch + off + 8);
  unsigned long long* reranked = reinterpret_cast<unsigned long long*>(scratch + off + 16);
  off += 256;
  a.LP = reinterpret_cast<float*>(scratch + off);
  int rc = 0;
  cudaEvent_t ev[4] = {};
  for (int i = 0; i < 4 && stats; ++i) cudaEventCreate(&ev[i]);
  do {
    cudaError_t e;
    if ((e = cudaMemsetAsync(a.Mx, 0, nb * sizeof(float), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(a.err, 0, 256, s)) != cudaSuccess) {
      rc = cuda_fail(e, "cudaMemsetAsync(dense scratch)");
      break;
    }
    if (stats) cudaEventRecord(ev[0], s);
    dense_prep_kernel<<<(unsigned)nb, 256, 0, s>>>(a);
    note_launch();
    if (stats) cudaEventRecord(ev[1], s);
    const int gsm = 100 * 1024;  // 48 KB used; asking for more keeps 2 CTAs (512 TMEM columns) per SM
    if ((e = cudaFuncSetAttribute(dense_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  gsm)) != cudaSuccess) {
      rc = cuda_fail(e, "cudaFuncSetAttribute(dense_gram_kernel)");
      break;
    }
    dense_gram_kernel<<<dim3(TC_ROWS / TC_M, TC_ROWS / TC_N, (unsigned)nb), TC_THREADS, gsm, s>>>(a);
    note_launch();
    if (stats) cudaEventRecord(ev[2], s);
    const int nch = (L.d * 4 + 15) / 16;
    const int ssm = SEL_WARPS * (8 * TC_ROWS + 16 * nch);
    if ((e = cudaFuncSetAttribute(sel, cudaFuncAttributeMaxDynamicSharedMemorySize, ssm)) !=
        cudaSuccess) {
      rc = cuda_fail(e, "cudaFuncSetAttribute(dense_select_kernel)");
      break;
    }
    const int64_t rows = nb * bs;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((rows + SEL_WARPS - 1) / SEL_WARPS,
                                                                 (int64_t)device_sms() * 16));
    sel<<<grid, SEL_WARPS * 32, ssm, s>>>(a, k, out_ids, out_dist, reranked);
    note_launch();
    if (stats) cudaEventRecord(ev[3], s);
    if ((e = cudaGetLastError()) != cudaSuccess) {
      rc = cuda_fail(e, "dense tensor-core kernels");
      break;
    }
    uint32_t h[10] = {};
    if ((e = cudaMemcpyAsync(h, a.err, 40, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess) {
      rc = cuda_fail(e, "dense tensor-core status");
      break;
    }
    if (h[0]) {
      set_error(5, "tensor-core dense block: a bounded wait for the MMA gave up");
      rc = 5;
      break;
    }
    if (stats) {
      const unsigned long long pairs = (unsigned long long)h[2] | ((unsigned long long)h[3] << 32);
      const unsigned long long rr = (unsigned long long)h[4] | ((unsigned long long)h[5] << 32);
      float t1 = 0, t2 = 0, t3 = 0;
      cudaEventElapsedTime(&t1, ev[0], ev[1]);
      cudaEventElapsedTime(&t2, ev[1], ev[2]);
      cudaEventElapsedTime(&t3, ev[2], ev[3]);
      stats[0] = pairs ? (double)rr / (double)pairs : 0.0;
      stats[1] = t2;
      stats[2] = t3;
      stats[3] = t1;
      float m1, m2;
      std::memcpy(&m1, &h[8], 4);
      std::memcpy(&m2, &h[9], 4);
      stats[4] = m1;
      stats[5] = m2;
    }
  } while (0);
  for (int i = 0; i < 4 && stats; ++i) cudaEventDestroy(ev[i]);
  cudaFreeAsync(scratch, s);
  return rc;
}

}  // namespace fg
