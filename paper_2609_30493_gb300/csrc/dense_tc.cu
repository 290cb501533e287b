// Dense-block ceiling on the 5th-generation tensor cores (Section 5.3: a pair
// set fixed before evaluation is a dense product and runs at arithmetic rate).
//
// Each block of up to 1024 points is centred on its float32 mean and rounded
// to BF16 (or to E4M3 with a scale per row).  dt_prep_kernel writes the
// rounded rows already in the shared-memory image the tensor cores read
// (K-major core matrices of 8 rows x 16 bytes, one 128 KB image per 128-byte
// K slice of the 1024 rows), so one bulk copy moves a whole operand tile.
//
// dt_fused_kernel is persistent (one CTA per SM) and warp-specialised:
//  - warp 8 (one lane) streams operand slices with bulk copies
//    (cp.async.bulk, completion counted on an mbarrier) into a 3-stage ring:
//    a 128-row A panel and a 256-row B chunk of the same block per stage;
//  - warp 9 (one lane) issues tcgen05.mma (128 x 256, FP32 accumulation in
//    tensor memory) into two 256-column accumulators, so that the epilogue of
//    one column chunk overlaps the products of the next;
//  - warps 0..7 read the accumulators with tcgen05.ld (thread = one row, one
//    half of the chunk's columns) and turn the Gram values into approximate
//    distances.
// The approximate distances are only a filter.  For row i, every pair of the
// exact top-k satisfies approx <= tau_k + 2 eps_i (tau_k: the k-th smallest
// approximate distance of the row; eps_i bounds |approx - canonical| for all
// its pairs): approx <= canonical + eps <= k-th canonical + eps
// <= tau_k + 2 eps.  The row's tau_k is located by a two-level histogram
// (32 bins over the row's value range, then 32 sub-bins of the bin holding
// the k-th value) in two passes over the products, and a third pass collects
// the columns whose approximate distance is at most an upper bound of tau_k
// plus 2 eps; the tensor-core products are recomputed for each pass (they
// cost far less than storing 1024 x 1024 distances).  dt_rerank_kernel then
// evaluates the collected pairs in the canonical float32 order and keeps the
// k smallest (delta, id): the result equals the canonical float32 top-k.
//
// eps_i comes from the rows' actual rounding residuals, not from the unit
// roundoff: with q the rounded centred rows, r_i = |x_i - q_i| and
// Qx = max_j |q_j|, Rq = max_j r_j, Mx = max_j |x_j| over the block,
//   |<q_i,q_j> - <x_i,x_j>| <= r_i Qx + |x_i| Rq        (Cauchy-Schwarz),
// plus the FP32 accumulation error gamma_K |q_i| Qx (any order), the float32
// norms, the centring and the canonical distance's own rounding, all times a
// safety factor of 2 (the tensor cores' accumulation order is undocumented).
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "dense_tc.cuh"
#include "internal.h"
#include "rowops.cuh"
#include "tc.cuh"

namespace fg {

// --------------------------------------------------------------------------
// 1. Centre, round, write the tile images; per-row and per-block norms
// --------------------------------------------------------------------------
// Grid (nb, 4): CTA (b, y) centres and rounds rows 256 y .. 256 y + 255 of
// block b.  The block mean is summed in one fixed order by every CTA: warp w
// adds the rows r = w, w + 8, w + 16, .. in turn, then the eight partial
// sums are added in warp order.
__global__ void __launch_bounds__(256) dt_prep_kernel(const DtArgs a) {
  __shared__ float mu[1024];
  __shared__ float part[8][128];
  __shared__ int nval;
  const int64_t blk = blockIdx.x;
  const int y = blockIdx.y;
  const int32_t* ids = a.block_ids + blk * a.bs;
  const int lane0 = threadIdx.x & 31, warp0 = threadIdx.x >> 5;
  if (threadIdx.x == 0) nval = 0;
  __syncthreads();
  int cnt = 0;
  for (int r = threadIdx.x; r < a.bs; r += blockDim.x) cnt += ids[r] >= 0;
  atomicAdd(&nval, cnt);
  __syncthreads();
  const int nv = nval;
  const float inv = nv > 0 ? 1.0f / (float)nv : 0.0f;
  if (threadIdx.x == 0 && y == 0) {
    a.nvalid[blk] = (uint32_t)nv;
    if (nv > 1) atomicAdd(a.pairs, (unsigned long long)nv * (unsigned long long)(nv - 1));
  }
  for (int j0 = 0; j0 < a.d; j0 += 128) {
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int r = warp0; r < a.bs; r += 8) {
      const int32_t id = ids[r];
      if (id < 0) continue;
      const float* xr = reinterpret_cast<const float*>(a.X + (int64_t)id * a.ld_bytes);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int j = j0 + lane0 + 32 * e;
        if (j < a.d) acc[e] += xr[j];
      }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) part[warp0][lane0 + 32 * e] = acc[e];
    __syncthreads();
    if (threadIdx.x < 128 && j0 + (int)threadIdx.x < a.d) {
      float s = part[0][threadIdx.x];
      for (int w = 1; w < 8; ++w) s += part[w][threadIdx.x];
      mu[j0 + threadIdx.x] = a.nocentre ? 0.0f : s * inv;
    }
    __syncthreads();
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int epu = a.fp8 ? 16 : 8;  // elements per 16-byte unit
  const int nunits = a.rowb / 16;
  unsigned char* img = a.Xt + blk * (int64_t)a.nsl * DT_SLICE_IMG;
  for (int r = 256 * y + warp; r < 256 * y + 256; r += 8) {
    const int32_t id = r < a.bs ? ids[r] : -1;
    const float* xr = id >= 0 ? reinterpret_cast<const float*>(a.X + (int64_t)id * a.ld_bytes)
                              : nullptr;
    // E4M3: the row's largest centred magnitude maps to 448, the largest
    // finite E4M3 value
    float scale = 1.0f;
    if (a.fp8) {
      float mx = 0.0f;
      if (id >= 0)
        for (int j = lane; j < a.d; j += 32) mx = fmaxf(mx, fabsf(xr[j] - mu[j]));
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, off));
      scale = mx > 0.0f ? mx / 448.0f : 1.0f;
    }
    const float rs = 1.0f / scale;
    float s2 = 0.0f, x2 = 0.0f, r2 = 0.0f, q2 = 0.0f;
    for (int u = lane; u < nunits; u += 32) {
      uint32_t w[4] = {0u, 0u, 0u, 0u};
      for (int e = 0; e < epu; ++e) {
        const int j = u * epu + e;
        float v = 0.0f;
        if (id >= 0 && j < a.d) {
          const float x = xr[j];
          v = x - mu[j];
          x2 = __fmaf_rn(x, x, x2);
        }
        s2 = __fmaf_rn(v, v, s2);
        float deq;
        uint32_t bits;
        if (a.fp8) {
          const __nv_fp8_storage_t c = __nv_cvt_float_to_fp8(v * rs, __NV_SATFINITE, __NV_E4M3);
          __nv_fp8_e4m3 qv;
          qv.__x = c;
          deq = scale * static_cast<float>(qv);
          bits = (uint32_t)c;
          w[e >> 2] |= bits << (8 * (e & 3));
        } else {
          const __nv_bfloat16 b = __float2bfloat16_rn(v);
          deq = __bfloat162float(b);
          bits = (uint32_t)__bfloat16_as_ushort(b);
          w[e >> 1] |= bits << (16 * (e & 1));
        }
        const float dr = v - deq;
        r2 = __fmaf_rn(dr, dr, r2);
        q2 = __fmaf_rn(deq, deq, q2);
      }
      const int sl = u >> 3, kb = (u & 7) * 16;
      *reinterpret_cast<uint4*>(img + (int64_t)sl * DT_SLICE_IMG + tile_off(r, kb)) =
          make_uint4(w[0], w[1], w[2], w[3]);
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
      s2 += __shfl_xor_sync(FULL, s2, off);
      x2 += __shfl_xor_sync(FULL, x2, off);
      r2 += __shfl_xor_sync(FULL, r2, off);
      q2 += __shfl_xor_sync(FULL, q2, off);
    }
    if (lane == 0) {
      const int64_t ri = blk * DT_ROWS + r;
      const float cc = id >= 0 ? 0.5f * (1.0f - x2) : 0.0f;
      a.rowA[ri] = make_float4(s2, cc, scale, id >= 0 ? 1.0f : 0.0f);
      a.rowB[ri] = make_float4(sqrtf(r2), sqrtf(q2), x2, 0.0f);
      if (id >= 0) {
        unsigned int* bs = reinterpret_cast<unsigned int*>(a.bst + blk * 8);
        atomicMax(bs + 0, __float_as_uint(sqrtf(s2)));
        atomicMax(bs + 1, __float_as_uint(sqrtf(r2)));
        atomicMax(bs + 2, __float_as_uint(sqrtf(q2)));
        atomicMax(bs + 3, __float_as_uint(x2));
        atomicMax(bs + 4, __float_as_uint(fmaxf(cc, 0.0f)));
      }
    }
  }
}

// --------------------------------------------------------------------------
// 2. Persistent fused Gram + filter
// --------------------------------------------------------------------------
struct DtSmem {
  static constexpr int hist = DT_STAGES * DT_STAGE_BYTES;            // [NBIN + 1][256] u32
  static constexpr int col = hist + (DT_NBIN + 1) * DT_EPI * 4;      // [1024] float2
  static constexpr int rowcnt = col + DT_ROWS * 8;                   // [128] u32
  static constexpr int xcnt = rowcnt + DT_M * 4;                     // [256] u32
  static constexpr int xval = xcnt + DT_EPI * 4;                     // [256] f32
  static constexpr int bars = xval + DT_EPI * 4;                     // 16 x u64
  static constexpr int misc = bars + 16 * 8;                         // tmem address, flags
  static constexpr int bytes = misc + 16;
};

__device__ __forceinline__ int dt_bin(float x, float lo, float iw) {
  const int b = __float2int_rz((x - lo) * iw);
  return min(DT_NBIN - 1, max(0, b));
}

// Per-thread state of one row in the filter's epilogue.
struct DtRow {
  float base;  // row term of the approximate distance
  float f;     // Gram factor (1 angular, 2 squared L2; times the row's E4M3 scale)
  int i;       // the row's column index (its own pair is skipped)
  float lo, iw1, lo2, iw2, ucut;
  int b1, s2;
  uint32_t cin;
  float vmax, vmin;
};

// The 32 Gram values v of columns j0..j0+31 for one row.  The approximate
// distance is base_i + col_j - f * g (angular: base = |x_i|^2 / 2 + c_i with
// the centred norm and c = (1 - |x|^2) / 2, f = 1; squared L2: base =
// |x_i|^2, f = 2; for E4M3 g is scaled by the column's scale here and by the
// row's in f).  Invalid columns carry col = +inf.  PASS 0 counts the values
// in the first-level bins, PASS 1 the sub-bins of bin b1, PASS 2 collects
// the candidates (the Gram-only mode's minimum is dt_gram_min).  Counts are
// shared-memory atomics whose results are not used, so they do not wait on
// one another.
template <int PASS, bool FP8>
__device__ __forceinline__ void dt_values(const uint32_t (&v)[32], const float2* col, int j0,
                                          DtRow& r, uint32_t* hcol, uint32_t* rowcnt_il,
                                          uint16_t* cand, float* cdt) {
  // no branch per value: a value that does not count goes to the unused bin
  // DT_NBIN, and the candidates of PASS 2 are appended from a bit mask
  uint32_t take = 0;
  float dts[32];
#pragma unroll
  for (int t = 0; t < 32; ++t) {
    const int j = j0 + t;
    const float2 cj = col[j];
    float g = __uint_as_float(v[t]);
    if (FP8) g *= cj.y;
    const float dt = __fmaf_rn(-r.f, g, r.base + cj.x);
    const bool ok = dt < INFINITY && j != r.i;
    if (PASS == 0) {
      atomicAdd(hcol + (ok ? dt_bin(dt, r.lo, r.iw1) : DT_NBIN) * DT_EPI, 1u);
    } else if (PASS == 1) {
      const bool in = ok && dt_bin(dt, r.lo, r.iw1) == r.b1;
      atomicAdd(hcol + (in ? dt_bin(dt, r.lo2, r.iw2) : DT_NBIN) * DT_EPI, 1u);
    } else if (PASS == 2) {
      const int k1 = dt_bin(dt, r.lo, r.iw1);
      const bool inkey = ok && (k1 < r.b1 || (k1 == r.b1 && dt_bin(dt, r.lo2, r.iw2) <= r.s2));
      r.cin += inkey ? 1u : 0u;
      r.vmax = inkey ? fmaxf(r.vmax, dt) : r.vmax;
      take |= (inkey || (ok && dt <= r.ucut)) ? (1u << t) : 0u;
      dts[t] = dt;
    }
  }
  if (PASS == 2) {
    while (take) {
      const int t = __ffs(take) - 1;
      take &= take - 1u;
      const uint32_t pos = atomicAdd(rowcnt_il, 1u);
      cand[pos] = (uint16_t)(j0 + t);
      if (cdt) {
        float dv = 0.0f;
#pragma unroll
        for (int q = 0; q < 32; ++q) dv = q == t ? dts[q] : dv;
        cdt[pos] = dv;
      }
    }
  }
}

// Gram-only mode: the smallest (column term - f g) of 32 columns, two
// columns per shared-memory read and two instructions per value; the row
// term is added once at the end.  Only the group that holds the row's own
// column (the same group for every lane of a warp) takes the slow path.
template <bool FP8>
__device__ __forceinline__ void dt_gram_min(const uint32_t (&v)[32], const float2* col, int j0,
                                            int i, float f, float& m) {
  const float4* c4 = reinterpret_cast<const float4*>(col + j0);
  if ((unsigned)(i - j0) >= 32u) {
#pragma unroll
    for (int t = 0; t < 32; t += 2) {
      const float4 cc = c4[t >> 1];
      float2 g = make_float2(__uint_as_float(v[t]), __uint_as_float(v[t + 1]));
      if (FP8) g = __fmul2_rn(g, make_float2(cc.y, cc.w));
      const float2 y = __ffma2_rn(make_float2(-f, -f), g, make_float2(cc.x, cc.z));
      m = fminf(m, fminf(y.x, y.y));
    }
  } else {
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      const float2 cj = col[j0 + t];
      float g = __uint_as_float(v[t]);
      if (FP8) g *= cj.y;
      const float y = __fmaf_rn(-f, g, cj.x);
      m = (j0 + t != i) ? fminf(m, y) : m;
    }
  }
}

__global__ void __launch_bounds__(DT_THREADS, 1) dt_fused_kernel(const DtArgs a) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  unsigned char* stages = dsm;
  uint32_t* hist = reinterpret_cast<uint32_t*>(dsm + DtSmem::hist);
  float4* coldata = reinterpret_cast<float4*>(dsm + DtSmem::col);
  uint32_t* rowcnt = reinterpret_cast<uint32_t*>(dsm + DtSmem::rowcnt);
  uint32_t* xcnt = reinterpret_cast<uint32_t*>(dsm + DtSmem::xcnt);
  float* xval = reinterpret_cast<float*>(dsm + DtSmem::xval);
  uint64_t* bars = reinterpret_cast<uint64_t*>(dsm + DtSmem::bars);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(dsm + DtSmem::misc);
  int* abort_flag = reinterpret_cast<int*>(dsm + DtSmem::misc + 4);
  int* zero_flag = reinterpret_cast<int*>(dsm + DtSmem::misc + 8);
  uint64_t* full = bars;        // [3] operand stage landed
  uint64_t* empty = bars + 3;   // [3] operand stage consumed by its MMAs
  uint64_t* tfull = bars + 6;   // [2] accumulator complete
  uint64_t* tempty = bars + 8;  // [2] accumulator read by the epilogue
  uint64_t* done = bars + 10;   // every MMA of the CTA complete
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < DT_STAGES; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull + b, 1);
      mbar_init(tempty + b, DT_EPI);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    *zero_flag = 0;
    fence_mbar_init();
  }
  if (warp == 9) {
    tmem_alloc(tmem_slot, DT_TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const volatile int* abortp = abort_flag;
  const int64_t ntiles = a.nb * (DT_ROWS / DT_M);
  const int npass = a.mode == 0 ? 1 : 3;
  const int nch = DT_ROWS / DT_NC;

  if (warp == 8) {
    // ---- producer: operand slices into the stage ring ----
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int64_t blk = tile >> 3;
        const int rt = (int)(tile & 7);
        const unsigned char* base = a.Xt + blk * (int64_t)a.nsl * DT_SLICE_IMG;
        for (int pass = 0; pass < npass && ok; ++pass)
          for (int c = 0; c < nch && ok; ++c)
            for (int sl = 0; sl < a.nsl; ++sl, ++it) {
              const uint32_t s = it % DT_STAGES, ph = (it / DT_STAGES) & 1u;
              if (!mbar_wait_backoff(empty + s, ph ^ 1u, a.wait_polls, abortp, 64)) {
                ok = false;
                break;
              }
              unsigned char* dst = stages + s * DT_STAGE_BYTES;
              const unsigned char* src = base + (int64_t)sl * DT_SLICE_IMG;
              mbar_arrive_expect_tx(full + s, DT_STAGE_BYTES);
              bulk_g2s(dst, src + rt * DT_A_BYTES, DT_A_BYTES, full + s);
              bulk_g2s(dst + DT_A_BYTES, src + c * DT_B_BYTES, DT_B_BYTES, full + s);
            }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(a.err, 1u);
      }
      // every issued copy lands before the CTA may exit
      for (uint32_t s = 0; s < DT_STAGES; ++s) {
        if (it <= s) continue;
        const uint32_t last = s + DT_STAGES * ((it - 1 - s) / DT_STAGES);
        mbar_wait_bounded(full + s, (last / DT_STAGES) & 1u, kDrainPolls, zero_flag);
      }
    }
  } else if (warp == 9) {
    // ---- MMA issuer ----
    if (lane == 0) {
      const uint32_t idesc = a.fp8 ? idesc_e4m3(DT_M, DT_NC) : idesc_bf16(DT_M, DT_NC);
      uint32_t it = 0, ci = 0;
      bool ok = true;
      for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x)
        for (int pass = 0; pass < npass && ok; ++pass)
          for (int c = 0; c < nch && ok; ++c, ++ci) {
            const uint32_t buf = ci & 1u, bph = (ci >> 1) & 1u;
            if (!mbar_wait_backoff(tempty + buf, bph ^ 1u, a.wait_polls, abortp, 64)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t dt = tmem + buf * DT_NC;
            for (int sl = 0; sl < a.nsl; ++sl, ++it) {
              const uint32_t s = it % DT_STAGES, ph = (it / DT_STAGES) & 1u;
              if (!mbar_wait_backoff(full + s, ph, a.wait_polls, abortp, 32)) {
                ok = false;
                break;
              }
              tc_fence_after();
              const uint32_t a0 = smem_u32(stages + s * DT_STAGE_BYTES);
              const uint32_t b0 = a0 + DT_A_BYTES;
#pragma unroll
              for (int kk = 0; kk < 4; ++kk) {
                // one MMA takes 32 K bytes (16 BF16 or 32 E4M3 elements): two
                // core matrices along K (2 x 128 bytes of shared memory)
                const uint64_t ad = smem_desc(a0 + kk * 256, 128, 1024);
                const uint64_t bd = smem_desc(b0 + kk * 256, 128, 1024);
                const uint32_t acc = (sl > 0 || kk > 0) ? 1u : 0u;
                if (a.fp8)
                  mma_e4m3(dt, ad, bd, idesc, acc);
                else
                  mma_bf16(dt, ad, bd, idesc, acc);
              }
              mma_commit(empty + s);  // the stage is free once these products are done
            }
            if (ok) mma_commit(tfull + buf);
          }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(a.err, 1u);
      }
      // every product issued lands before the tensor memory is released
      mma_commit(done);
      mbar_wait_bounded(done, 0u, kDrainPolls, zero_flag);
    }
  } else {
    // ---- epilogue: warps 0..7, thread = (row il, column half h) ----
    const int etid = tid;  // 0..255
    const int q = warp & 3, h = warp >> 2;
    const int il = 32 * q + lane;
    const bool ang = a.metric == ANGULAR_F32;
    float2* col = reinterpret_cast<float2*>(coldata);
    uint32_t* hcol = hist + etid;
    uint32_t ci = 0;
    bool aborted = false;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      const int64_t blk = tile >> 3;
      const int rt = (int)(tile & 7);
      const int i = rt * DT_M + il;
      for (int j = etid; j < DT_ROWS; j += DT_EPI) {
        const float4 cj = a.rowA[blk * DT_ROWS + j];
        const float cterm = ang ? __fmaf_rn(0.5f, cj.x, cj.y) : cj.x;
        col[j] = make_float2(j < a.bs && cj.w != 0.0f ? cterm : INFINITY, cj.z);
      }
      if (etid < DT_M) rowcnt[etid] = 0u;
      for (int b = 0; b < DT_NBIN; ++b) hcol[b * DT_EPI] = 0u;
      aborted = named_sync_or(1, DT_EPI, aborted || *abortp);
      if (aborted) break;
      // row constants and the error bound eps of this row (see the file header)
      const float4 ra = a.rowA[blk * DT_ROWS + i];
      const float4 rb = a.rowB[blk * DT_ROWS + i];
      const float* bst = a.bst + blk * 8;
      const float Mx = bst[0], Rq = bst[1], Qx = bst[2], X2m = bst[3], Cm = bst[4];
      const bool vrow = ra.w != 0.0f && i < a.bs;
      const float ni = ra.x, cci = ra.y, si = ra.z;
      const float ri = rb.x, qi = rb.y, x2i = rb.z;
      const float eps = dt_row_eps(ang, a.dpad, a.d, ni, ri, qi, x2i, Mx, Rq, Qx, X2m);
      DtRow r;
      r.base = ang ? __fmaf_rn(0.5f, ni, cci) : ni;
      r.f = (ang ? 1.0f : 2.0f) * (a.fp8 ? si : 1.0f);
      r.i = vrow ? i : -1;
      // value range of the row's approximate distances for the histogram
      const float span = ni + Mx * Mx + 2.0f * qi * Qx;
      r.lo = 0.0f;
      float hi = ang ? 0.5f * span + cci + Cm : span;
      if (!(hi > r.lo + 1e-30f)) hi = r.lo + 1.0f;
      r.iw1 = (float)DT_NBIN / (hi - r.lo);
      r.lo2 = r.lo;
      r.iw2 = r.iw1;
      r.ucut = 0.0f;
      r.b1 = 0;
      r.s2 = DT_NBIN - 1;
      r.cin = 0;
      r.vmax = -INFINITY;
      r.vmin = INFINITY;
      const int nvr = vrow ? (int)a.nvalid[blk] - 1 : 0;
      const bool all_mode = nvr <= a.k;
      uint32_t below = 0;
      uint16_t* crow = a.cand + (blk * DT_ROWS + i) * (int64_t)DT_ROWS;
      float* cdrow = a.cdt ? a.cdt + (blk * DT_ROWS + i) * (int64_t)DT_ROWS : nullptr;
      for (int pass = 0; pass < npass && !aborted; ++pass) {
        // rows that take every valid column need no histogram
        const int kind = a.mode == 0 ? 3 : (all_mode && pass < 2 ? -1 : pass);
        if (all_mode && pass == 2) r.b1 = DT_NBIN;  // every bin is below b1: all collected
        for (int c = 0; c < nch; ++c, ++ci) {
          const uint32_t buf = ci & 1u, bph = (ci >> 1) & 1u;
          if (!aborted && !mbar_wait_bounded(tfull + buf, bph, a.wait_polls, abortp))
            aborted = true;
          // tcgen05.ld is warp-collective: the warp goes on only if every lane's wait ended
          aborted = __any_sync(FULL, aborted);
          if (!aborted && kind == 3) {
            // Gram-only: two loads in flight per wait
            tc_fence_after();
#pragma unroll 1
            for (int t4 = 0; t4 < 4; t4 += 2) {
              const int cb = h * 128 + 32 * t4;
              uint32_t v0[32], v1[32];
              const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + buf * DT_NC + (uint32_t)cb;
              tmem_ld32_async(ta, v0);
              tmem_ld32_async(ta + 32, v1);
              tmem_wait_ld();
              tmem_ld_fence(v0);
              tmem_ld_fence(v1);
              if (!vrow) continue;
              const int j0 = c * DT_NC + cb;
              if (a.fp8) {
                dt_gram_min<true>(v0, col, j0, r.i, r.f, r.vmin);
                dt_gram_min<true>(v1, col, j0 + 32, r.i, r.f, r.vmin);
              } else {
                dt_gram_min<false>(v0, col, j0, r.i, r.f, r.vmin);
                dt_gram_min<false>(v1, col, j0 + 32, r.i, r.f, r.vmin);
              }
            }
          } else if (!aborted) {
            tc_fence_after();
#pragma unroll 1
            for (int t4 = 0; t4 < 4; ++t4) {
              const int cb = h * 128 + 32 * t4;  // first column within the chunk
              uint32_t v[32];
              tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + buf * DT_NC + (uint32_t)cb, v);
              if (!vrow || kind < 0) continue;
              const int j0 = c * DT_NC + cb;
              if (a.fp8) {
                if (kind == 0) dt_values<0, true>(v, col, j0, r, hcol, rowcnt + il, crow, cdrow);
                else if (kind == 1) dt_values<1, true>(v, col, j0, r, hcol, rowcnt + il, crow, cdrow);
                else dt_values<2, true>(v, col, j0, r, hcol, rowcnt + il, crow, cdrow);
              } else {
                if (kind == 0) dt_values<0, false>(v, col, j0, r, hcol, rowcnt + il, crow, cdrow);
                else if (kind == 1) dt_values<1, false>(v, col, j0, r, hcol, rowcnt + il, crow, cdrow);
                else dt_values<2, false>(v, col, j0, r, hcol, rowcnt + il, crow, cdrow);
              }
            }
          }
          tc_fence_before();
          mbar_arrive(tempty + buf);
        }
        if (a.mode == 0) {
          xval[etid] = r.vmin;
          aborted = named_sync_or(1, DT_EPI, aborted || *abortp);
          if (!aborted && h == 0 && i < a.bs)
            a.rowmin[blk * a.bs + i] = vrow ? r.base + fminf(r.vmin, xval[etid ^ 128]) : INFINITY;
          break;
        }
        if (pass == 2) {
          xcnt[etid] = r.cin;
          xval[etid] = r.vmax;
        }
        aborted = named_sync_or(1, DT_EPI, aborted || *abortp);
        if (aborted) break;
        if (pass == 0 && !all_mode) {
          uint32_t cum = 0;
          r.b1 = DT_NBIN - 1;
          for (int b = 0; b < DT_NBIN; ++b) {
            const uint32_t cnt = hcol[b * DT_EPI] + hist[b * DT_EPI + (etid ^ 128)];
            if (cum + cnt >= (uint32_t)a.k) {
              r.b1 = b;
              break;
            }
            cum += cnt;
          }
          below = cum;
          r.lo2 = r.lo + (float)r.b1 / r.iw1;
          r.iw2 = r.iw1 * (float)DT_NBIN;
        } else if (pass == 1 && !all_mode) {
          uint32_t cum = below;
          r.s2 = DT_NBIN - 1;
          for (int b = 0; b < DT_NBIN; ++b) {
            cum += hcol[b * DT_EPI] + hist[b * DT_EPI + (etid ^ 128)];
            if (cum >= (uint32_t)a.k) {
              r.s2 = b;
              break;
            }
          }
          const float ub = r.lo2 + (float)(r.s2 + 1) / r.iw2;
          r.ucut = ub + 2.0f * eps + 1e-6f * (fabsf(r.lo) + (hi - r.lo)) + 1e-30f;
        } else if (pass == 2 && h == 0) {
          // the collected columns hold every pair within 2 eps of the k-th
          // approximate distance when at least k values lie at or below the
          // sub-bin of the k-th value and 2 eps above their largest is still
          // under the cut; otherwise the row takes every valid column
          uint32_t n = rowcnt[il];
          if (vrow && !all_mode) {
            const uint32_t tin = r.cin + xcnt[etid ^ 128];
            const float top = fmaxf(r.vmax, xval[etid ^ 128]);
            float need = top + 2.0f * eps;
            need += fabsf(need) * 2.4e-7f;
            if (tin < (uint32_t)a.k || !(need <= r.ucut)) n = DT_FALLBACK;
          }
          a.ccnt[blk * DT_ROWS + i] = vrow ? n : 0u;
          if (a.reps) a.reps[blk * DT_ROWS + i] = eps;
        }
        if (pass == 0) {
          // the partner's histogram column has been read: clear this one
          aborted = named_sync_or(1, DT_EPI, aborted || *abortp);
          if (aborted) break;
          for (int b = 0; b < DT_NBIN; ++b) hcol[b * DT_EPI] = 0u;
        }
      }
      aborted = named_sync_or(1, DT_EPI, aborted || *abortp);
      if (aborted) break;
    }
    // a wait of the epilogue that gave up is an error too (and stops the others)
    if (aborted && etid == 0) {
      *abort_flag = 1;
      atomicOr(a.err, 1u);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 9) {
    tc_fence_after();
    tmem_dealloc(tmem, DT_TMEM_COLS);
  }
}

// --------------------------------------------------------------------------
// 3. Per row: canonical rerank of the collected columns, top-k
// --------------------------------------------------------------------------
constexpr int RR_WARPS = 4;

// One warp per row.  The collected columns (every valid column when the
// filter could not bound the row) are taken 32 at a time; lane groups of P
// lanes evaluate them in the canonical float32 order with the row's vector
// in registers, and each batch is merged into a register pool of the k
// smallest (delta, id) by the bitonic network of the harvest (the keys of a
// row are distinct: a block's members are distinct points).  S = pool slots
// of 32 (k <= 32 S).
template <int METRIC, int G, int K, int S>
__global__ void __launch_bounds__(RR_WARPS * 32)
    dt_rerank_kernel(const DtArgs a, int32_t* out_ids, float* out_dist) {
  using L = Lanes<G, K>;
  extern __shared__ __align__(16) unsigned char ssm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane / L::P, j = lane % L::P;
  const int nch = (a.d * 4 + 15) / 16;
  uint4* qs = reinterpret_cast<uint4*>(ssm + warp * 16 * nch);
  const int64_t rows = a.nb * a.bs;
  unsigned long long nre = 0;
  for (int64_t r = (int64_t)blockIdx.x * RR_WARPS + warp; r < rows;
       r += (int64_t)gridDim.x * RR_WARPS) {
    const int64_t blk = r / a.bs;
    const int i = (int)(r - blk * a.bs);
    const int32_t* ids = a.block_ids + blk * a.bs;
    const int32_t xi = ids[i];
    uint64_t pool[S];
#pragma unroll
    for (int s = 0; s < S; ++s) pool[s] = PAD;
    // after a give-up of the filter kernel its candidate lists are not valid
    if (xi >= 0 && *reinterpret_cast<const volatile uint32_t*>(a.err) == 0u) {
      const int64_t crow = (blk * DT_ROWS + i) * (int64_t)DT_ROWS;
      const uint32_t m0 = a.ccnt[blk * DT_ROWS + i];
      const bool fallback = m0 == DT_FALLBACK || m0 >= (uint32_t)a.bs;
      const int total = fallback ? a.bs : (int)m0;  // fallback: scan every column
      const float eps = a.reps ? a.reps[blk * DT_ROWS + i] : 0.0f;
      stage_row(qs, a.X + (int64_t)xi * a.ld_bytes, nch, lane);
      uint4 qr[L::VL][K];
      load_slots_smem<G, K>(qs, nch, j, qr);
      for (int base = 0; base < total; base += 32) {
        // this lane's candidate of the batch: its column, id, approximate distance
        int col = -1;
        float adt = 0.0f;
        if (base + lane < total) {
          if (fallback) {
            const int c = base + lane;
            col = (c != i && ids[c] >= 0) ? c : -1;
          } else {
            const uint32_t cv = a.cand[crow + base + lane];
            col = cv < (uint32_t)a.bs ? (int)cv : -1;
            if (a.errstat) adt = a.cdt[crow + base + lane];
          }
        }
        const int32_t myid = col >= 0 ? ids[col] : -1;
        nre += (unsigned long long)__popc(__ballot_sync(FULL, col >= 0));
        uint64_t mykey = PAD;
        for (int sb = 0; sb < 32; sb += L::CPW * L::UW) {
          uint4 y[L::UW][L::VL][K];
#pragma unroll
          for (int uu = 0; uu < L::UW; ++uu) {
            const int idx = sb + uu * L::CPW + g;
            const int32_t cid = __shfl_sync(FULL, myid, idx);
            load_slots<G, K>(a.X + (int64_t)(cid >= 0 ? cid : xi) * a.ld_bytes, nch, j, y[uu]);
          }
#pragma unroll
          for (int uu = 0; uu < L::UW; ++uu) {
            const float dd = regs_dist<METRIC, G, K>(qr, y[uu], nch, a.d, j, FULL);
            const int rel = lane - sb - uu * L::CPW;
            const float got = __shfl_sync(FULL, dd, (rel & (L::CPW - 1)) * L::P);
            if (rel >= 0 && rel < L::CPW && myid >= 0) mykey = make_key(got, myid);
          }
        }
        if (a.errstat && !fallback && myid >= 0) {
          // the same pair in float64 (plain order): the filter's error
          // relative to the bound used, the canonical value's absolute error
          const float* xa = reinterpret_cast<const float*>(a.X + (int64_t)xi * a.ld_bytes);
          const float* xb = reinterpret_cast<const float*>(a.X + (int64_t)myid * a.ld_bytes);
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
          const float e1 = (float)(fabs((double)adt - d64) / (double)eps);
          const float e2 = (float)fabs((double)key_dist(mykey) - d64);
          atomicMax(a.err + 8, __float_as_uint(e1));
          atomicMax(a.err + 9, __float_as_uint(e2));
        }
        merge_into_pool<S>(pool, mykey, a.k, lane);
      }
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const int t = s * 32 + lane;
      if (t < a.k) {
        out_ids[r * a.k + t] = pool[s] == PAD ? -1 : key_id(pool[s]);
        out_dist[r * a.k + t] = pool[s] == PAD ? __int_as_float(0x7f800000) : key_dist(pool[s]);
      }
    }
  }
  if (lane == 0 && nre) atomicAdd(a.reranked, nre);
}

using RerankFn = void (*)(const DtArgs, int32_t*, float*);

static RerankFn rerank_kernel_for(int metric, int G, int K, int S) {
#define SX(M, GG, KK, SS) \
  if (metric == M && G == GG && K == KK && S == SS) return dt_rerank_kernel<M, GG, KK, SS>;
#define SS_(M, GG, KK) SX(M, GG, KK, 1) SX(M, GG, KK, 2)
#define SF(M) SS_(M, 4, 1) SS_(M, 8, 1) SS_(M, 16, 1) SS_(M, 32, 1) SS_(M, 32, 2) \
  SS_(M, 32, 4) SS_(M, 32, 8)
  SF(0)
  SF(1)
#undef SF
#undef SS_
#undef SX
  return nullptr;
}

// --------------------------------------------------------------------------
// Host side
// --------------------------------------------------------------------------
namespace {

// Blocks per launch group: the candidate lists take 2 MB per block (and the
// approximate distances for the error check 4 MB more).
constexpr int64_t kGroup = 64;
constexpr int64_t kGroupErr = 16;

struct DtScratch {
  char* base = nullptr;
  size_t off = 0;
  template <typename T>
  T* take(size_t count) {
    T* p = reinterpret_cast<T*>(base + off);
    off += (sizeof(T) * count + 255) / 256 * 256;
    return p;
  }
};

size_t dt_scratch_bytes(int64_t gn, int nsl, bool errstat) {
  size_t b = 0;
  auto add = [&](size_t x) { b += (x + 255) / 256 * 256; };
  add((size_t)gn * nsl * DT_SLICE_IMG);      // Xt
  add(sizeof(float4) * gn * DT_ROWS * 2);    // rowA, rowB
  add(sizeof(float) * gn * 8);               // bst
  add(sizeof(uint32_t) * gn);                // nvalid
  add(sizeof(uint16_t) * gn * DT_ROWS * DT_ROWS);
  add(sizeof(uint32_t) * gn * DT_ROWS);      // ccnt
  if (errstat) {
    add(sizeof(float) * gn * DT_ROWS * DT_ROWS);
    add(sizeof(float) * gn * DT_ROWS);
  }
  add(256);                                  // err, pairs, reranked
  return b;
}

int dt_setup(const VecLayout& L, int fp8, DtArgs* a) {
  a->X = L.X;
  a->ld_bytes = L.ld_bytes;
  a->d = L.d;
  a->metric = L.metric;
  a->fp8 = fp8 ? 1 : 0;
  const int slice = a->fp8 ? DT_KB : DT_KB / 2;  // elements per slice
  a->dpad = (L.d + slice - 1) / slice * slice;
  a->rowb = a->fp8 ? a->dpad : 2 * a->dpad;
  a->nsl = a->rowb / DT_KB;
  a->wait_polls = g_mma_wait_polls;
  cudaError_t e = raise_smem_limit(reinterpret_cast<const void*>(dt_fused_kernel), DtSmem::bytes);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(dt_fused_kernel)");
  return 0;
}

}  // namespace

int dense_block_tc(const VecLayout& L, const int32_t* block_ids, int64_t nb, int bs, int k,
                   int fp8, bool err64, int32_t* out_ids, float* out_dist, double* stats,
                   cudaStream_t s) {
  RerankFn rr = rerank_kernel_for(L.metric, L.G, L.K, k <= 32 ? 1 : 2);
  if (!rr || L.metric == L2_U8) {
    set_error(1, "tensor-core dense blocks take float32 metrics");
    return 1;
  }
  if (bs > DT_ROWS || nb > 65535) {
    set_error(1, "tensor-core dense blocks: bs <= 1024 and nb <= 65535");
    return 1;
  }
  DtArgs a{};
  int rc = dt_setup(L, fp8, &a);
  if (rc) return rc;
  a.errstat = stats && err64 ? 1 : 0;
  a.bs = bs;
  a.k = k;
  a.mode = 1;
  const int64_t group = a.errstat ? kGroupErr : kGroup;
  const int64_t gmax = std::min<int64_t>(nb, group);
  const size_t total = dt_scratch_bytes(gmax, a.nsl, a.errstat != 0);
  const int nch = (L.d * 4 + 15) / 16;
  const int rsm = RR_WARPS * 16 * nch;
  {
    cudaError_t e = raise_smem_limit(reinterpret_cast<const void*>(rr), rsm);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(dt_rerank_kernel)");
  }
  char* scratch = nullptr;
  FG_CUDA(cudaMallocAsync(&scratch, total, s));
  cudaEvent_t ev[4] = {};
  for (int i = 0; i < 4 && stats; ++i) cudaEventCreate(&ev[i]);
  float t_prep = 0.0f, t_fused = 0.0f, t_rr = 0.0f;
  uint32_t h[10] = {};
  unsigned long long pairs = 0, reranked = 0;
  for (int64_t b0 = 0; b0 < nb && !rc; b0 += group) {
    const int64_t gn = std::min<int64_t>(group, nb - b0);
    DtScratch S{scratch, 0};
    a.block_ids = block_ids + b0 * bs;
    a.nb = gn;
    a.Xt = S.take<unsigned char>((size_t)gn * a.nsl * DT_SLICE_IMG);
    a.rowA = S.take<float4>(gn * DT_ROWS);
    a.rowB = S.take<float4>(gn * DT_ROWS);
    a.bst = S.take<float>(gn * 8);
    a.nvalid = S.take<uint32_t>(gn);
    a.cand = S.take<uint16_t>((size_t)gn * DT_ROWS * DT_ROWS);
    a.ccnt = S.take<uint32_t>(gn * DT_ROWS);
    a.cdt = a.errstat ? S.take<float>((size_t)gn * DT_ROWS * DT_ROWS) : nullptr;
    a.reps = a.errstat ? S.take<float>(gn * DT_ROWS) : nullptr;
    a.err = S.take<uint32_t>(64);
    a.pairs = reinterpret_cast<unsigned long long*>(a.err + 2);
    a.reranked = reinterpret_cast<unsigned long long*>(a.err + 4);
    cudaError_t e;
    if ((e = cudaMemsetAsync(a.bst, 0, sizeof(float) * gn * 8, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(a.err, 0, 256, s)) != cudaSuccess) {
      rc = cuda_fail(e, "cudaMemsetAsync(dense scratch)");
      break;
    }
    if (stats) cudaEventRecord(ev[0], s);
    dt_prep_kernel<<<dim3((unsigned)gn, DT_ROWS / 256), 256, 0, s>>>(a);
    note_launch();
    if (stats) cudaEventRecord(ev[1], s);
    const int64_t ntiles = gn * (DT_ROWS / DT_M);
    const int grid = (int)std::min<int64_t>(ntiles, device_sms());
    dt_fused_kernel<<<grid, DT_THREADS, DtSmem::bytes, s>>>(a);
    note_launch();
    if (stats) cudaEventRecord(ev[2], s);
    const int64_t rows = gn * bs;
    const int rgrid = (int)std::max<int64_t>(
        1, std::min<int64_t>((rows + RR_WARPS - 1) / RR_WARPS, (int64_t)device_sms() * 16));
    rr<<<rgrid, RR_WARPS * 32, rsm, s>>>(a, out_ids + b0 * bs * k, out_dist + b0 * bs * k);
    note_launch();
    if (stats) cudaEventRecord(ev[3], s);
    if ((e = cudaGetLastError()) != cudaSuccess) {
      rc = cuda_fail(e, "dense tensor-core kernels");
      break;
    }
    uint32_t hg[10] = {};
    if ((e = cudaMemcpyAsync(hg, a.err, 40, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess) {
      rc = cuda_fail(e, "dense tensor-core status");
      break;
    }
    if (hg[0]) {
      set_error(5, "tensor-core dense block: a bounded wait for the MMA gave up");
      rc = 5;
      break;
    }
    pairs += (unsigned long long)hg[2] | ((unsigned long long)hg[3] << 32);
    reranked += (unsigned long long)hg[4] | ((unsigned long long)hg[5] << 32);
    h[8] = std::max(h[8], hg[8]);  // non-negative float bits order like the floats
    h[9] = std::max(h[9], hg[9]);
    if (stats) {
      float t1 = 0, t2 = 0, t3 = 0;
      cudaEventElapsedTime(&t1, ev[0], ev[1]);
      cudaEventElapsedTime(&t2, ev[1], ev[2]);
      cudaEventElapsedTime(&t3, ev[2], ev[3]);
      t_prep += t1;
      t_fused += t2;
      t_rr += t3;
    }
  }
  if (!rc && stats) {
    stats[0] = pairs ? (double)reranked / (double)pairs : 0.0;
    stats[1] = t_fused;
    stats[2] = t_rr;
    stats[3] = t_prep;
    float m1, m2;
    std::memcpy(&m1, &h[8], 4);
    std::memcpy(&m2, &h[9], 4);
    stats[4] = m1;
    stats[5] = m2;
  }
  for (int i = 0; i < 4 && stats; ++i) cudaEventDestroy(ev[i]);
  cudaFreeAsync(scratch, s);
  return rc;
}

int dense_gram_tc(const VecLayout& L, const int32_t* block_ids, int64_t nb, int bs, int fp8,
                  float* out_min, double* ms, cudaStream_t s) {
  if (L.metric == L2_U8) {
    set_error(1, "tensor-core dense blocks take float32 metrics");
    return 1;
  }
  if (bs > DT_ROWS || nb > 65535) {
    set_error(1, "tensor-core dense blocks: bs <= 1024 and nb <= 65535");
    return 1;
  }
  DtArgs a{};
  int rc = dt_setup(L, fp8, &a);
  if (rc) return rc;
  a.bs = bs;
  a.k = 1;
  a.mode = 0;
  const int64_t group = 256;
  const int64_t gmax = std::min<int64_t>(nb, group);
  size_t total = 0;
  {
    auto add = [&](size_t x) { total += (x + 255) / 256 * 256; };
    add((size_t)gmax * a.nsl * DT_SLICE_IMG);
    add(sizeof(float4) * gmax * DT_ROWS * 2);
    add(sizeof(float) * gmax * 8);
    add(sizeof(uint32_t) * gmax);
    add(256);
  }
  char* scratch = nullptr;
  FG_CUDA(cudaMallocAsync(&scratch, total, s));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (ms) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
  }
  float tsum = 0.0f;
  for (int64_t b0 = 0; b0 < nb && !rc; b0 += group) {
    const int64_t gn = std::min<int64_t>(group, nb - b0);
    DtScratch S{scratch, 0};
    a.block_ids = block_ids + b0 * bs;
    a.nb = gn;
    a.Xt = S.take<unsigned char>((size_t)gn * a.nsl * DT_SLICE_IMG);
    a.rowA = S.take<float4>(gn * DT_ROWS);
    a.rowB = S.take<float4>(gn * DT_ROWS);
    a.bst = S.take<float>(gn * 8);
    a.nvalid = S.take<uint32_t>(gn);
    a.err = S.take<uint32_t>(64);
    a.pairs = reinterpret_cast<unsigned long long*>(a.err + 2);
    a.reranked = reinterpret_cast<unsigned long long*>(a.err + 4);
    a.rowmin = out_min + b0 * bs;
    cudaError_t e;
    if ((e = cudaMemsetAsync(a.bst, 0, sizeof(float) * gn * 8, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(a.err, 0, 256, s)) != cudaSuccess) {
      rc = cuda_fail(e, "cudaMemsetAsync(dense scratch)");
      break;
    }
    dt_prep_kernel<<<dim3((unsigned)gn, DT_ROWS / 256), 256, 0, s>>>(a);
    note_launch();
    if (ms) cudaEventRecord(e0, s);
    const int grid = (int)std::min<int64_t>(gn * (DT_ROWS / DT_M), device_sms());
    dt_fused_kernel<<<grid, DT_THREADS, DtSmem::bytes, s>>>(a);
    note_launch();
    if (ms) cudaEventRecord(e1, s);
    uint32_t hg = 0;
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(&hg, a.err, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess) {
      rc = cuda_fail(e, "dense Gram kernel");
      break;
    }
    if (hg) {
      set_error(5, "tensor-core dense block: a bounded wait for the MMA gave up");
      rc = 5;
      break;
    }
    if (ms) {
      float t = 0.0f;
      cudaEventElapsedTime(&t, e0, e1);
      tsum += t;
    }
  }
  if (!rc && ms) *ms = tsum;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(scratch, s);
  return rc;
}

}  // namespace fg
