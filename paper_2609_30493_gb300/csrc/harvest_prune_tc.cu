// Occlusion prune on the tensor cores (Section 3): dominance bits of the
// harvest's and the final graph's candidate lists from a TF32 Gram matrix,
// with the canonical float32 test wherever the Gram value cannot decide.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "hprune.cuh"
#include "internal.h"
#include "tc.cuh"
#include "tcdist.cuh"

namespace fg {

// ---------------------------------------------------------------------------
// Tensor-core variant for the float32 metrics and lists of at most 128.
//
// The candidates are staged once, as float32, in the canonical K-major
// operand layout of tcgen05 (core matrices of 8 rows x 16 bytes); their Gram
// matrix C C^T is one chain of kind::tf32 MMAs (M = N = 128, 128 TMEM
// columns), which reads the same float32 words with the low mantissa bits
// ignored.  Thread i then reads row i of the Gram matrix from TMEM and
// decides each bit j > i from the approximate distance when the decision is
// certain: with |approx - canonical| <= eps (input rounding to 10 mantissa
// bits, float32 accumulation in any order, the canonical sum's own rounding,
// times 2), the canonical test fl(alpha2 * delta) <= delta(p, c_j) has the
// same outcome whenever alpha2 * (approx +- eps) lies on one side of
// delta(p, c_j) with a margin for the rounding of the test.  Otherwise the
// thread computes the canonical float32 distance itself, in the same order
// as the lane-group kernels (virtual lane l sums elements 128k + 4l + c by
// fused multiply-adds, then the pairwise tree over the lanes).  The bits,
// and so the prune, are identical to the float32 path.
// ---------------------------------------------------------------------------
constexpr int TCP_M = 128;  // rows of one MMA tile: TMEM lanes
constexpr int TCP_QCAP = 1024;  // queued tests the Gram value cannot decide
// Shared layout for lists of at most NC candidates (NC = 128 or 256):
// keys[NC] (sorted) | kraw[NC] (list order) | dom[NC][NC/32] |
// col[NC] (float4: norm, delta(p, c), rounding margin) | queue[1024] |
// mbarrier | tmem slot (and the queue count) | Cs (NC staged candidates,
// sorted order).  NC = 256 takes two MMA tiles: rows 0..127 against all 256
// columns (TMEM columns 0..255) and rows 128..255 against columns 128..255
// (TMEM columns 256..383), 512 columns allocated.
template <int NC>
struct Tcp {
  static constexpr int W = NC / 32;
  static constexpr int KRAW = 8 * NC;
  static constexpr int DOM = KRAW + 8 * NC;
  static constexpr int COL = DOM + 4 * NC * W;
  static constexpr int UQ = COL + 16 * NC;
  static constexpr int BAR = UQ + 4 * TCP_QCAP;
  static constexpr int SLOT = BAR + 8;
  static constexpr int CS = (SLOT + 8 + 127) & ~127;
  static constexpr uint32_t TMEM_COLS = NC == 128 ? 128u : 512u;
};
int harvest_prune_tc_smem(int nchunks, int nc) {
  return (nc == 128 ? Tcp<128>::CS : Tcp<256>::CS) + nc * tcp_nq(nchunks) * 16;
}

template <int METRIC, int G, int K, int NC>
__global__ void __launch_bounds__(NC) harvest_prune_tc_kernel(const HPruneArgs a) {
  using T = Tcp<NC>;
  constexpr int W = T::W;
  extern __shared__ __align__(128) unsigned char tsm_[];
  unsigned char* psm = tsm_;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int nch = a.nchunks, NQ = tcp_nq(nch);
  uint64_t* keys = reinterpret_cast<uint64_t*>(psm);
  uint32_t* dom = reinterpret_cast<uint32_t*>(psm + T::DOM);
  uint64_t* kraw = reinterpret_cast<uint64_t*>(psm + T::KRAW);
  float4* col = reinterpret_cast<float4*>(psm + T::COL);
  uint32_t* uq = reinterpret_cast<uint32_t*>(psm + T::UQ);
  uint32_t* qn = reinterpret_cast<uint32_t*>(psm + T::SLOT + 4);
  uint64_t* bar = reinterpret_cast<uint64_t*>(psm + T::BAR);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(psm + T::SLOT);
  uint4* Cs = reinterpret_cast<uint4*>(psm + T::CS);
  // rows no list fills stay zero
  for (int idx = tid; idx < NC * NQ; idx += NC) Cs[idx] = make_uint4(0u, 0u, 0u, 0u);
  if (warp == 0) {
    tmem_alloc(tslot, T::TMEM_COLS);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    *qn = 0u;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = idesc_tf32(TCP_M, NC);        // rows 0..127 x all NC columns
  const uint32_t idesc1 = idesc_tf32(TCP_M, TCP_M);    // NC = 256: rows 128..255 x 128..255
  const uint32_t cs0 = smem_u32(Cs);
  const uint32_t sbo = (uint32_t)NQ * 128u;
  uint32_t phase = 0;
  bool ok = true;
  unsigned long long ev = 0;
  const int64_t nq = a.nq_dev ? (int64_t)*a.nq_dev : a.nq;
  for (int64_t w = blockIdx.x; w < nq; w += gridDim.x) {
    const int64_t qidx = a.qlist ? (int64_t)a.qlist[w] : w;
    const int ne = a.Eg_cnt[qidx];
    if (ne < 0) continue;  // pruned by the re-run pass (uniform over the CTA)
    if (ne > NC) {         // longer than a tile: left to the next kernel
      if (tid == 0) a.long_list[atomicAdd(a.long_cnt, 1u)] = (int32_t)qidx;
      continue;
    }
    const int64_t p = a.rows ? (int64_t)a.rows[qidx] : a.q_first + qidx * a.q_step;
    const uint64_t* src = a.Eg_off ? a.Eg + a.Eg_off[p] : a.Eg + qidx * (int64_t)a.ecap;
    // keys: each thread ranks its own among the list (the point itself out)
    uint64_t kt = tid < ne ? src[tid] : PAD;
    if (kt != PAD && key_id(kt) == (int32_t)p) kt = PAD;
    kraw[tid] = kt;
    __syncthreads();
    if (kt != PAD) {
      int r = 0;
      for (int s2 = 0; s2 < ne; ++s2) r += kraw[s2] < kt ? 1 : 0;
      keys[r] = kt;
    }
    const int m = __syncthreads_count(kt != PAD);
    // stage the sorted candidates (element tails past d zeroed), one row per
    // thread with its chunks in flight together
    if (tid < m)
      tc_stage_row(Cs, tid, a.X + (int64_t)key_id(keys[tid]) * a.ld_bytes, NQ, nch, a.d);
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      for (int kk = 0; kk < NQ / 2; ++kk) {
        // a K = 8 step spans two core matrices along K (2 x 128 bytes)
        const uint64_t desc = smem_desc(cs0 + kk * 256, 128, sbo);
        mma_tf32(tmem, desc, desc, idesc, kk > 0 ? 1u : 0u);
      }
      if (NC == 256) {
        // rows 128..255 start 16 row groups (of 8 rows) into the staged tile
        for (int kk = 0; kk < NQ / 2; ++kk) {
          const uint64_t desc = smem_desc(cs0 + 16 * sbo + kk * 256, 128, sbo);
          mma_tf32(tmem + 256u, desc, desc, idesc1, kk > 0 ? 1u : 0u);
        }
      }
      mma_commit(bar);
    }
    if (tid < m) {
      const float dpt = key_dist(keys[tid]);
      col[tid] = make_float4(tc_norm2(Cs, tid, NQ, nch), dpt,
                             fabsf(dpt) * 4.76837158e-7f + 1e-30f, 0.0f);  // 2^-21 |dp|
    }
    // wait (bounded) for the Gram matrix; every thread takes the same decision
    bool done = false;
    for (int it = 0; it < a.wait_polls && !done; ++it) done = mbar_try_wait(bar, phase);
    done = __syncthreads_and(done);  // also publishes col
    if (!done) {
      ok = false;
      if (tid == 0) atomicOr(a.err, 1u);
      break;
    }
    phase ^= 1u;
    tc_fence_after();
    // dominance bits of row i = tid, one word per 32 columns.  With
    // x = alpha2 * approx - delta(p, c_j) and
    // B = alpha2 * eps + 2^-21 (alpha2 |approx| + |delta(p, c_j)|) + tiny,
    // x <= -B means the canonical test certainly holds, x > B that it
    // certainly fails (the margins cover the rounding of the test and of x).
    const int i = tid;
    const float ni = i < m ? col[i].x : 0.0f;
    float c1, c0;  // eps = c1 * n_j + c0 for this row
    if constexpr (METRIC == ANGULAR_F32) {
      c1 = 0.5f * a.tc_e1;
      c0 = 0.5f * a.tc_e1 * ni + a.tc_e0;
    } else {
      c1 = a.tc_e1;
      c0 = a.tc_e1 * ni + a.tc_e0;
    }
    const float a2 = a.alpha2, a2m = a.alpha2 * 4.76837158e-7f;
    for (int cb = 0; cb < W && 32 * cb < m; ++cb) {
      if (32 * cb + 31 <= 32 * warp) {  // every column of the block is at or left of i
        if (i < m) dom[i * W + cb] = 0u;
        continue;
      }
      // rows 0..127: lane i, column j; rows 128..255: lane i - 128, column
      // 256 + j - 128 (only blocks right of the diagonal get here)
      uint32_t v[32];
      const uint32_t tcol = warp < 4 ? (uint32_t)(32 * cb) : 256u + (uint32_t)(32 * cb - 128);
      tmem_ld32(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + tcol, v);
      if (i < m) {
        uint32_t word = 0, unsure = 0;
#pragma unroll
        for (int t = 0; t < 32; ++t) {
          const int jj = 32 * cb + t;
          if (jj <= i || jj >= m) continue;
          const float4 cj = col[jj];
          const float g = __uint_as_float(v[t]);
          float dt;
          if constexpr (METRIC == ANGULAR_F32)
            dt = 1.0f - g;
          else
            dt = (ni + cj.x) - 2.0f * g;
          const float eps = fmaf(c1, cj.x, c0);
          const float x = fmaf(a2, dt, -cj.y);
          const float B = fmaf(a2, eps, fmaf(a2m, fabsf(dt), cj.z));
          if (x <= -B)
            word |= 1u << t;
          else if (!(x > B))
            unsure |= 1u << t;
        }
        // the tests the Gram value cannot decide go to a CTA-wide queue (a
        // full queue leaves them to this thread)
        while (unsure) {
          const int t = __ffs(unsure) - 1;
          unsure &= unsure - 1u;
          const int jj = 32 * cb + t;
          const uint32_t slot = atomicAdd(qn, 1u);
          if (slot < TCP_QCAP) {
            uq[slot] = (uint32_t)(i << 8 | jj);
          } else {
            const float dd = canon_dist_thread<METRIC, G, K>(Cs, i, Cs, jj, NQ, nch, a.d);
            if (__fmul_rn(a.alpha2, dd) <= key_dist(keys[jj])) word |= 1u << t;
          }
        }
        dom[i * W + cb] = word;
      }
    }
    __syncthreads();
    // the queued tests in canonical float32, spread over the CTA
    {
      const int nu = min((int)*qn, TCP_QCAP);
      for (int e = tid; e < nu; e += NC) {
        const int ii = (int)(uq[e] >> 8), jj = (int)(uq[e] & 255u);
        const float dd = canon_dist_thread<METRIC, G, K>(Cs, ii, Cs, jj, NQ, nch, a.d);
        if (__fmul_rn(a.alpha2, dd) <= key_dist(keys[jj]))
          atomicOr(&dom[ii * W + (jj >> 5)], 1u << (jj & 31));
      }
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0) *qn = 0u;  // read by every thread before the barrier above
    if (tid == 0) {
      // the prune as a walk over the bit words, one thread: keep the first
      // alive candidate, remove the alive ones it dominates
      uint32_t al[W];
#pragma unroll
      for (int w = 0; w < W; ++w)
        al[w] = m >= 32 * w + 32 ? FULL : (m > 32 * w ? (1u << (m - 32 * w)) - 1u : 0u);
      int32_t* row = a.K_out ? nullptr : a.A_out + p * a.R;
      uint64_t* krow = a.K_out ? a.K_out + qidx * a.R : nullptr;
      int kept = 0;
      unsigned long long q_pe = 0;
      while (kept < a.R) {
        int cur = -1;
#pragma unroll
        for (int w = W - 1; w >= 0; --w)
          if (al[w]) cur = 32 * w + __ffs(al[w]) - 1;
        if (cur < 0) break;
#pragma unroll
        for (int w = 0; w < W; ++w)
          if (w == cur / 32) al[w] &= al[w] - 1u;  // the word without c*
        if (krow) {
          krow[kept] = keys[cur];
        } else {
          row[kept] = key_id(keys[cur]);
          if (a.D_out) a.D_out[p * a.R + kept] = key_dist(keys[cur]);
        }
        ++kept;
        if (kept == a.R) break;
        // the removal pass examines every alive candidate after c* (all alive
        // ones are after it: c* was the first)
        uint32_t alive = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) alive += (uint32_t)__popc(al[w]);
        q_pe += alive;
        const uint4* dm = reinterpret_cast<const uint4*>(dom + cur * W);
#pragma unroll
        for (int w4 = 0; w4 < W / 4; ++w4) {
          const uint4 d4 = dm[w4];
          al[4 * w4 + 0] &= ~d4.x;
          al[4 * w4 + 1] &= ~d4.y;
          al[4 * w4 + 2] &= ~d4.z;
          al[4 * w4 + 3] &= ~d4.w;
        }
      }
      if (krow) {
        a.cnt_out[qidx] = kept;
      } else {
        for (int r = kept; r < a.R; ++r) row[r] = -1;
        a.cnt_out[p] = kept;
      }
      ev += q_pe;
    }
    __syncthreads();
  }
  if (!ok) {
    // let the products in flight land before the tensor memory is released
    for (int it = 0; it < kDrainPolls; ++it)
      if (mbar_try_wait(bar, phase)) break;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, T::TMEM_COLS);
  if (tid == 0 && ev) atomicAdd(a.prune_ctr, ev);
}

HPruneFn hprune_tc_kernel_for(int metric, int G, int K, int nc) {
#define HX(M, GG, KK)                                                            \
  if (metric == M && G == GG && K == KK)                                         \
    return nc == 128 ? harvest_prune_tc_kernel<M, GG, KK, 128>                   \
                     : harvest_prune_tc_kernel<M, GG, KK, 256>;
#define HF(M) HX(M, 4, 1) HX(M, 8, 1) HX(M, 16, 1) HX(M, 32, 1) HX(M, 32, 2) HX(M, 32, 4) \
  HX(M, 32, 8)
  HF(0)
  HF(1)
#undef HF
#undef HX
  return nullptr;
}

}  // namespace fg
