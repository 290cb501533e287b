// Exact k nearest neighbours of points among all n points (self excluded),
// for local completeness (Section 2: the fraction of a point's true 10-NN
// that its adjacency row holds).  The answer is the canonical float32 top-k
// by (delta, id), the same key as the brute force of Section 2, computed as a
// filtered dense product on the 5th-generation tensor cores:
//
//  1. dt_prep_kernel rounds every row to BF16 as it is (no centring) and
//     writes the tensor cores' shared-memory image of 1024 consecutive ids
//     per block, with each row's norms and rounding residual; the maxima of
//     the per-block statistics bound the Gram error of every pair
//     (dt_row_eps, Cauchy-Schwarz on the actual residuals).
//  2. kn_fused_kernel (persistent, warp-specialised like the dense-block
//     filter: one bulk-copy producer lane, one tcgen05.mma issuer lane, eight
//     epilogue warps reading the two TMEM accumulators with tcgen05.ld) takes
//     tiles of 128 query rows against all columns in chunks of 256, twice:
//     pass 0 keeps each row's k smallest approximate distances (two sorted
//     register lists per row, one per column half), giving tau_k; pass 1
//     collects every column j != i whose approximate distance is at most
//     tau_k + 2 eps_i.  Every pair of the exact top-k is collected:
//     approx_j <= canonical_j + eps <= k-th canonical + eps <= tau_k + 2 eps.
//  3. kn_rerank_kernel evaluates the collected columns of each row in the
//     canonical float32 order and keeps the k smallest (delta, id); a row
//     that collected more columns than its list holds scans all n points.
#include <algorithm>

#include "common.cuh"
#include "dense_tc.cuh"
#include "internal.h"
#include "rowops.cuh"
#include "tc.cuh"

namespace fg {

namespace {

constexpr int KN_KQ = 32;          // register list length (k <= 32)
constexpr int KN_CAP = 256;        // collected columns kept per row
constexpr int64_t KN_GROUP = 65536;  // query rows per fused launch (a multiple of 128)
constexpr int KN_RR_WARPS = 4;

struct KnArgs {
  const unsigned char* Xt;  // image of nbk blocks of 1024 consecutive ids
  const float4* rowA;       // per id: {|x|^2, (1 - |x|^2)/2, scale, valid}
  const float4* rowB;       // per id: {|x - q|, |q|, |x|^2, 0}
  const float* colterm;     // per id (padded to whole blocks): column term, +inf past n
  const float* gm;          // {Mx, Rq, Qx, X2max, Cmax} over all ids
  int64_t n;
  int32_t nsl;
  int32_t dpad;
  int32_t d;
  int32_t metric;
  int32_t k;
  int64_t row0;   // query rows row0 .. row1 - 1 of this launch
  int64_t row1;
  int32_t* cand;  // [(row - row0)][KN_CAP]
  uint32_t* ccnt; // [(row - row0)]
  uint32_t* err;  // [0] timeout flag
  int32_t wait_polls;
};

struct KnSmem {
  static constexpr int lists = DT_STAGES * DT_STAGE_BYTES;       // [KN_KQ][256] f32
  static constexpr int rowcnt = lists + KN_KQ * DT_EPI * 4;       // [128] u32
  static constexpr int bars = rowcnt + DT_M * 4;                  // 16 x u64
  static constexpr int misc = bars + 16 * 8;
  static constexpr int bytes = misc + 16;
};

// The ids 0..n-1 in blocks of 1024 (-1 past n), as the image prep takes them.
__global__ void kn_ids_kernel(int64_t n, int64_t total, int32_t* ids) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x)
    ids[i] = i < n ? (int32_t)i : -1;
}

// Maxima of the per-block statistics, and each column's term of the
// approximate distance (angular: |x|^2 / 2 + (1 - |x|^2) / 2; squared L2:
// |x|^2), +inf for padding.
__global__ void kn_cols_kernel(const float4* rowA, const float* bst, int64_t nbk, int ang,
                               float* colterm, float* gm) {
  const int64_t total = nbk * DT_ROWS;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < total;
       j += (int64_t)gridDim.x * blockDim.x) {
    const float4 cj = rowA[j];
    const float ct = ang ? __fmaf_rn(0.5f, cj.x, cj.y) : cj.x;
    colterm[j] = cj.w != 0.0f ? ct : INFINITY;
    if (j < nbk * 5) {
      const int64_t b = j / 5, f = j % 5;
      atomicMax(reinterpret_cast<unsigned int*>(gm) + f, __float_as_uint(bst[b * 8 + f]));
    }
  }
}

// Sorted insertion of v into the ascending list tk (the largest drops out);
// worst becomes the k-th smallest.
__device__ __forceinline__ void kn_insert(float (&tk)[KN_KQ], float v, int k, float& worst) {
#pragma unroll
  for (int s = 0; s < KN_KQ; ++s) {
    const float lo = fminf(tk[s], v);
    v = fmaxf(tk[s], v);
    tk[s] = lo;
  }
  // the largest of the first k (a reduction, not an index: tk stays in registers)
  float w = -INFINITY;
#pragma unroll
  for (int s = 0; s < KN_KQ; ++s) w = fmaxf(w, s < k ? tk[s] : -INFINITY);
  worst = w;
}

__global__ void __launch_bounds__(DT_THREADS, 1) kn_fused_kernel(const KnArgs a) {
  extern __shared__ __align__(1024) unsigned char ksm[];
  unsigned char* stages = ksm;
  float* lists = reinterpret_cast<float*>(ksm + KnSmem::lists);
  uint32_t* rowcnt = reinterpret_cast<uint32_t*>(ksm + KnSmem::rowcnt);
  uint64_t* bars = reinterpret_cast<uint64_t*>(ksm + KnSmem::bars);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(ksm + KnSmem::misc);
  int* abort_flag = reinterpret_cast<int*>(ksm + KnSmem::misc + 4);
  int* zero_flag = reinterpret_cast<int*>(ksm + KnSmem::misc + 8);
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
  const int64_t t0 = a.row0 / DT_M, t1 = (a.row1 + DT_M - 1) / DT_M;
  const int64_t nch = (a.n + DT_NC - 1) / DT_NC;
  const int64_t blk_bytes = (int64_t)a.nsl * DT_SLICE_IMG;

  if (warp == 8) {
    // ---- producer: A slice of the query tile, B slice of the column chunk ----
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      for (int64_t tile = t0 + blockIdx.x; tile < t1 && ok; tile += gridDim.x) {
        const unsigned char* abase = a.Xt + (tile / 8) * blk_bytes + (tile % 8) * DT_A_BYTES;
        for (int pass = 0; pass < 2 && ok; ++pass)
          for (int64_t c = 0; c < nch && ok; ++c) {
            const unsigned char* bbase = a.Xt + (c / 4) * blk_bytes + (c % 4) * DT_B_BYTES;
            for (int sl = 0; sl < a.nsl; ++sl, ++it) {
              const uint32_t s = it % DT_STAGES, ph = (it / DT_STAGES) & 1u;
              if (!mbar_wait_backoff(empty + s, ph ^ 1u, a.wait_polls, abortp, 64)) {
                ok = false;
                break;
              }
              unsigned char* dst = stages + s * DT_STAGE_BYTES;
              mbar_arrive_expect_tx(full + s, DT_STAGE_BYTES);
              bulk_g2s(dst, abase + (int64_t)sl * DT_SLICE_IMG, DT_A_BYTES, full + s);
              bulk_g2s(dst + DT_A_BYTES, bbase + (int64_t)sl * DT_SLICE_IMG, DT_B_BYTES, full + s);
            }
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
    // ---- MMA issuer: 128 x 256 BF16 products into two TMEM accumulators ----
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(DT_M, DT_NC);
      uint32_t it = 0, ci = 0;
      bool ok = true;
      for (int64_t tile = t0 + blockIdx.x; tile < t1 && ok; tile += gridDim.x)
        for (int pass = 0; pass < 2 && ok; ++pass)
          for (int64_t c = 0; c < nch && ok; ++c, ++ci) {
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
                const uint64_t ad = smem_desc(a0 + kk * 256, 128, 1024);
                const uint64_t bd = smem_desc(b0 + kk * 256, 128, 1024);
                mma_bf16(dt, ad, bd, idesc, (sl > 0 || kk > 0) ? 1u : 0u);
              }
              mma_commit(empty + s);
            }
            if (ok) mma_commit(tfull + buf);
          }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(a.err, 1u);
      }
      mma_commit(done);
      mbar_wait_bounded(done, 0u, kDrainPolls, zero_flag);
    }
  } else {
    // ---- epilogue: warps 0..7, thread = (row il, column half h) ----
    const int etid = tid;
    const int q = warp & 3, h = warp >> 2;
    const int il = 32 * q + lane;
    const bool ang = a.metric == ANGULAR_F32;
    const float Mx = a.gm[0], Rq = a.gm[1], Qx = a.gm[2], X2m = a.gm[3];
    uint32_t ci = 0;
    bool aborted = false;
    for (int64_t tile = t0 + blockIdx.x; tile < t1; tile += gridDim.x) {
      const int64_t i = tile * DT_M + il;
      const bool vrow = i >= a.row0 && i < a.row1 && i < a.n;
      const float4 ra = a.rowA[i];
      const float4 rb = a.rowB[i];
      const float base = ang ? __fmaf_rn(0.5f, ra.x, ra.y) : ra.x;
      const float f = ang ? 1.0f : 2.0f;
      const float eps = dt_row_eps(ang, a.dpad, a.d, ra.x, rb.x, rb.y, rb.z, Mx, Rq, Qx, X2m);
      float tk[KN_KQ];
#pragma unroll
      for (int s = 0; s < KN_KQ; ++s) tk[s] = INFINITY;
      float worst = INFINITY, cut = -INFINITY;
      if (etid < DT_M) rowcnt[etid] = 0u;
      aborted = named_sync_or(1, DT_EPI, aborted || *abortp);
      if (aborted) break;
      for (int pass = 0; pass < 2 && !aborted; ++pass) {
        for (int64_t c = 0; c < nch; ++c, ++ci) {
          const uint32_t buf = ci & 1u, bph = (ci >> 1) & 1u;
          if (!aborted && !mbar_wait_bounded(tfull + buf, bph, a.wait_polls, abortp))
            aborted = true;
          // tcgen05.ld is warp-collective: the warp goes on only if every lane's wait ended
          aborted = __any_sync(FULL, aborted);
          if (!aborted) {
            tc_fence_after();
#pragma unroll 1
            for (int t4 = 0; t4 < 4; t4 += 2) {
              // two loads in flight per wait
              const int cb0 = h * 128 + 32 * t4;
              uint32_t vv[2][32];
              const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + buf * DT_NC + (uint32_t)cb0;
              tmem_ld32_async(ta, vv[0]);
              tmem_ld32_async(ta + 32, vv[1]);
              tmem_wait_ld();
              tmem_ld_fence(vv[0]);
              tmem_ld_fence(vv[1]);
              if (!vrow) continue;
#pragma unroll
              for (int hh = 0; hh < 2; ++hh) {
                const uint32_t (&v)[32] = vv[hh];
                const int64_t j0 = c * DT_NC + cb0 + 32 * hh;
                float ct[32];
                const float4* cp = reinterpret_cast<const float4*>(a.colterm + j0);
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                  const float4 w = __ldg(cp + e);
                  ct[4 * e] = w.x;
                  ct[4 * e + 1] = w.y;
                  ct[4 * e + 2] = w.z;
                  ct[4 * e + 3] = w.w;
                }
                // two values per packed instruction (each lane rounds as the
                // scalar fma(-f, g, base + ct) would), and only the minimum is
                // compared: a group with nothing under the limit costs no more
                float dts[32];
                float mn = INFINITY;
                const float lim = pass == 0 ? worst : cut;
#pragma unroll
                for (int t = 0; t < 32; t += 2) {
                  const float2 bc = __fadd2_rn(make_float2(base, base), make_float2(ct[t], ct[t + 1]));
                  const float2 d2 = __ffma2_rn(
                      make_float2(-f, -f),
                      make_float2(__uint_as_float(v[t]), __uint_as_float(v[t + 1])), bc);
                  dts[t] = d2.x;
                  dts[t + 1] = d2.y;
                  mn = fminf(mn, fminf(d2.x, d2.y));
                }
                if (!(pass == 0 ? mn < lim : mn <= lim)) continue;
                uint32_t take = 0;
#pragma unroll
                for (int t = 0; t < 32; ++t)
                  // padding columns carry +inf and are never taken, even under an infinite cut
                  take |= (pass == 0 ? dts[t] < lim : (dts[t] <= lim && dts[t] < INFINITY))
                              ? (1u << t) : 0u;
                if (i >= j0 && i < j0 + 32) take &= ~(1u << (int)(i - j0));  // not the point itself
                while (take) {
                  const int t = __ffs(take) - 1;
                  take &= take - 1u;
                  if (pass == 0) {
                    float dv = 0.0f;
#pragma unroll
                    for (int q2 = 0; q2 < 32; ++q2) dv = q2 == t ? dts[q2] : dv;
                    kn_insert(tk, dv, a.k, worst);
                  } else {
                    const uint32_t pos = atomicAdd(rowcnt + il, 1u);
                    if (pos < (uint32_t)KN_CAP)
                      a.cand[(i - a.row0) * KN_CAP + pos] = (int32_t)(j0 + t);
                  }
                }
              }
            }
          }
          tc_fence_before();
          mbar_arrive(tempty + buf);
        }
        if (pass == 0) {
          // tau_k: the k-th smallest of the two halves' lists of this row
#pragma unroll
          for (int s = 0; s < KN_KQ; ++s) lists[s * DT_EPI + etid] = tk[s];
          aborted = named_sync_or(1, DT_EPI, aborted || *abortp);
          if (aborted) break;
          const float* la = lists + etid;
          const float* lb = lists + (etid ^ 128);
          int ia = 0, ib = 0;
          float tau = INFINITY;
          for (int s = 0; s < a.k; ++s) {
            const float va = ia < KN_KQ ? la[ia * DT_EPI] : INFINITY;
            const float vb = ib < KN_KQ ? lb[ib * DT_EPI] : INFINITY;
            if (va <= vb) {
              tau = va;
              ++ia;
            } else {
              tau = vb;
              ++ib;
            }
          }
          // fewer than k other points: every column is collected
          cut = tau + 2.0f * eps;
          cut += fabsf(cut) * 2.4e-7f + 1e-30f;
          if (!(tau < INFINITY)) cut = INFINITY;
        }
      }
      aborted = named_sync_or(1, DT_EPI, aborted || *abortp);
      if (aborted) break;
      if (h == 0 && vrow) a.ccnt[i - a.row0] = rowcnt[il];
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

// One warp per query row: the canonical float32 distance of every collected
// column (of every point when the row collected more than KN_CAP), 32 at a
// time by lane groups, merged into a register pool of the k smallest
// (delta, id) keys.
template <int METRIC, int G, int K>
__global__ void __launch_bounds__(KN_RR_WARPS * 32)
    kn_rerank_kernel(const KnArgs a, const char* X, int64_t ld_bytes, int32_t* out_ids,
                     float* out_dist, unsigned long long* stat) {
  using L = Lanes<G, K>;
  extern __shared__ __align__(16) unsigned char rsm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane / L::P, j = lane % L::P;
  const int nch = (a.d * 4 + 15) / 16;
  uint4* qs = reinterpret_cast<uint4*>(rsm + warp * 16 * nch);
  unsigned long long nre = 0, nfull = 0;
  for (int64_t i = a.row0 + (int64_t)blockIdx.x * KN_RR_WARPS + warp; i < a.row1;
       i += (int64_t)gridDim.x * KN_RR_WARPS) {
    uint64_t pool[1] = {PAD};
    if (*reinterpret_cast<const volatile uint32_t*>(a.err) == 0u) {
      const uint32_t m0 = a.ccnt[i - a.row0];
      const bool scan = m0 > (uint32_t)KN_CAP;
      const int64_t total = scan ? a.n : (int64_t)m0;
      const int32_t* lst = a.cand + (i - a.row0) * KN_CAP;
      stage_row(qs, X + i * ld_bytes, nch, lane);
      uint4 qr[L::VL][K];
      load_slots_smem<G, K>(qs, nch, j, qr);
      nre += (unsigned long long)(total - (scan ? 1 : 0));
      nfull += scan ? 1ull : 0ull;
      for (int64_t base = 0; base < total; base += 32) {
        int32_t myid = -1;
        if (base + lane < total) {
          const int64_t c = base + lane;
          myid = scan ? (c != i ? (int32_t)c : -1) : lst[c];
          if (myid >= a.n) myid = -1;
        }
        uint64_t mykey = PAD;
        for (int sb = 0; sb < 32; sb += L::CPW * L::UW) {
          uint4 y[L::UW][L::VL][K];
#pragma unroll
          for (int uu = 0; uu < L::UW; ++uu) {
            const int idx = sb + uu * L::CPW + g;
            const int32_t cid = __shfl_sync(FULL, myid, idx);
            load_slots<G, K>(X + (int64_t)(cid >= 0 ? cid : i) * ld_bytes, nch, j, y[uu]);
          }
#pragma unroll
          for (int uu = 0; uu < L::UW; ++uu) {
            const float dd = regs_dist<METRIC, G, K>(qr, y[uu], nch, a.d, j, FULL);
            const int rel = lane - sb - uu * L::CPW;
            const float got = __shfl_sync(FULL, dd, (rel & (L::CPW - 1)) * L::P);
            if (rel >= 0 && rel < L::CPW && myid >= 0) mykey = make_key(got, myid);
          }
        }
        merge_into_pool<1>(pool, mykey, a.k, lane);
      }
    }
    if (lane < a.k) {
      out_ids[(i - a.row0) * a.k + lane] = pool[0] == PAD ? -1 : key_id(pool[0]);
      out_dist[(i - a.row0) * a.k + lane] =
          pool[0] == PAD ? __int_as_float(0x7f800000) : key_dist(pool[0]);
    }
  }
  if (lane == 0 && nre) atomicAdd(stat, nre);
  if (lane == 0 && nfull) atomicAdd(stat + 1, nfull);
}

using KnRerankFn = void (*)(const KnArgs, const char*, int64_t, int32_t*, float*,
                            unsigned long long*);

KnRerankFn kn_rerank_for(int metric, int G, int K) {
#define KX(M, GG, KK) \
  if (metric == M && G == GG && K == KK) return kn_rerank_kernel<M, GG, KK>;
#define KF(M) KX(M, 4, 1) KX(M, 8, 1) KX(M, 16, 1) KX(M, 32, 1) KX(M, 32, 2) KX(M, 32, 4) \
  KX(M, 32, 8)
  KF(0)
  KF(1)
#undef KF
#undef KX
  return nullptr;
}

}  // namespace

int knn_tc(const VecLayout& L, int64_t row0, int64_t nrows, int k, int32_t* out_ids,
           float* out_dist, double* stats, cudaStream_t s) {
  KnRerankFn rr = kn_rerank_for(L.metric, L.G, L.K);
  if (!rr || L.metric == L2_U8) {
    set_error(1, "exact k-NN takes float32 metrics");
    return 1;
  }
  const int64_t n = L.n;
  const int64_t nbk = (n + DT_ROWS - 1) / DT_ROWS;
  DtArgs t{};
  t.X = L.X;
  t.ld_bytes = L.ld_bytes;
  t.d = L.d;
  t.metric = L.metric;
  t.fp8 = 0;
  t.dpad = (L.d + DT_KB / 2 - 1) / (DT_KB / 2) * (DT_KB / 2);
  t.rowb = 2 * t.dpad;
  t.nsl = t.rowb / DT_KB;
  t.bs = DT_ROWS;
  t.nb = nbk;
  t.nocentre = 1;
  t.wait_polls = g_mma_wait_polls;
  {
    cudaError_t e = raise_smem_limit(reinterpret_cast<const void*>(kn_fused_kernel), KnSmem::bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(kn_fused_kernel)");
    const int nch16 = (L.d * 4 + 15) / 16;
    e = raise_smem_limit(reinterpret_cast<const void*>(rr), KN_RR_WARPS * 16 * nch16);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(kn_rerank_kernel)");
  }
  const int64_t group = std::min<int64_t>(KN_GROUP, ((nrows + DT_M - 1) / DT_M + 1) * DT_M);
  size_t total = 0;
  auto add = [&](size_t x) {
    const size_t o = total;
    total += (x + 255) / 256 * 256;
    return o;
  };
  const size_t o_xt = add((size_t)nbk * t.nsl * DT_SLICE_IMG);
  const size_t o_ra = add(sizeof(float4) * nbk * DT_ROWS);
  const size_t o_rb = add(sizeof(float4) * nbk * DT_ROWS);
  const size_t o_bst = add(sizeof(float) * nbk * 8);
  const size_t o_nv = add(sizeof(uint32_t) * nbk);
  const size_t o_ids = add(sizeof(int32_t) * nbk * DT_ROWS);
  const size_t o_col = add(sizeof(float) * nbk * DT_ROWS);
  const size_t o_cand = add(sizeof(int32_t) * group * KN_CAP);
  const size_t o_cnt = add(sizeof(uint32_t) * group);
  const size_t o_misc = add(512);  // gm (8 f32), err (16 u32), pairs, stats
  char* scratch = nullptr;
  FG_CUDA(cudaMallocAsync(&scratch, total, s));
  int rc = 0;
  cudaEvent_t ev[4] = {};
  for (int e = 0; e < 4 && stats; ++e) cudaEventCreate(&ev[e]);
  float t_fused = 0.0f, t_rr = 0.0f;
  unsigned long long hst[2] = {0, 0};
  do {
    t.Xt = reinterpret_cast<unsigned char*>(scratch + o_xt);
    t.rowA = reinterpret_cast<float4*>(scratch + o_ra);
    t.rowB = reinterpret_cast<float4*>(scratch + o_rb);
    t.bst = reinterpret_cast<float*>(scratch + o_bst);
    t.nvalid = reinterpret_cast<uint32_t*>(scratch + o_nv);
    int32_t* ids = reinterpret_cast<int32_t*>(scratch + o_ids);
    t.block_ids = ids;
    float* gm = reinterpret_cast<float*>(scratch + o_misc);
    uint32_t* err = reinterpret_cast<uint32_t*>(scratch + o_misc + 32);
    t.err = err;
    t.pairs = reinterpret_cast<unsigned long long*>(scratch + o_misc + 96);
    unsigned long long* st = reinterpret_cast<unsigned long long*>(scratch + o_misc + 128);
    cudaError_t e;
    if ((e = cudaMemsetAsync(t.bst, 0, sizeof(float) * nbk * 8, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(scratch + o_misc, 0, 512, s)) != cudaSuccess) {
      rc = cuda_fail(e, "cudaMemsetAsync(k-NN scratch)");
      break;
    }
    const int grid = (int)std::min<int64_t>((nbk * DT_ROWS + 255) / 256, (int64_t)device_sms() * 8);
    kn_ids_kernel<<<grid, 256, 0, s>>>(n, nbk * DT_ROWS, ids);
    note_launch();
    dt_prep_kernel<<<dim3((unsigned)nbk, DT_ROWS / 256), 256, 0, s>>>(t);
    note_launch();
    float* colterm = reinterpret_cast<float*>(scratch + o_col);
    kn_cols_kernel<<<grid, 256, 0, s>>>(t.rowA, t.bst, nbk, L.metric == ANGULAR_F32 ? 1 : 0,
                                        colterm, gm);
    note_launch();
    KnArgs a{};
    a.Xt = t.Xt;
    a.rowA = t.rowA;
    a.rowB = t.rowB;
    a.colterm = colterm;
    a.gm = gm;
    a.n = n;
    a.nsl = t.nsl;
    a.dpad = t.dpad;
    a.d = L.d;
    a.metric = L.metric;
    a.k = k;
    a.cand = reinterpret_cast<int32_t*>(scratch + o_cand);
    a.ccnt = reinterpret_cast<uint32_t*>(scratch + o_cnt);
    a.err = err;
    a.wait_polls = g_mma_wait_polls;
    const int nch16 = (L.d * 4 + 15) / 16;
    // query rows in groups aligned to the 128-row tiles
    int64_t g0 = row0 / DT_M * DT_M;
    for (; g0 < row0 + nrows && !rc; g0 += group) {
      a.row0 = std::max<int64_t>(g0, row0);
      a.row1 = std::min<int64_t>(g0 + group, row0 + nrows);
      const int64_t ntiles = (a.row1 + DT_M - 1) / DT_M - a.row0 / DT_M;
      if (stats) cudaEventRecord(ev[0], s);
      kn_fused_kernel<<<(int)std::min<int64_t>(ntiles, device_sms()), DT_THREADS, KnSmem::bytes,
                        s>>>(a);
      note_launch();
      if (stats) cudaEventRecord(ev[1], s);
      const int64_t rows = a.row1 - a.row0;
      const int rgrid = (int)std::max<int64_t>(
          1, std::min<int64_t>((rows + KN_RR_WARPS - 1) / KN_RR_WARPS, (int64_t)device_sms() * 16));
      rr<<<rgrid, KN_RR_WARPS * 32, KN_RR_WARPS * 16 * nch16, s>>>(
          a, L.X, L.ld_bytes, out_ids + (a.row0 - row0) * k, out_dist + (a.row0 - row0) * k, st);
      note_launch();
      if (stats) cudaEventRecord(ev[2], s);
      uint32_t herr = 0;
      if ((e = cudaGetLastError()) != cudaSuccess ||
          (e = cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
          (e = cudaStreamSynchronize(s)) != cudaSuccess) {
        rc = cuda_fail(e, "exact k-NN kernels");
        break;
      }
      if (herr) {
        set_error(5, "exact k-NN: a bounded wait for the tensor cores gave up");
        rc = 5;
        break;
      }
      if (stats) {
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, ev[0], ev[1]);
        t_fused += ms;
        cudaEventElapsedTime(&ms, ev[1], ev[2]);
        t_rr += ms;
      }
    }
    if (!rc && stats) {
      if ((e = cudaMemcpyAsync(hst, st, sizeof(hst), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
          (e = cudaStreamSynchronize(s)) != cudaSuccess)
        rc = cuda_fail(e, "k-NN statistics");
    }
  } while (false);
  if (stats && !rc) {
    stats[0] = (double)hst[0];  // canonical evaluations of the rerank
    stats[1] = (double)hst[1];  // rows that scanned every point
    stats[2] = t_fused;
    stats[3] = t_rr;
  }
  for (int e = 0; e < 4 && stats; ++e) cudaEventDestroy(ev[e]);
  cudaFreeAsync(scratch, s);
  return rc;
}

}  // namespace fg
