// Occlusion prune of the harvest (Section 3) as its own kernel.  One CTA per
// point of the block: warp 0 takes the expanded list the search wrote, drops
// the point itself and sorts it by (delta, id); the CTA stages all m
// candidate vectors in shared memory and computes, for every pair i < j, the
// dominance bit fl(alpha2 * delta(c_i, c_j)) <= delta(p, c_j) (canonical
// float32 distances, all pairs at once, no dependency between them); the
// prune itself -- keep the first alive c*, remove the alive candidates it
// dominates, stop at R -- is then a walk over bit words.  The evaluation
// count is the prune's own (the alive candidates each removal pass
// examines), not the number of pairs computed here.  The final graph's rows
// that need a prune take the same kernel (lists given by row, kept keys out).
#include <algorithm>
#include <cmath>

#include "beam.cuh"
#include "internal.h"
#include "tcdist.cuh"

namespace fg {

struct HPruneArgs {
  const char* X;
  int64_t ld_bytes;
  int32_t d;
  int32_t nchunks;
  const uint64_t* Eg;
  const int32_t* Eg_cnt;
  int32_t ecap;    // entries per point in Eg (power of two, >= 64)
  int32_t smem;    // shared bytes of a CTA
  int64_t nq;
  int64_t q_first;
  int64_t q_step;
  int32_t R;
  float alpha2;
  int32_t* A_out;
  int32_t* cnt_out;
  unsigned long long* prune_ctr;
  // the final graph's rows (all null for the harvest): point of list qidx,
  // start of its keys in Eg by point, list count on the device, and kept
  // keys out (R per list, count in cnt_out[qidx]) instead of rows of A_out
  const int32_t* rows;
  const int64_t* Eg_off;
  const uint32_t* nq_dev;
  uint64_t* K_out;
  // tensor-core variant: error bound coefficients and the timeout flag
  float tc_e1;
  float tc_e0;
  uint32_t* err;
  int32_t wait_polls;  // first bounded wait for the Gram matrix
  // lists longer than the tensor-core tile: the tensor-core kernel appends
  // their qidx to long_list (count in *long_cnt) for the lane-group kernel,
  // which then takes work item w as qidx = qlist[w], *nq_dev items
  int32_t* long_list;
  uint32_t* long_cnt;
  const int32_t* qlist;
};

constexpr int HP_WARPS = 4;
// tensor-core dominance bits on (1) or off (0, the lane-group kernel for all
// lists); results do not depend on it
int g_prune_tc = 1;

// shared layout: keys[ecap] | dom[ecap][ecap/32] | alive[ecap/32] + m | Cs[ecap][nchunks]
__host__ __device__ inline int hp_dom_off(int ecap) { return 8 * ecap; }
__host__ __device__ inline int hp_alive_off(int ecap) { return 8 * ecap + ecap * (ecap / 32) * 4; }
__host__ __device__ inline int hp_cs_off(int ecap) {
  return (hp_alive_off(ecap) + 4 * (ecap / 32) + 16 + 15) & ~15;
}

template <int METRIC, int G, int K>
__global__ void __launch_bounds__(HP_WARPS * 32) harvest_prune_kernel(const HPruneArgs a) {
  using L = Lanes<G, K>;
  extern __shared__ __align__(16) unsigned char psm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane / L::P, j = lane % L::P;
  const int nch = a.nchunks;
  const int W = a.ecap / 32;
  uint64_t* keys = reinterpret_cast<uint64_t*>(psm);
  uint32_t* dom = reinterpret_cast<uint32_t*>(psm + hp_dom_off(a.ecap));
  uint32_t* alive = reinterpret_cast<uint32_t*>(psm + hp_alive_off(a.ecap));
  int* mshared = reinterpret_cast<int*>(alive + W);
  uint4* Cs = reinterpret_cast<uint4*>(psm + hp_cs_off(a.ecap));
  unsigned long long ev = 0;
  constexpr int NG = HP_WARPS * L::CPW;  // lane groups of the CTA
  const int gid = warp * L::CPW + g;
  // lane groups of a warp run different column counts below: shuffles use the
  // group's own lanes
  const unsigned gmask = L::P == 32 ? FULL : (((1u << L::P) - 1u) << (g * L::P));
  const int64_t nq = a.nq_dev ? (int64_t)*a.nq_dev : a.nq;
  for (int64_t w = blockIdx.x; w < nq; w += gridDim.x) {
    const int64_t qidx = a.qlist ? (int64_t)a.qlist[w] : w;
    const int ne = a.Eg_cnt[qidx];
    if (ne < 0) continue;  // pruned by the re-run pass (uniform over the CTA)
    const int64_t p = a.rows ? (int64_t)a.rows[qidx] : a.q_first + qidx * a.q_step;
    if (warp == 0) {
      const uint64_t* src = a.Eg_off ? a.Eg + a.Eg_off[p] : a.Eg + qidx * (int64_t)a.ecap;
      int NE2 = 32;
      while (NE2 < ne) NE2 <<= 1;
      int m = 0;
      for (int i0 = 0; i0 < NE2; i0 += 32) {
        const int i = i0 + lane;
        uint64_t kk = i < ne ? src[i] : PAD;
        if (kk != PAD && key_id(kk) == (int32_t)p) kk = PAD;
        keys[i] = kk;
        m += __popc(__ballot_sync(FULL, kk != PAD));
      }
      __syncwarp();
      warp_sort_mem(keys, NE2, lane);
      if (lane == 0) *mshared = m;
    }
    __syncthreads();
    const int m = *mshared;
    for (int idx = threadIdx.x; idx < m * nch; idx += HP_WARPS * 32) {
      const int c = idx / nch, ch = idx - c * nch;
      Cs[idx] = __ldg(reinterpret_cast<const uint4*>(a.X + (int64_t)key_id(keys[c]) * a.ld_bytes) + ch);
    }
    for (int idx = threadIdx.x; idx < m * W; idx += HP_WARPS * 32) dom[idx] = 0u;
    __syncthreads();
    // dominance bits: the m(m-1)/2 pairs i < j in row-major order are cut
    // into NG equal chunks, one per lane group; bit j of row i of dom is set
    // when c_i removes c_j.  Words shared by two chunks are merged with
    // atomicOr.
    {
      const int npairs = m * (m - 1) / 2;
      const int chunk = (npairs + NG - 1) / NG;
      int t = gid * chunk;
      const int tend = min(npairs, t + chunk);
      // locate the first pair (i, jj) of the chunk
      int i = 0, rowlen = m - 1;
      while (i < m - 1 && t >= rowlen) {
        t -= rowlen;
        ++i;
        rowlen = m - 1 - i;
      }
      int jj = i + 1 + t;
      uint4 xq[L::VL][K];
      if (gid * chunk < tend) load_slots_smem<G, K>(Cs + (int64_t)i * nch, nch, j, xq);
      uint32_t word = 0;
      int wrow = i, wcur = jj / 32;
      for (int pidx = gid * chunk; pidx < tend; ++pidx) {
        uint4 y[L::VL][K];
        load_slots_smem<G, K>(Cs + (int64_t)jj * nch, nch, j, y);
        const float dd = regs_dist<METRIC, G, K>(xq, y, nch, a.d, j, gmask);
        const bool kill = __fmul_rn(a.alpha2, dd) <= key_dist(keys[jj]);
        word |= (kill ? 1u : 0u) << (jj % 32);
        // advance to the next pair; flush the word when it is complete
        int ni = i, nj = jj + 1;
        if (nj == m) {
          ni = i + 1;
          nj = ni + 1;
        }
        if (pidx + 1 == tend || ni != wrow || nj / 32 != wcur) {
          if (j == 0 && word) atomicOr(&dom[wrow * W + wcur], word);
          word = 0;
          wrow = ni;
          wcur = nj / 32;
        }
        if (ni != i && pidx + 1 < tend) load_slots_smem<G, K>(Cs + (int64_t)ni * nch, nch, j, xq);
        i = ni;
        jj = nj;
      }
    }
    __syncthreads();
    if (warp == 0) {
      // the prune as a walk over bit words; lane w holds alive word w
      uint32_t al = lane < W ? (lane * 32 + 32 <= m ? FULL
                                                    : (lane * 32 < m ? ((1u << (m - lane * 32)) - 1u) : 0u))
                             : 0u;
      int32_t* row = a.K_out ? nullptr : a.A_out + p * a.R;
      uint64_t* krow = a.K_out ? a.K_out + qidx * a.R : nullptr;
      int kept = 0;
      unsigned long long q_pe = 0;
      while (kept < a.R) {
        const unsigned nz = __ballot_sync(FULL, al != 0u);
        if (nz == 0u) break;
        const int w0 = __ffs(nz) - 1;
        const uint32_t bw = __shfl_sync(FULL, al, w0);
        const int cur = w0 * 32 + __ffs(bw) - 1;
        if (lane == 0) {
          if (krow)
            krow[kept] = keys[cur];
          else
            row[kept] = key_id(keys[cur]);
        }
        ++kept;
        if (lane == w0) al &= ~(1u << (cur % 32));
        if (kept == a.R) break;
        // the removal pass examines every alive candidate after c* (all alive
        // ones are after it: c* was the first)
        q_pe += (unsigned long long)__reduce_add_sync(FULL, __popc(al));
        if (lane < W) al &= ~dom[cur * W + lane];
      }
      if (krow) {
        if (lane == 0) a.cnt_out[qidx] = kept;
      } else {
        for (int r = kept + lane; r < a.R; r += 32) row[r] = -1;
        if (lane == 0) a.cnt_out[p] = kept;
      }
      ev += q_pe;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && ev) atomicAdd(a.prune_ctr, ev);
}


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
constexpr int TCP_M = 128;  // candidates of one tile: TMEM lanes and columns
constexpr int TCP_W = TCP_M / 32;
// shared layout: keys[128] (sorted) | kraw[128] (list order) | dom[128][4] |
// col[128] (float4: norm, delta(p, c), rounding margin) | queue[1024] |
// mbarrier | tmem slot (and the queue count) |
// Cs (128 staged candidates, sorted order)
constexpr int TCP_KRAW = 8 * TCP_M;
constexpr int TCP_DOM = TCP_KRAW + 8 * TCP_M;
constexpr int TCP_COL = TCP_DOM + 4 * TCP_M * TCP_W;
constexpr int TCP_QCAP = 1024;  // queued tests the Gram value cannot decide
constexpr int TCP_UQ = TCP_COL + 16 * TCP_M;
constexpr int TCP_BAR = TCP_UQ + 4 * TCP_QCAP;
constexpr int TCP_SLOT = TCP_BAR + 8;
constexpr int TCP_CS = (TCP_SLOT + 8 + 127) & ~127;
int harvest_prune_tc_smem(int nchunks) { return TCP_CS + TCP_M * tcp_nq(nchunks) * 16; }

template <int METRIC, int G, int K>
__global__ void __launch_bounds__(TCP_M) harvest_prune_tc_kernel(const HPruneArgs a) {
  extern __shared__ __align__(128) unsigned char psm[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nch = a.nchunks, NQ = tcp_nq(nch);
  uint64_t* keys = reinterpret_cast<uint64_t*>(psm);
  uint32_t* dom = reinterpret_cast<uint32_t*>(psm + TCP_DOM);
  uint64_t* kraw = reinterpret_cast<uint64_t*>(psm + TCP_KRAW);
  float4* col = reinterpret_cast<float4*>(psm + TCP_COL);
  uint32_t* uq = reinterpret_cast<uint32_t*>(psm + TCP_UQ);
  uint32_t* qn = reinterpret_cast<uint32_t*>(psm + TCP_SLOT + 4);
  uint64_t* bar = reinterpret_cast<uint64_t*>(psm + TCP_BAR);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(psm + TCP_SLOT);
  uint4* Cs = reinterpret_cast<uint4*>(psm + TCP_CS);
  // rows no list fills stay zero
  for (int idx = tid; idx < TCP_M * NQ; idx += TCP_M) Cs[idx] = make_uint4(0u, 0u, 0u, 0u);
  if (warp == 0) {
    tmem_alloc(tslot, TCP_M);
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
  const uint32_t idesc = idesc_tf32(TCP_M, TCP_M);
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
    if (ne > TCP_M) {      // longer than a tile: left to the lane-group kernel
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
    for (int cb = 0; cb < TCP_W && 32 * cb < m; ++cb) {
      if (32 * cb + 31 <= 32 * warp) {  // every column of the block is at or left of i
        if (i < m) dom[i * TCP_W + cb] = 0u;
        continue;
      }
      uint32_t v[32];
      tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(32 * cb), v);
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
        dom[i * TCP_W + cb] = word;
      }
    }
    __syncthreads();
    // the queued tests in canonical float32, spread over the CTA
    {
      const int nu = min((int)*qn, TCP_QCAP);
      for (int e = tid; e < nu; e += TCP_M) {
        const int ii = (int)(uq[e] >> 8), jj = (int)(uq[e] & 255u);
        const float dd = canon_dist_thread<METRIC, G, K>(Cs, ii, Cs, jj, NQ, nch, a.d);
        if (__fmul_rn(a.alpha2, dd) <= key_dist(keys[jj]))
          atomicOr(&dom[ii * TCP_W + (jj >> 5)], 1u << (jj & 31));
      }
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0) *qn = 0u;  // read by every thread before the barrier above
    if (tid == 0) {
      // the prune as a walk over the four bit words, one thread: keep the
      // first alive candidate, remove the alive ones it dominates
      uint32_t al0 = m >= 32 ? FULL : (m > 0 ? (1u << m) - 1u : 0u);
      uint32_t al1 = m >= 64 ? FULL : (m > 32 ? (1u << (m - 32)) - 1u : 0u);
      uint32_t al2 = m >= 96 ? FULL : (m > 64 ? (1u << (m - 64)) - 1u : 0u);
      uint32_t al3 = m >= 128 ? FULL : (m > 96 ? (1u << (m - 96)) - 1u : 0u);
      int32_t* row = a.K_out ? nullptr : a.A_out + p * a.R;
      uint64_t* krow = a.K_out ? a.K_out + qidx * a.R : nullptr;
      int kept = 0;
      unsigned long long q_pe = 0;
      while (kept < a.R) {
        const uint32_t nz = (al0 ? 1u : 0u) | (al1 ? 2u : 0u) | (al2 ? 4u : 0u) | (al3 ? 8u : 0u);
        if (nz == 0u) break;
        const int w = __ffs(nz) - 1;
        const uint32_t aw = w == 0 ? al0 : (w == 1 ? al1 : (w == 2 ? al2 : al3));
        const int cur = 32 * w + __ffs(aw) - 1;
        const uint32_t cl = aw & (aw - 1u);  // the word without c*
        al0 = w == 0 ? cl : al0;
        al1 = w == 1 ? cl : al1;
        al2 = w == 2 ? cl : al2;
        al3 = w == 3 ? cl : al3;
        if (krow)
          krow[kept] = keys[cur];
        else
          row[kept] = key_id(keys[cur]);
        ++kept;
        if (kept == a.R) break;
        // the removal pass examines every alive candidate after c* (all alive
        // ones are after it: c* was the first)
        q_pe += (unsigned long long)(__popc(al0) + __popc(al1) + __popc(al2) + __popc(al3));
        const uint4 dm = *reinterpret_cast<const uint4*>(dom + cur * TCP_W);
        al0 &= ~dm.x;
        al1 &= ~dm.y;
        al2 &= ~dm.z;
        al3 &= ~dm.w;
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
  if (warp == 0) tmem_dealloc(tmem, TCP_M);
  if (tid == 0 && ev) atomicAdd(a.prune_ctr, ev);
}

using HPruneFn = void (*)(const HPruneArgs);

static HPruneFn hprune_tc_kernel_for(int metric, int G, int K) {
#define HX(M, GG, KK) \
  if (metric == M && G == GG && K == KK) return harvest_prune_tc_kernel<M, GG, KK>;
#define HF(M) HX(M, 4, 1) HX(M, 8, 1) HX(M, 16, 1) HX(M, 32, 1) HX(M, 32, 2) HX(M, 32, 4) \
  HX(M, 32, 8)
  HF(0)
  HF(1)
#undef HF
#undef HX
  return nullptr;
}

static HPruneFn hprune_kernel_for(int metric, int G, int K) {
#define HX(M, GG, KK) \
  if (metric == M && G == GG && K == KK) return harvest_prune_kernel<M, GG, KK>;
#define HF(M) HX(M, 4, 1) HX(M, 8, 1) HX(M, 16, 1) HX(M, 32, 1) HX(M, 32, 2) HX(M, 32, 4) \
  HX(M, 32, 8)
  HF(0)
  HF(1)
  HX(2, 4, 1) HX(2, 8, 1) HX(2, 16, 1)
#undef HF
#undef HX
  return nullptr;
}

// Shared bytes of a prune CTA for lists of up to ecap candidates.
int harvest_prune_smem(int ecap, int nchunks) { return hp_cs_off(ecap) + 16 * nchunks * ecap; }

int harvest_prune(const VecLayout& L, const uint64_t* Eg, const int32_t* Eg_cnt, int ecap,
                  int64_t nq, int64_t q_first, int64_t q_step, int R, float alpha2,
                  int32_t* A_out, int32_t* cnt_out, unsigned long long* prune_ctr, int num_sms,
                  cudaStream_t s, const int32_t* rows, const int64_t* Eg_off,
                  const uint32_t* nq_dev, uint64_t* K_out, uint32_t* err, int32_t* long_list,
                  uint32_t* long_cnt, const int32_t* qlist) {
  HPruneFn kern = hprune_kernel_for(L.metric, L.G, L.K);
  if (!kern) {
    set_error(1, "no prune kernel for this metric and dimension");
    return 1;
  }
  HPruneArgs a{L.X, L.ld_bytes, L.d, L.nchunks, Eg, Eg_cnt, ecap,
               harvest_prune_smem(ecap, L.nchunks), nq, q_first, q_step, R, alpha2,
               A_out, cnt_out, prune_ctr, rows, Eg_off, nq_dev, K_out, 0.0f, 0.0f, err,
               g_mma_wait_polls, nullptr, nullptr, qlist};
  HPruneFn tck = hprune_tc_kernel_for(L.metric, L.G, L.K);
  int optin = 0, dev = 0, sm_bytes = 0;
  FG_CUDA(cudaGetDevice(&dev));
  FG_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  FG_CUDA(cudaDeviceGetAttribute(&sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  // lists of at most 128 entries on the tensor cores; longer ones (possible
  // when the list buffer is larger) go to the lane-group kernel afterwards
  const bool split = ecap > TCP_M && long_list && long_cnt;
  if (tck && err && g_prune_tc && (ecap <= TCP_M || split) &&
      harvest_prune_tc_smem(L.nchunks) <= optin) {
    HPruneArgs t = a;
    tc_error_bound(L.metric, L.nchunks, &t.tc_e1, &t.tc_e0);
    // at most 512 / 128 CTAs on an SM (its tensor memory columns): the
    // shared memory request is raised so that no more can be resident
    const int tc_ctas = 512 / TCP_M;
    t.smem = std::max(harvest_prune_tc_smem(L.nchunks), sm_bytes / (tc_ctas + 1));
    const int per_sm = std::min(tc_ctas, sm_bytes / (t.smem + 1024));
    if (per_sm < 1) {
      set_error(1, "prune launch does not fit an SM");
      return 1;
    }
    if (split) {
      t.long_list = long_list;
      t.long_cnt = long_cnt;
      FG_CUDA(cudaMemsetAsync(long_cnt, 0, sizeof(uint32_t), s));
    }
    FG_CUDA(raise_smem_limit(reinterpret_cast<const void*>(tck), t.smem));
    tck<<<per_sm * num_sms, TCP_M, t.smem, s>>>(t);
    note_launch();
    FG_CUDA(cudaGetLastError());
    if (!split) return 0;
    a.qlist = long_list;
    a.nq_dev = long_cnt;
  }
  FG_CUDA(raise_smem_limit(reinterpret_cast<const void*>(kern), a.smem));
  int per_sm = 0;
  FG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, HP_WARPS * 32, a.smem));
  if (per_sm < 1) {
    set_error(1, "prune launch does not fit an SM");
    return 1;
  }
  kern<<<per_sm * num_sms, HP_WARPS * 32, a.smem, s>>>(a);
  note_launch();
  FG_CUDA(cudaGetLastError());
  return 0;
}

}  // namespace fg
