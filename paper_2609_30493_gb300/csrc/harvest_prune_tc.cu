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
// Tensor-core variant for the float32 metrics and lists of at most 128 or
// 256 candidates.
//
// The candidates are staged once, as float32, in the canonical K-major
// operand layout of tcgen05 (core matrices of 8 rows x 16 bytes); their Gram
// matrix C C^T is one chain of kind::tf32 MMAs (M = N = 128, 128 TMEM
// columns), which reads the same float32 words with the low mantissa bits
// ignored.  Thread i then reads row i of the Gram matrix from TMEM (or, for
// a block taken by columns, thread j row j) and decides each bit "c_i
// dominates c_j", j > i, from the approximate distance when the decision is
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
// keys[S][NC] (sorted; S slots) | kraw[NC] (list order) |
// dom[S][NC][NC/32] | col[NC] (float4: norm, delta(p, c), rounding margin) |
// queue[1024] | mbarriers (MMA, full[S], empty[S]) | slot rows (point, list
// index, m) | tmem slot (and the queue count) | Cs (NC
// staged candidates, sorted order).  NC = 256 takes two MMA tiles: rows
// 0..127 against all 256 columns (TMEM columns 0..255) and rows 128..255
// against columns 128..255 (TMEM columns 256..383), 512 columns allocated.
//
// The NC compute threads fill a slot (sorted keys and dominance words) per
// list, list j in slot j mod S, and hand it to one of TCP_WALKERS more warps
// (walker j mod TCP_WALKERS), which turns the bit words into the pruned list
// while the compute threads go on with the next lists.  full[s] and empty[s]
// (one arrival each) pass slot s back and forth; every wait on them is
// bounded.
struct TcpSlotRow {
  int64_t p, qidx;
  int32_t m, pad;
};
template <int NC>
struct Tcp {
  static constexpr int W = NC / 32;
  static constexpr int S = 2 * TCP_WALKERS;
  static constexpr int KEYS = 0;
  static constexpr int KRAW = KEYS + 8 * NC * S;
  static constexpr int DOM = KRAW + 8 * NC;
  static constexpr int COL = DOM + 4 * NC * W * S;
  static constexpr int UQ = COL + 16 * NC;
  static constexpr int BAR = UQ + 4 * TCP_QCAP;  // MMA, full[S], empty[S]
  static constexpr int ROWS = BAR + 8 * (1 + 2 * S);
  static constexpr int SLOT = ROWS + S * (int)sizeof(TcpSlotRow);
  static constexpr int CS = (SLOT + 8 + 127) & ~127;
  static constexpr uint32_t TMEM_COLS = NC == 128 ? 128u : 512u;
};
int harvest_prune_tc_smem(int nchunks, int nc) {
  return (nc == 128 ? Tcp<128>::CS : Tcp<256>::CS) + nc * tcp_nq(nchunks) * 16;
}

template <int METRIC, int G, int K, int NC>
__global__ void __launch_bounds__(NC + 32 * TCP_WALKERS, NC == 128 ? 3 : 1)
    harvest_prune_tc_kernel(const HPruneArgs a) {
  using T = Tcp<NC>;
  constexpr int W = T::W, S = T::S;
  extern __shared__ __align__(128) unsigned char tsm_[];
  unsigned char* psm = tsm_;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nch = a.nchunks, NQ = tcp_nq(nch);
  uint64_t* keys2 = reinterpret_cast<uint64_t*>(psm + T::KEYS);
  uint32_t* dom2 = reinterpret_cast<uint32_t*>(psm + T::DOM);
  uint64_t* kraw = reinterpret_cast<uint64_t*>(psm + T::KRAW);
  float4* col = reinterpret_cast<float4*>(psm + T::COL);
  uint32_t* uq = reinterpret_cast<uint32_t*>(psm + T::UQ);
  uint32_t* qn = reinterpret_cast<uint32_t*>(psm + T::SLOT + 4);
  uint64_t* bar = reinterpret_cast<uint64_t*>(psm + T::BAR);
  uint64_t* full = bar + 1;
  uint64_t* empty = bar + 1 + S;
  TcpSlotRow* srow = reinterpret_cast<TcpSlotRow*>(psm + T::ROWS);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(psm + T::SLOT);
  uint4* Cs = reinterpret_cast<uint4*>(psm + T::CS);
  // rows no list fills stay zero
  if (tid < NC)
    for (int idx = tid; idx < NC * NQ; idx += NC) Cs[idx] = make_uint4(0u, 0u, 0u, 0u);
  if (warp == 0) {
    tmem_alloc(tslot, T::TMEM_COLS);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int b = 0; b < 1 + 2 * S; ++b) mbar_init(bar + b, 1);
    fence_mbar_init();
    *qn = 0u;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  bool ok = true;
  uint32_t phase = 0;
  unsigned long long ev = 0;
  if (tid >= NC) {
    // walker k: lists k, k + TCP_WALKERS, ..., the prune as a walk over the
    // bit words.
    // Lane l < W holds alive word l with every removal pass so far applied;
    // the word being walked is held by every lane.  Keep the first alive
    // candidate c*; its removal pass examines every alive candidate after it
    // (the rest of its word and the later words) and drops those it
    // dominates.
    for (int jw = (tid - NC) >> 5;; jw += TCP_WALKERS) {
      const int s = jw % S;
      bool got = false;
      for (int it = 0; it < a.wait_polls && !got; ++it)
        got = mbar_try_wait(full + s, (uint32_t)(jw / S) & 1u);
      if (!got) {
        if (lane == 0) atomicOr(a.err, 1u);
        break;
      }
      const int m = srow[s].m;
      if (m < 0) break;  // no more lists
      const int64_t p = srow[s].p, qidx = srow[s].qidx;
      const uint64_t* keys = keys2 + s * NC;
      const uint32_t* dom = dom2 + s * NC * W;
      uint32_t al = lane < W ? (m >= 32 * lane + 32 ? FULL
                                                    : (m > 32 * lane ? (1u << (m - 32 * lane)) - 1u
                                                                     : 0u))
                             : 0u;
      uint32_t kmine = 0;  // lane l < W: the kept bits of word l
      int kept = 0;
      uint32_t q = 0;
      for (int w = 0; w < W && kept < a.R; ++w) {
        uint32_t alw = __shfl_sync(FULL, al, w), km = 0;
        while (alw != 0u) {
          const uint32_t low = alw & (0u - alw);
          const int cur = 32 * w + __ffs(alw) - 1;
          km |= low;
          alw ^= low;
          if (++kept == a.R) break;
          const uint32_t dw = dom[cur * W + w];
          const uint32_t dl = lane < W ? dom[cur * W + lane] : 0u;
          q += (lane == 0 ? (uint32_t)__popc(alw) : 0u) + (lane > w ? (uint32_t)__popc(al) : 0u);
          alw &= ~dw;
          if (lane > w) al &= ~dl;
        }
        if (lane == w) kmine = km;
      }
      // the kept candidates, in order, at their ranks
      int32_t* row = a.K_out ? nullptr : a.A_out + p * a.R;
      uint64_t* krow = a.K_out ? a.K_out + qidx * a.R : nullptr;
      int base = 0;
      for (int l = 0; l < W; ++l) {
        const uint32_t kml = __shfl_sync(FULL, kmine, l);
        if (kml >> lane & 1u) {
          const int r = base + __popc(kml & ((1u << lane) - 1u));
          const uint64_t kc = keys[32 * l + lane];
          if (krow) {
            krow[r] = kc;
          } else {
            row[r] = key_id(kc);
            if (a.D_out) a.D_out[p * a.R + r] = key_dist(kc);
          }
        }
        base += __popc(kml);
      }
      if (krow) {
        if (lane == 0) a.cnt_out[qidx] = kept;
      } else {
        for (int r = kept + lane; r < a.R; r += 32) row[r] = -1;
        if (lane == 0) a.cnt_out[p] = kept;
      }
      const uint32_t qs = __reduce_add_sync(FULL, q);
      if (lane == 0) ev += qs;
      __syncwarp();
      if (lane == 0) mbar_arrive(empty + s);  // the slot's keys and words are read
    }
  } else {
    const uint32_t idesc = idesc_tf32(TCP_M, NC);      // rows 0..127 x all NC columns
    const uint32_t idesc1 = idesc_tf32(TCP_M, TCP_M);  // NC = 256: rows 128..255 x 128..255
    const uint32_t cs0 = smem_u32(Cs);
    const uint32_t sbo = (uint32_t)NQ * 128u;
    int jr = 0;  // lists handed to the walker
    const int64_t nq = a.nq_dev ? (int64_t)*a.nq_dev : a.nq;
    for (int64_t w = blockIdx.x; w < nq; w += gridDim.x) {
      const int64_t qidx = a.qlist ? (int64_t)a.qlist[w] : w;
      const int ne = a.Eg_cnt[qidx];
      if (ne < 0) continue;  // pruned by the re-run pass (uniform over the compute threads)
      if (ne > NC) {         // longer than a tile: left to the next kernel
        if (tid == 0) a.long_list[atomicAdd(a.long_cnt, 1u)] = (int32_t)qidx;
        continue;
      }
      const int64_t p = a.rows ? (int64_t)a.rows[qidx] : a.q_first + qidx * a.q_step;
      const uint64_t* src = a.Eg_off ? a.Eg + a.Eg_off[p] : a.Eg + qidx * (int64_t)a.ecap;
      const int s = jr % S;
      uint64_t* keys = keys2 + s * NC;
      uint32_t* dom = dom2 + s * NC * W;
      // keys: each thread ranks its own among the list (the point itself out)
      uint64_t kt = tid < ne ? src[tid] : PAD;
      if (kt != PAD && key_id(kt) == (int32_t)p) kt = PAD;
      kraw[tid] = kt;
      // the walker is done with this slot's previous list (bounded wait; the
      // same decision on every thread)
      bool freed = jr < S;
      for (int it = 0; it < a.wait_polls && !freed; ++it)
        freed = mbar_try_wait(empty + s, (uint32_t)(jr / S - 1) & 1u);
      freed = named_sync_and(1, NC, freed);  // also publishes kraw
      if (!freed) {
        ok = false;
        if (tid == 0) atomicOr(a.err, 1u);
        break;
      }
      if (kt != PAD) {
        int r = 0;
        for (int s2 = 0; s2 < ne; ++s2) r += kraw[s2] < kt ? 1 : 0;
        keys[r] = kt;
      }
      const int m = named_sync_count(1, NC, kt != PAD);
      // stage the sorted candidates (element tails past d zeroed), one row per
      // thread with its chunks in flight together
      if (tid < m)
        tc_stage_row(Cs, tid, a.X + (int64_t)key_id(keys[tid]) * a.ld_bytes, NQ, nch, a.d);
      fence_proxy_async();
      named_sync(1, NC);
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
      done = named_sync_and(1, NC, done);  // also publishes col
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
      const float a2 = a.alpha2, a2m = a.alpha2 * 4.76837158e-7f;
      // A warp reads the TMEM lanes of its quarter, 32 (warp & 3) ..; the
      // blocks (row block rb, column block cb >= rb) are spread over the
      // warps so that none takes more than 3 (NC = 128) or 6 (NC = 256).
      //
      // Row job: thread i = 32 rb + lane reads row i of the Gram matrix and
      // builds its word of block cb.
      auto row_job = [&](int rb, int cb) {
        if (32 * rb >= m || 32 * cb >= m) return;  // uniform over the warp
        const int i = 32 * rb + lane;
        const float ni = i < m ? col[i].x : 0.0f;
        float c1, c0;  // eps = c1 * n_j + c0 for this row
        if constexpr (METRIC == ANGULAR_F32) {
          c1 = 0.5f * a.tc_e1;
          c0 = 0.5f * a.tc_e1 * ni + a.tc_e0;
        } else {
          c1 = a.tc_e1;
          c0 = a.tc_e1 * ni + a.tc_e0;
        }
        // rows 0..127: lane i, column j; rows 128..255: lane i - 128, column
        // 256 + j - 128 (only blocks right of the diagonal get here)
        uint32_t v[32];
        const uint32_t tcol = rb < 4 ? (uint32_t)(32 * cb) : 256u + (uint32_t)(32 * cb - 128);
        tmem_ld32(tmem + ((uint32_t)(32 * (rb & 3)) << 16) + tcol, v);
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
      };
      // Column job (rb < cb, rows 0..127 only): thread j = 32 cb + lane reads
      // row j of the Gram matrix, whose columns 32 rb .. are the block's
      // entries transposed, tests every row i of block rb against column j,
      // and 32 ballots turn the columns' bits into the rows' words.  The
      // Gram value's error bound holds in either orientation, and an
      // undecided test is the canonical one (symmetric in its two rows), so
      // the bits are those of the row job.
      auto col_job = [&](int rb, int cb) {
        if (32 * rb >= m || 32 * cb >= m) return;  // uniform over the warp
        const int j = 32 * cb + lane;
        const float4 cj = j < m ? col[j] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        uint32_t v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * (cb & 3)) << 16) + (uint32_t)(32 * rb), v);
        uint32_t bits = 0;
        if (j < m) {
          uint32_t unsure = 0;
#pragma unroll
          for (int t = 0; t < 32; ++t) {
            const int ii = 32 * rb + t;
            if (ii >= m) continue;
            const float ni = col[ii].x;
            float c1, c0;  // eps = c1 * n_j + c0 for row ii
            if constexpr (METRIC == ANGULAR_F32) {
              c1 = 0.5f * a.tc_e1;
              c0 = 0.5f * a.tc_e1 * ni + a.tc_e0;
            } else {
              c1 = a.tc_e1;
              c0 = a.tc_e1 * ni + a.tc_e0;
            }
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
              bits |= 1u << t;
            else if (!(x > B))
              unsure |= 1u << t;
          }
          while (unsure) {
            const int t = __ffs(unsure) - 1;
            unsure &= unsure - 1u;
            const int ii = 32 * rb + t;
            const uint32_t slot = atomicAdd(qn, 1u);
            if (slot < TCP_QCAP) {
              uq[slot] = (uint32_t)(ii << 8 | j);
            } else {
              const float dd = canon_dist_thread<METRIC, G, K>(Cs, ii, Cs, j, NQ, nch, a.d);
              if (__fmul_rn(a.alpha2, dd) <= key_dist(keys[j])) bits |= 1u << t;
            }
          }
        }
        uint32_t word = 0;
#pragma unroll
        for (int t = 0; t < 32; ++t) {
          const uint32_t b = __ballot_sync(FULL, (bits >> t) & 1u);
          if (lane == t) word = b;
        }
        const int i = 32 * rb + lane;
        if (i < m) dom[i * W + cb] = word;
      };
      if constexpr (NC == 256) {
        // lane quarter q: row blocks q (8 - q column blocks) and q + 4
        // (4 - q); warp q + 4 takes row block q's last two
        const int q4 = warp & 3;
        if (warp < 4) {
          for (int cb = q4; cb < 6; ++cb) row_job(q4, cb);
        } else {
          for (int cb = q4 + 4; cb < 8; ++cb) row_job(q4 + 4, cb);
          row_job(q4, 6);
          row_job(q4, 7);
        }
      } else {
        // warp 0 rows 0..31 x blocks 0 and 1; warps 2 and 3 take blocks
        // (0, 2) and (0, 3) by columns
        for (int cb = warp == 0 ? 0 : warp; cb < (warp == 0 ? 2 : W); ++cb) row_job(warp, cb);
        if (warp >= 2) col_job(0, warp);
      }
      named_sync(1, NC);
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
      named_sync(1, NC);
      if (tid == 0) {
        *qn = 0u;  // read by every compute thread before the barrier above
        srow[s].p = p;
        srow[s].qidx = qidx;
        srow[s].m = m;
        mbar_arrive(full + s);  // the slot goes to the walker
      }
      ++jr;
    }
    if (tid == 0) {
      // no more lists: the next list of each walker, once its slot is free,
      // is a slot row with m = -1, which ends the walker's loop (a walker
      // that gave up is left alone)
      for (int j = jr; j < jr + TCP_WALKERS; ++j) {
        const int s = j % S;
        bool freed = j < S;
        for (int it = 0; it < a.wait_polls && !freed; ++it)
          freed = mbar_try_wait(empty + s, (uint32_t)(j / S - 1) & 1u);
        if (freed) {
          srow[s].m = -1;
          mbar_arrive(full + s);
        } else {
          atomicOr(a.err, 1u);
        }
      }
    }
    if (!ok) {
      // let the products in flight land before the tensor memory is released
      for (int it = 0; it < kDrainPolls; ++it)
        if (mbar_try_wait(bar, phase)) break;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, T::TMEM_COLS);
  if (tid >= NC && lane == 0 && ev) atomicAdd(a.prune_ctr, ev);
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
