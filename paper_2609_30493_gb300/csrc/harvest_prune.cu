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
#include "hprune.cuh"
#include "internal.h"
#include "tcdist.cuh"

namespace fg {


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
          if (krow) {
            krow[kept] = keys[cur];
          } else {
            row[kept] = key_id(keys[cur]);
            if (a.D_out) a.D_out[p * a.R + kept] = key_dist(keys[cur]);
          }
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
                  uint32_t* long_cnt, const int32_t* qlist, float* D_out) {
  HPruneFn kern = hprune_kernel_for(L.metric, L.G, L.K);
  if (!kern) {
    set_error(1, "no prune kernel for this metric and dimension");
    return 1;
  }
  HPruneArgs a{L.X, L.ld_bytes, L.d, L.nchunks, Eg, Eg_cnt, ecap,
               harvest_prune_smem(ecap, L.nchunks), nq, q_first, q_step, R, alpha2,
               A_out, cnt_out, D_out, prune_ctr, rows, Eg_off, nq_dev, K_out, 0.0f, 0.0f, err,
               g_mma_wait_polls, nullptr, nullptr, qlist};
  int optin = 0, dev = 0, sm_bytes = 0;
  FG_CUDA(cudaGetDevice(&dev));
  FG_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  FG_CUDA(cudaDeviceGetAttribute(&sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  // Tensor-core tiles of 128 and 256 candidates.  A tile kernel appends the
  // lists longer than its tile to long_list; the next kernel takes that list.
  // At most 512 / (TMEM columns of a CTA) CTAs fit an SM: the shared memory
  // request is raised so that no more can be resident.
  auto launch_tc = [&](int nc, const int32_t* ql, const uint32_t* qcnt, int32_t* ll,
                       uint32_t* lcnt) -> int {
    HPruneFn tk = hprune_tc_kernel_for(L.metric, L.G, L.K, nc);
    HPruneArgs t = a;
    tc_error_bound(L.metric, L.nchunks, &t.tc_e1, &t.tc_e0);
    const int ctas = nc == 128 ? 4 : 1;
    t.smem = std::max(harvest_prune_tc_smem(L.nchunks, nc), sm_bytes / (ctas + 1));
    const int per_sm = std::min(ctas, sm_bytes / (t.smem + 1024));
    if (!tk || per_sm < 1) {
      set_error(1, "prune launch does not fit an SM");
      return 1;
    }
    t.qlist = ql;
    if (qcnt) t.nq_dev = qcnt;
    t.long_list = ll;
    t.long_cnt = lcnt;
    if (lcnt) FG_CUDA(cudaMemsetAsync(lcnt, 0, sizeof(uint32_t), s));
    FG_CUDA(raise_smem_limit(reinterpret_cast<const void*>(tk), t.smem));
    tk<<<per_sm * num_sms, nc + 32 * TCP_WALKERS, t.smem, s>>>(t);  // compute threads, walkers
    note_launch();
    FG_CUDA(cudaGetLastError());
    return 0;
  };
  const bool tc_ok = hprune_tc_kernel_for(L.metric, L.G, L.K, 128) && err && g_prune_tc &&
                     harvest_prune_tc_smem(L.nchunks, 128) <= optin;
  const bool tc256_ok = tc_ok && harvest_prune_tc_smem(L.nchunks, 256) <= optin;
  if (tc_ok && ecap <= 128) return launch_tc(128, qlist, nullptr, nullptr, nullptr);
  if (tc_ok && long_list && long_cnt) {
    // every list the 128 tile leaves fits the 256 tile when ecap <= 256;
    // longer list buffers leave them to the lane-group kernel
    int rc = launch_tc(128, qlist, nullptr, long_list, long_cnt);
    if (rc) return rc;
    if (tc256_ok && ecap <= 256) return launch_tc(256, long_list, long_cnt, nullptr, nullptr);
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
