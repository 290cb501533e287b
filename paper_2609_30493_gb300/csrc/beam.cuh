// Persistent warp-per-query beam search: the harvest of Section 3 (every
// point of block b searches S_b with itself as the query and its expanded set
// is occlusion-pruned into its own row) and the query search over the final
// graph.
//
// One warp owns one query at a time (claimed with an atomic counter).  The
// pool is the ef smallest (delta, id) keys evaluated so far, held sorted in
// registers (entry i in slot i/32 of lane i%32, bit 0 = expanded).  Each step
// expands the smallest unexpanded entry, streams the neighbour lists of S_b
// 32 ids at a time through an exact shared-memory visited hash, gathers the
// new vectors with 16-byte loads by G-lane groups, and merges the batch into
// the pool with a bitonic network.  The pool is by definition the ef best of
// everything evaluated, so the order in which neighbours arrive does not
// change it.  A query whose visited set or expanded list outgrows shared
// memory is abandoned and listed; the host runs the list again with the same
// kernel on per-warp global scratch.
#pragma once
#include "common.cuh"
#include "internal.h"
#include "tc.cuh"

namespace fg {

struct BeamArgs {
  // points: n rows of d elements, row stride ld_bytes, nchunks 16-byte chunks used
  const char* X;
  int64_t ld_bytes;
  int32_t d;
  int32_t nchunks;
  int64_t n;
  // first neighbour source: the scaffold (harvest) or the final graph (search)
  const int64_t* s_off;
  const int32_t* s_ids;
  // harvest: rows of earlier blocks and their reverse lists
  const int32_t* A;
  const int32_t* cnt;
  int32_t R;
  const int64_t* r_off;
  const int32_t* r_ids;
  int32_t B;  // >= 1
  int32_t b;
  // entry points
  const int32_t* roots;
  int32_t T;
  // work items w < nwork map to qidx = qlist ? qlist[w] : w; the harvest query
  // point is p = q_first + qidx * q_step, the search query row is Q + qidx*ldq
  const int32_t* qlist;
  const uint32_t* qlist_len;  // device count of qlist (NULL: use nq)
  int64_t nq;
  int64_t q_first;
  int64_t q_step;
  const char* Q;
  int64_t ldq_bytes;
  int32_t ef;
  int32_t mode;  // 0 = harvest + prune, 1 = search
  float alpha2;
  int32_t* A_out;
  int32_t* cnt_out;
  float* Ad_out;  // optional: delta(p, A_out[p][i]) beside each kept id
  int32_t k;
  int32_t* top_ids;
  float* top_d;
  uint32_t* q_evals;
  // scratch
  uint32_t* work;
  int32_t hash_log2;
  int32_t bitmap;     // 1: visited set is an n-bit bitmap, 0: bucketed hash
  int32_t vis_bytes;  // bytes of the visited region per warp (multiple of 16)
  int32_t vis_cap;
  // per-warp n-bit bitmaps in global memory: a query whose hash fills up moves
  // its visited ids there and continues (NULL: abandon and re-run instead)
  uint32_t* gvbits;
  int64_t gvbits_words;  // per warp, a multiple of 4
  int32_t ecap;  // power of two, >= 32
  int32_t wbytes;  // shared bytes per warp
  int32_t qbytes;  // staging bytes per warp for one vector (16 * nchunks, rounded)
  int32_t global_scratch;
  char* gscratch;
  int64_t gscratch_per_warp;
  int32_t* ovf_list;
  uint32_t* ovf_count;
  uint32_t ovf_cap;  // capacity of ovf_list
  // harvest with a separate prune kernel: the expanded list of query qidx is
  // written to Eg[qidx * ecap ..] with its length in Eg_cnt[qidx] (-1 when the
  // query was handed to the re-run pass, which prunes in place)
  uint64_t* Eg;
  int32_t* Eg_cnt;
  uint32_t* err_flag;
  unsigned long long* counters;  // evals, expansions, prune evals, ids scanned, overflows
  // gather: 1 = the queued vectors are bulk-copied into a per-warp shared
  // buffer of 32 rows (after the staged query) and evaluated from there;
  // 0 = loaded into registers by the lane groups.  id_batch: chunks of 32
  // neighbour ids whose bitmap visited tests are issued together (1..2).
  int32_t gather;
  int32_t id_batch;
  int32_t wait_polls;
  // visited-set log (Section 5.5, a measurement): with vlog set, a harvest
  // search (mode 0) only searches; the ids it inserts into its visited set,
  // in insertion order, go to vlog[qidx * vlog_cap ..] (the first vlog_cap of
  // them) and the set's size to vlog_cnt[qidx] (-1 for a query point outside
  // [0, n)); no expanded list, prune or row is written.  qpoints: the query
  // point of work item qidx is qpoints[qidx] (NULL: q_first + qidx * q_step).
  const int32_t* qpoints;
  int32_t* vlog;
  int32_t* vlog_cnt;
  int32_t vlog_cap;
};

// Up to kMaxMulti independent builds in one launch (many indices harvested
// together): work item w belongs to build k with start[k] <= w < start[k+1]
// and is that build's work item w - start[k].  The descriptors travel in the
// kernel parameters (__grid_constant__, read in place); every field that
// shapes the per-warp shared layout is the same in all of them.
constexpr int kMaxMulti = 64;
struct BeamMulti {
  int32_t nidx;
  uint32_t* work;
  int64_t start[kMaxMulti + 1];
  BeamArgs d[kMaxMulti];
};
static_assert(sizeof(BeamMulti) <= 32764, "kernel parameters are limited to 32,764 bytes");

// Where a beam launch takes its work items from: one build (BeamArgs) or
// several (BeamMulti).
struct BeamSrcOne {
  static constexpr bool kMulti = false;
  const BeamArgs& a;
  __device__ const BeamArgs& first() const { return a; }
  __device__ uint32_t* work() const { return a.work; }
  __device__ int64_t total() const {
    return a.qlist_len ? min((int64_t)*a.qlist_len, (int64_t)a.ovf_cap) : a.nq;
  }
  __device__ int find(uint32_t) const { return 0; }
  __device__ const BeamArgs& desc(int) const { return a; }
  __device__ int64_t local(int, uint32_t w) const { return (int64_t)w; }
};
struct BeamSrcMany {
  static constexpr bool kMulti = true;
  const BeamMulti& P;
  __device__ const BeamArgs& first() const { return P.d[0]; }
  __device__ uint32_t* work() const { return P.work; }
  __device__ int64_t total() const { return P.start[P.nidx]; }
  __device__ int find(uint32_t w) const {
    int lo = 0, hi = P.nidx - 1;  // the last k with start[k] <= w
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (P.start[mid] <= (int64_t)w) lo = mid; else hi = mid - 1;
    }
    return lo;
  }
  __device__ const BeamArgs& desc(int k) const { return P.d[k]; }
  __device__ int64_t local(int k, uint32_t w) const { return (int64_t)w - P.start[k]; }
};

// Chunks of 32 neighbour ids whose bitmap visited tests are issued together
// (two keeps the harvest kernels within 128 registers without spills).
constexpr int kIdBatch = 2;

template <int METRIC, int G, int K, int S, bool GATHER>
struct Beam {

  // Evaluate queue[0..cnt) (cnt <= 32) against the staged query qs and merge
  // the keys into the pool.  Lane groups of P lanes take one candidate each.
  static __device__ __forceinline__ void eval_merge(const BeamArgs& a, const uint4* qs,
                                                    const int32_t* queue, int cnt,
                                                    uint64_t (&pool)[S], int lane, uint4* gb,
                                                    uint64_t* gbar, uint32_t& gphase) {
    using L = Lanes<G, K>;
    const int g = lane / L::P, j = lane % L::P;
    uint64_t mykey = PAD;
    if constexpr (GATHER) {
      // every queued row in flight at once: one bulk copy per lane into the
      // warp's buffer, completion counted in bytes on the warp's barrier
      const uint32_t rb = 16u * (uint32_t)a.nchunks;
      if (lane == 0) mbar_arrive_expect_tx(gbar, rb * (uint32_t)cnt);
      __syncwarp();
      if (lane < cnt)
        bulk_g2s(gb + (int64_t)lane * a.nchunks, a.X + (int64_t)queue[lane] * a.ld_bytes, rb, gbar);
      bool ok = false;
      for (int it = 0; it < a.wait_polls && !ok; ++it) ok = mbar_try_wait(gbar, gphase);
      if (!ok) {
        // a copy did not land in time: record it, and let it land before the
        // buffer is used again (the results of this launch are reported bad)
        if (lane == 0) atomicOr(a.err_flag + 3, 1u);
        for (int it = 0; it < kDrainPolls && !ok; ++it) ok = mbar_try_wait(gbar, gphase);
      }
      gphase ^= 1u;
      __syncwarp();
    }
    // float32 metrics keep this lane's query chunks in registers for the
    // whole batch (uint8 rows read them from shared memory)
    uint4 qr[L::VL][K];
    if constexpr (METRIC != L2_U8) load_slots_smem<G, K>(qs, a.nchunks, j, qr);
    for (int base = 0; base < cnt; base += L::CPW * L::UW) {
      uint4 y[L::UW][L::VL][K];
#pragma unroll
      for (int u = 0; u < L::UW; ++u) {
        const int idx = base + u * L::CPW + g;
        if constexpr (GATHER) {
          load_slots_smem<G, K>(gb + (int64_t)(idx < cnt ? idx : 0) * a.nchunks, a.nchunks, j,
                                y[u]);
        } else {
          const int32_t id = idx < cnt ? queue[idx] : queue[0];
          load_slots<G, K>(a.X + (int64_t)id * a.ld_bytes, a.nchunks, j, y[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < L::UW; ++u) {
        float dd;
        if constexpr (METRIC != L2_U8)
          dd = regs_dist<METRIC, G, K>(qr, y[u], a.nchunks, a.d, j, FULL);
        else
          dd = slots_dist<METRIC, G, K>(qs, y[u], a.nchunks, a.d, j);
        const int rel = lane - base - u * L::CPW;
        const float got = __shfl_sync(FULL, dd, (rel & (L::CPW - 1)) * L::P);
        if (rel >= 0 && rel < L::CPW && lane < cnt) mykey = make_key(got, queue[lane]);
      }
    }
    merge_into_pool<S>(pool, mykey, a.ef, lane);
  }

  template <class Src>
  static __device__ void run(const Src& src, unsigned char* smem) {
    using L = Lanes<G, K>;
    const BeamArgs& a0 = src.first();  // the per-warp layout (the same in every descriptor)
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int g = lane / L::P, j = lane % L::P;
    const int64_t gwarp = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    unsigned char* wsm = smem + (int64_t)wib * a0.wbytes;
    const uint32_t nslots = 1u << a0.hash_log2;
    const uint32_t mask_buckets = nslots / 4 - 1;
    // Shared-memory pass: [visited | expanded list | alive bits | queue | staged vector]
    // per warp.  Re-run pass (global_scratch): the visited set is this warp's
    // n-bit bitmap in gvbits, the expanded list and alive bits live in gscratch,
    // and shared memory holds only the queue and the staged vector.
    uint32_t* vis0;
    uint64_t* E;
    uint32_t* alive;
    unsigned char* tail;
    if (a0.global_scratch) {
      vis0 = a0.gvbits + gwarp * a0.gvbits_words;
      E = reinterpret_cast<uint64_t*>(a0.gscratch + gwarp * a0.gscratch_per_warp);
      alive = reinterpret_cast<uint32_t*>(E + a0.ecap);
      tail = wsm;
    } else {
      vis0 = reinterpret_cast<uint32_t*>(wsm);
      E = reinterpret_cast<uint64_t*>(wsm + a0.vis_bytes);
      alive = reinterpret_cast<uint32_t*>(wsm + a0.vis_bytes + 8ll * a0.ecap);
      // the alive bits take ecap/8 bytes, rounded up so that the staged vector
      // after the queue keeps its 16-byte alignment
      tail = wsm + a0.vis_bytes + 8ll * a0.ecap + ((a0.ecap / 8 + 15) & ~15);
    }
    int32_t* queue = reinterpret_cast<int32_t*>(tail);
    uint4* qs = reinterpret_cast<uint4*>(tail + 256);
    // gather buffer (32 rows) and its barrier after the staged query
    uint4* gb = GATHER ? reinterpret_cast<uint4*>(tail + 256 + a0.qbytes) : nullptr;
    uint64_t* gbar =
        GATHER ? reinterpret_cast<uint64_t*>(tail + 256 + a0.qbytes + 32ll * 16 * a0.nchunks)
               : nullptr;
    uint32_t gphase = 0;
    if (GATHER) {
      if (lane == 0) {
        mbar_init(gbar, 1);
        fence_mbar_init();
      }
      __syncwarp();
    }
    const int64_t nwork = src.total();
    unsigned long long c_ev = 0, c_ex = 0, c_pe = 0, c_sc = 0, c_ovf = 0;
    int kcur = 0;  // the build whose counters accumulate in c_*
    auto flush = [&](const BeamArgs& ab) {
      if (lane == 0) {
        atomicAdd(ab.counters + 0, c_ev);
        atomicAdd(ab.counters + 1, c_ex);
        atomicAdd(ab.counters + 2, c_pe);
        atomicAdd(ab.counters + 3, c_sc);
        atomicAdd(ab.counters + 4, c_ovf);
      }
      c_ev = c_ex = c_pe = c_sc = c_ovf = 0;
    };

    for (;;) {
      uint32_t w0 = 0;
      if (lane == 0) w0 = atomicAdd(src.work(), 1u);
      w0 = __shfl_sync(FULL, w0, 0);
      if ((int64_t)w0 >= nwork) break;
      const int kb = src.find(w0);
      if (Src::kMulti && kb != kcur) {
        flush(src.desc(kcur));
        kcur = kb;
      }
      const BeamArgs& a = src.desc(kb);
      const int64_t w = src.local(kb, w0);
      const int64_t qidx = a.qlist ? (int64_t)a.qlist[w] : w;
      int64_t p = -1;
      const char* qrow;
      if (a.mode == 0) {
        p = a.qpoints ? (int64_t)a.qpoints[qidx] : a.q_first + qidx * a.q_step;
        if (p < 0 || p >= a.n) {  // only a logged query list can hold such an id
          if (lane == 0 && a.vlog_cnt) a.vlog_cnt[qidx] = -1;
          continue;
        }
        qrow = a.X + p * a.ld_bytes;
      } else {
        qrow = a.Q + qidx * a.ldq_bytes;
      }
      stage_row(qs, qrow, a.nchunks, lane);
      uint32_t* hash = vis0;
      bool bm = a.bitmap != 0;
      int vis_cap = a.vis_cap;
      {
        const uint4 fill = bm ? make_uint4(0u, 0u, 0u, 0u) : make_uint4(EMPTY, EMPTY, EMPTY, EMPTY);
        for (int i = lane; i < a.vis_bytes / 16; i += 32) reinterpret_cast<uint4*>(hash)[i] = fill;
      }
      __syncwarp();
      uint64_t pool[S];
#pragma unroll
      for (int s = 0; s < S; ++s) pool[s] = PAD;
      int qn = 0;
      int nvis = 0, ne = 0;
      bool ovf = false;
      unsigned long long q_sc = 0;

      // One id stream per step, cut in up to three segments: first the tree
      // roots, then for each expansion the scaffold row, the row of an earlier
      // block and the reverse list of the expanded vertex.  New ids (visited
      // set insert) are queued; full batches of 32 are evaluated and merged.
      const int32_t* sp0 = a.roots;
      const int32_t* sp1 = nullptr;
      const int32_t* sp2 = nullptr;
      int len0 = a.T, len1 = 0, len2 = 0;
      for (;;) {
        const int total = len0 + len1 + len2;
        // the ids of the next chunk of 32 are loaded before this chunk is
        // processed, so their latency overlaps its visited inserts and merge
        auto load_id = [&](int i) -> int32_t {
          if (i < len0) return sp0[i];
          if (i < len0 + len1) return sp1[i - len0];
          if (i < total) return sp2[i - len0 - len1];
          return -1;
        };
        int32_t v_next = load_id(lane);
        for (int base = 0; base < total;) {
          // With a bitmap the visited tests of up to kIdBatch chunks of 32 ids
          // are issued together (independent atomics, one round trip); the
          // hash inserts one chunk at a time.  Either way the chunks are queued
          // in stream order, and the visited set is the same set.
          int32_t vv[kIdBatch];
          bool nw[kIdBatch];
          int nchk = 1;
          vv[0] = v_next;
          if (bm) {
            nchk = min(min(kIdBatch, a.id_batch), (total - base + 31) >> 5);
#pragma unroll
            for (int u = 1; u < kIdBatch; ++u)
              vv[u] = u < nchk ? load_id(base + 32 * u + lane) : -1;
            if (base + 32 * nchk < total) v_next = load_id(base + 32 * nchk + lane);
            uint32_t old[kIdBatch];
#pragma unroll
            for (int u = 0; u < kIdBatch; ++u)
              old[u] = vv[u] >= 0 ? atomicOr(hash + (vv[u] >> 5), 1u << (vv[u] & 31)) : FULL;
#pragma unroll
            for (int u = 0; u < kIdBatch; ++u)
              nw[u] = vv[u] >= 0 && (old[u] & (1u << (vv[u] & 31))) == 0u;
          } else {
            if (base + 32 < total) v_next = load_id(base + 32 + lane);
            nw[0] = vv[0] >= 0 && hash_insert(hash, mask_buckets, (uint32_t)vv[0]);
#pragma unroll
            for (int u = 1; u < kIdBatch; ++u) nw[u] = false;
          }
#pragma unroll
          for (int u = 0; u < kIdBatch; ++u) {
          if (u < nchk) {
          const int32_t v = vv[u];
          const bool isnew = nw[u];
          const unsigned m = __ballot_sync(FULL, isnew);
          if (isnew) queue[qn + __popc(m & ((1u << lane) - 1u))] = v;
          if (a.vlog != nullptr && isnew) {
            const int pos = nvis + __popc(m & ((1u << lane) - 1u));
            if (pos < a.vlog_cap) a.vlog[qidx * (int64_t)a.vlog_cap + pos] = v;
          }
          qn += __popc(m);
          nvis += __popc(m);
          __syncwarp();
          if (nvis > vis_cap) {
            if (a.gvbits == nullptr) {
              ovf = true;
              break;
            }
            // move the hash's ids into this warp's global bitmap and go on
            uint32_t* gb = a.gvbits + gwarp * a.gvbits_words;
            for (int64_t w = lane; w < a.gvbits_words / 4; w += 32)
              reinterpret_cast<uint4*>(gb)[w] = make_uint4(0u, 0u, 0u, 0u);
            __syncwarp();
            for (uint32_t slot = lane; slot < nslots; slot += 32) {
              const uint32_t id = hash[slot];
              if (id != EMPTY) atomicOr(gb + (id >> 5), 1u << (id & 31));
            }
            __syncwarp();
            hash = gb;
            bm = true;
            vis_cap = INT_MAX;
          }
          if (qn >= 32) {
            eval_merge(a, qs, queue, 32, pool, lane, gb, gbar, gphase);
            const int rest = qn - 32;
            const int32_t t = lane < rest ? queue[32 + lane] : 0;
            __syncwarp();
            if (lane < rest) queue[lane] = t;
            __syncwarp();
            qn = rest;
          }
          }
          }
          if (ovf) break;
          base += 32 * nchk;
        }
        if (ovf) break;
        if (qn > 0) {
          eval_merge(a, qs, queue, qn, pool, lane, gb, gbar, gphase);
          __syncwarp();
          qn = 0;
        }
        // expand the smallest unexpanded pool entry
        int idx = -1;
#pragma unroll
        for (int s = 0; s < S; ++s) {
          const unsigned m = __ballot_sync(FULL, (pool[s] & 1ull) == 0ull);
          if (m && idx < 0) idx = s * 32 + __ffs(m) - 1;
        }
        if (idx < 0) break;
        if (ne >= a.ecap) {
          ovf = true;
          break;
        }
        uint64_t ck = 0;
#pragma unroll
        for (int s = 0; s < S; ++s) {
          if (s == idx / 32) {
            ck = __shfl_sync(FULL, pool[s], idx % 32);
            if (lane == idx % 32) pool[s] |= 1ull;
          }
        }
        if (lane == 0) E[ne] = ck;
        ++ne;
        const int32_t c = key_id(ck);
        const int64_t s0 = a.s_off[c];
        sp0 = a.s_ids + s0;
        len0 = (int)(a.s_off[c + 1] - s0);
        len1 = len2 = 0;
        if (a.mode == 0) {
          sp1 = a.A + (int64_t)c * a.R;
          len1 = (c % a.B) < a.b ? a.cnt[c] : 0;
          if (a.r_off) {
            const int64_t r0 = a.r_off[c];
            sp2 = a.r_ids + r0;
            len2 = (int)(a.r_off[c + 1] - r0);
          }
        }
        q_sc += (unsigned long long)(len0 + len1 + len2);
      }
      __syncwarp();

      if (ovf) {
        if (lane == 0) {
          if (a.Eg) a.Eg_cnt[qidx] = -1;
          if (a.global_scratch) {
            atomicOr(a.err_flag, 1u);
          } else {
            uint32_t pos = atomicAdd(a.ovf_count, 1u);
            if (pos < a.ovf_cap) {
              a.ovf_list[pos] = (int32_t)qidx;
            } else {
              atomicOr(a.err_flag, 1u);
            }
          }
        }
        c_ovf++;
        continue;
      }
      c_ev += (unsigned long long)nvis;
      c_ex += (unsigned long long)ne;
      c_sc += q_sc;

      if (a.vlog != nullptr) {
        if (lane == 0) a.vlog_cnt[qidx] = nvis;
        continue;
      }
      if (a.mode == 1) {
#pragma unroll
        for (int s = 0; s < S; ++s) {
          int i = s * 32 + lane;
          if (i < a.k) {
            uint64_t kk = pool[s];
            a.top_ids[qidx * a.k + i] = kk == PAD ? -1 : key_id(kk);
            a.top_d[qidx * a.k + i] = kk == PAD ? __int_as_float(0x7f800000) : key_dist(kk);
          }
        }
        if (lane == 0 && a.q_evals) a.q_evals[qidx] = (uint32_t)nvis;
        continue;
      }

      if (a.Eg) {
        // the prune runs in its own kernel with the candidates staged on chip
        uint64_t* dst = a.Eg + qidx * (int64_t)a.ecap;
        for (int i = lane; i < ne; i += 32) dst[i] = E[i];
        if (lane == 0) a.Eg_cnt[qidx] = ne;
        __syncwarp();
        continue;
      }

      // ---- occlusion prune of the expanded set (Section 3) ----
      int NE2 = 32;
      while (NE2 < ne) NE2 <<= 1;
      int m = 0;
      for (int i0 = 0; i0 < NE2; i0 += 32) {
        int i = i0 + lane;
        uint64_t kk = i < ne ? E[i] : PAD;
        if (kk != PAD && key_id(kk) == (int32_t)p) kk = PAD;
        E[i] = kk;
        m += __popc(__ballot_sync(FULL, kk != PAD));
      }
      __syncwarp();
      warp_sort_mem(E, NE2, lane);
      const int nw = (m + 31) / 32;
      for (int w2 = lane; w2 < nw; w2 += 32)
        alive[w2] = (w2 * 32 + 32 <= m) ? FULL : ((1u << (m - w2 * 32)) - 1u);
      __syncwarp();
      int32_t* row = a.A_out + p * a.R;
      int kept = 0, cur = -1;
      unsigned long long q_pe = 0;
      while (kept < a.R) {
        int nxt = -1;
        for (int w2 = (cur + 1) / 32; w2 < nw && nxt < 0; ++w2) {
          uint32_t bits = alive[w2];
          if (w2 == (cur + 1) / 32) bits &= ~((1u << ((cur + 1) % 32)) - 1u);
          if (bits) nxt = w2 * 32 + __ffs(bits) - 1;
        }
        if (nxt < 0) break;
        cur = nxt;
        const int32_t cid = key_id(E[cur]);
        if (lane == 0) {
          row[kept] = cid;
          if (a.Ad_out) a.Ad_out[p * a.R + kept] = key_dist(E[cur]);
          alive[cur / 32] &= ~(1u << (cur % 32));
        }
        ++kept;
        __syncwarp();
        if (kept == a.R) break;
        // the query is no longer needed: stage c* in its place
        __syncwarp();
        stage_row(qs, a.X + (int64_t)cid * a.ld_bytes, a.nchunks, lane);
        for (int w2 = cur / 32; w2 < nw; ++w2) {
          uint32_t bits = alive[w2];
          if (w2 == cur / 32) bits &= ~((2u << (cur % 32)) - 1u);
          q_pe += (unsigned long long)__popc(bits);
          uint32_t kill = 0;
          while (bits) {
            const int nb = __popc(bits);
            uint4 y[L::UW][L::VL][K];
            int jj[L::UW];
#pragma unroll
            for (int u = 0; u < L::UW; ++u) {
              const int r = u * L::CPW + g;
              jj[u] = r < nb ? nth_set_bit(bits, r) : -1;
              const int e = w2 * 32 + (jj[u] >= 0 ? jj[u] : 0);
              load_slots<G, K>(a.X + (int64_t)key_id(E[e]) * a.ld_bytes, a.nchunks, j, y[u]);
            }
#pragma unroll
            for (int u = 0; u < L::UW; ++u) {
              const float dd = slots_dist<METRIC, G, K>(qs, y[u], a.nchunks, a.d, j);
              if (jj[u] >= 0 && j == 0) {
                const float dp = key_dist(E[w2 * 32 + jj[u]]);
                if (__fmul_rn(a.alpha2, dd) <= dp) kill |= 1u << jj[u];
              }
            }
            const int consumed = nb < L::CPW * L::UW ? nb : L::CPW * L::UW;
            if (consumed >= nb) {
              bits = 0;
            } else {
              bits &= ~((1u << nth_set_bit(bits, consumed)) - 1u);
            }
          }
          kill = __reduce_or_sync(FULL, kill);
          if (lane == 0) alive[w2] &= ~kill;
          __syncwarp();
        }
      }
      for (int r = kept + lane; r < a.R; r += 32) row[r] = -1;
      if (lane == 0) a.cnt_out[p] = kept;
      c_pe += q_pe;
      __syncwarp();
    }
    flush(src.desc(kcur));
  }
};

// GATHER: candidate rows bulk-copied into a shared buffer (BeamArgs::gather);
// instantiated for rows of at most 64 chunks.
template <int METRIC, int G, int K, int S, bool GATHER>
__global__ void __launch_bounds__(128, 4) beam_kernel(const BeamArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  Beam<METRIC, G, K, S, GATHER>::run(BeamSrcOne{a}, smem);
}

// The same search over the work items of several builds in one launch.
template <int METRIC, int G, int K, int S, bool GATHER>
__global__ void __launch_bounds__(128, 4) beam_multi_kernel(const __grid_constant__ BeamMulti P) {
  extern __shared__ __align__(16) unsigned char smem[];
  Beam<METRIC, G, K, S, GATHER>::run(BeamSrcMany{P}, smem);
}

// Host-side launcher table entry (defined per metric in beam_*.cu, the
// gather variants in beam_*_g.cu).
using BeamKernelFn = void (*)(const BeamArgs);
using BeamMultiFn = void (*)(const BeamMulti);
BeamKernelFn beam_kernel_metric0(int G, int K, int S);
BeamKernelFn beam_kernel_metric1(int G, int K, int S);
BeamKernelFn beam_kernel_metric2(int G, int K, int S);
BeamKernelFn beam_kernel_metric0_gather(int G, int K, int S);
BeamKernelFn beam_kernel_metric1_gather(int G, int K, int S);
BeamKernelFn beam_kernel_metric2_gather(int G, int K, int S);
BeamMultiFn beam_multi_metric0(int G, int K, int S);
BeamMultiFn beam_multi_metric1(int G, int K, int S);
BeamMultiFn beam_multi_metric2(int G, int K, int S);

}  // namespace fg
