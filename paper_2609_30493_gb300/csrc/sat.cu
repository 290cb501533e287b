// Spatial-approximation forest on the GPU (the scaffold of Section 1 and
// Section 3, after Navarro 2002), built level by level for all T trees at
// once.
//
// A node a holding the point set P picks its children by the sorted greedy
// scan: in (delta(x,a), id) order, x joins iff delta(x,a) < delta(x,b) for
// every child b already chosen.  Here the scan is run without a sort, as a
// sequence of minimum selections: the next child is the smallest key among
// the points no child has rejected yet (every smaller key is a child or
// rejected, so this is exactly the point the scan would accept next), and the
// new child then rejects every remaining point y with delta(y,b) <= delta(y,a).
// Only the points not yet rejected are evaluated in this phase, a few percent
// of |P| x children on clustered data.  A second, coherent phase then gives
// every other point its closest child by (delta, id): the children are staged
// in shared memory and each point is read once per chunk of children.
// Small nodes get one CTA; nodes of many points are split across CTAs, one
// launch per child selection.  The points of all nodes of a level are grouped
// by a counting sort keyed on (tree, node).
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "tcdist.cuh"

namespace fg {

struct SatSegArgs {
  const char* X;
  int64_t ld_bytes;
  int32_t d;
  int32_t nchunks;
  int64_t n;
  const int32_t* item_pt;
  const int64_t* seg_start;
  const int32_t* seg_len;
  const int32_t* seg_node;
  const int32_t* seg_tree;
  uint64_t* lst0;  // open lists: keys (delta to the node's point, id) of the points
  uint64_t* lst1;  // no child has rejected yet, two buffers over each item range
  uint64_t* best;  // closest child by (delta, id); bit 0 marks a child itself
  int32_t* kid;    // kid[start + t] = t-th child of the node of that item range
  int32_t kc;      // children staged per chunk in the assignment phase
  int32_t ls;      // open points the selection can stage in shared memory
  int64_t seg_off; // first segment of a launch of the one-CTA-per-node kernel
  int32_t* seg_k;  // children per segment when the assignment runs as its own launch,
                   // else null (the node's CTA assigns its points itself)
  int32_t* node_of;
  int32_t* parent;
  unsigned long long* ctr;
  int32_t wait_polls;  // first bounded wait of the tensor-core assignment
};

// Minimum of one key per thread over the CTA; rk[parity] is the scratch, and
// consecutive calls alternate the parity so no second barrier is needed.
template <int NW>
__device__ __forceinline__ uint64_t block_min64(uint64_t key, uint64_t (*rk)[NW], int parity) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) key = umin64(key, __shfl_xor_sync(FULL, key, off));
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) rk[parity][warp] = key;
  __syncthreads();
  key = PAD;
#pragma unroll
  for (int w = 0; w < NW; ++w) key = umin64(key, rk[parity][w]);
  return key;
}

// The same with the index of the minimum carried along (keys are unique).
template <int NW>
__device__ __forceinline__ uint64_t block_argmin64(uint64_t key, int& idx, uint64_t (*rk)[NW],
                                                   int (*ri)[NW], int parity) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const uint64_t ok = __shfl_xor_sync(FULL, key, off);
    const int oi = __shfl_xor_sync(FULL, idx, off);
    if (ok < key) {
      key = ok;
      idx = oi;
    }
  }
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    rk[parity][warp] = key;
    ri[parity][warp] = idx;
  }
  __syncthreads();
  key = PAD;
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    const uint64_t kk = rk[parity][w];
    if (kk < key) {
      key = kk;
      idx = ri[parity][w];
    }
  }
  return key;
}

__device__ __forceinline__ uint64_t warp_min64(uint64_t v) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) v = umin64(v, __shfl_xor_sync(FULL, v, off));
  return v;
}

// Slot in an append-only list for every lane with keep set (one atomic per
// warp).  All 32 lanes must call it.
__device__ __forceinline__ uint32_t warp_append(bool keep, uint32_t* counter) {
  const unsigned bal = __ballot_sync(FULL, keep);
  if (bal == 0) return 0;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(bal) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(counter, (uint32_t)__popc(bal));
  base = __shfl_sync(FULL, base, leader);
  return base + (uint32_t)__popc(bal & ((1u << lane) - 1u));
}

// Stage a row in shared memory with the whole CTA.
__device__ __forceinline__ void stage_row_cta(uint4* dst, const char* __restrict__ row,
                                              int nchunks) {
  for (int c = threadIdx.x; c < nchunks; c += blockDim.x)
    dst[c] = __ldg(reinterpret_cast<const uint4*>(row) + c);
}

// Distances from the node's point (staged in cvec) to the items [t0, t1) of
// the node: their keys go to lst[t0 .. t1); returns this thread's minimum.
template <int METRIC, int G, int K, int NW>
__device__ uint64_t sat_first(const SatSegArgs& a, int64_t start, int t0, int t1,
                              const uint4* cvec, uint64_t* lst) {
  using L = Lanes<G, K>;
  constexpr int STEP = L::CPW * L::U;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane / L::P, j = lane % L::P;
  uint64_t lmin = PAD;
  for (int base = t0 + warp * STEP; base < t1; base += NW * STEP) {
    uint4 y[L::U][L::VL][K];
    int32_t pt[L::U];
#pragma unroll
    for (int u = 0; u < L::U; ++u) {
      pt[u] = a.item_pt[start + min(base + u * L::CPW + g, t1 - 1)];
      load_slots<G, K>(a.X + (int64_t)pt[u] * a.ld_bytes, a.nchunks, j, y[u]);
    }
#pragma unroll
    for (int u = 0; u < L::U; ++u) {
      const float dd = slots_dist<METRIC, G, K>(cvec, y[u], a.nchunks, a.d, j);
      const int idx = base + u * L::CPW + g;
      if (idx < t1 && j == 0) {
        const uint64_t key = make_key(dd, pt[u]);
        lst[idx] = key;
        lmin = umin64(lmin, key);
      }
    }
  }
  return lmin;
}

// One child selection step over the open entries lin[e0, e1): the child b
// (key bk, staged in cvec) leaves the list, every entry y with
// delta(y, b) <= delta(y, a) is rejected, the rest are appended to lout
// through *cnt.  Returns this thread's minimum surviving key.
template <int METRIC, int G, int K, int NW>
__device__ uint64_t sat_step(const SatSegArgs& a, const uint64_t* lin, uint64_t* lout, int e0,
                             int e1, uint64_t bk, const uint4* cvec, uint32_t* cnt) {
  using L = Lanes<G, K>;
  constexpr int STEP = L::CPW * L::U;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane / L::P, j = lane % L::P;
  uint64_t lmin = PAD;
  for (int base = e0 + warp * STEP; base < e1; base += NW * STEP) {  // warp-uniform
    uint4 y[L::U][L::VL][K];
    uint64_t e[L::U];
#pragma unroll
    for (int u = 0; u < L::U; ++u) {
      e[u] = lin[min(base + u * L::CPW + g, e1 - 1)];
      load_slots<G, K>(a.X + (int64_t)key_id(e[u]) * a.ld_bytes, a.nchunks, j, y[u]);
    }
#pragma unroll
    for (int u = 0; u < L::U; ++u) {
      const float dd = slots_dist<METRIC, G, K>(cvec, y[u], a.nchunks, a.d, j);
      const bool keep =
          j == 0 && base + u * L::CPW + g < e1 && e[u] != bk && dd > key_dist(e[u]);
      const uint32_t pos = warp_append(keep, cnt);
      if (keep) {
        lout[pos] = e[u];
        lmin = umin64(lmin, e[u]);
      }
    }
  }
  return lmin;
}

// Shared-memory state of a CTA's selection once the open list is short: the
// rows of the open points, their keys and two index lists over them.
struct SelSmem {
  uint4* rows;     // ls rows of nchunks chunks
  uint64_t* skey;  // ls keys
  int32_t* sl0;    // ls indices
  int32_t* sl1;    // ls indices
  int32_t* krow;   // ls: staged row of the t-th child (while t < ls)
  int32_t ls;      // capacity
};

// The rest of a node's selection inside one CTA: starting from the open list
// lin (L entries, smallest key bk) and k children chosen so far, select until
// the list is empty.  Steps read the open points from global memory while
// the list is longer than sm.ls; then the open points are staged once in
// shared memory and the remaining steps touch no global memory.
// Step k appends through scnt[k % 3] and clears scnt[(k + 2) % 3] after its
// barrier (that counter was last read in step k - 1 and is next appended to
// in step k + 2, after another barrier), so all three must be zero and
// visible before the call.  Returns the number of children.
template <int METRIC, int G, int K, int NW>
__device__ int sat_select(const SatSegArgs& a, int64_t start, int32_t anode, int64_t tbase,
                          uint64_t* lin, uint64_t* lout, int L, uint64_t bk, int k, uint4* cvec,
                          const SelSmem& sm, uint64_t (*rk)[NW], int (*ri)[NW], uint32_t* scnt) {
  using Ln = Lanes<G, K>;
  const int nch = a.nchunks;
  int parity = 1;
  while (bk != PAD && L > sm.ls) {
    const int32_t b = key_id(bk);
    if (threadIdx.x == 0) {
      a.kid[start + k] = b;
      a.parent[tbase + b] = anode;
    }
    ++k;
    const int c = k % 3;
    stage_row_cta(cvec, a.X + (int64_t)b * a.ld_bytes, nch);
    __syncthreads();
    const uint64_t lmin = sat_step<METRIC, G, K, NW>(a, lin, lout, 0, L, bk, cvec, scnt + c);
    bk = block_min64<NW>(lmin, rk, parity);
    parity ^= 1;
    L = (int)scnt[c];
    uint64_t* t = lin;
    lin = lout;
    lout = t;
    if (threadIdx.x == 0) scnt[(k + 2) % 3] = 0;
  }
  if (bk == PAD) return k;
  // stage the open points
  __shared__ int sib;
  for (int i = threadIdx.x; i < L; i += NW * 32) {
    const uint64_t e = lin[i];
    sm.skey[i] = e;
    sm.sl0[i] = i;
    if (e == bk) sib = i;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < L * nch; idx += NW * 32) {
    const int i = idx / nch, ch = idx - i * nch;
    sm.rows[idx] =
        __ldg(reinterpret_cast<const uint4*>(a.X + (int64_t)key_id(sm.skey[i]) * a.ld_bytes) +
              ch);
  }
  __syncthreads();
  int ib = sib;
  int32_t* cl = sm.sl0;
  int32_t* nl = sm.sl1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane / Ln::P, j = lane % Ln::P;
  while (bk != PAD) {
    const int32_t b = key_id(bk);
    if (threadIdx.x == 0) {
      a.kid[start + k] = b;
      a.parent[tbase + b] = anode;
    }
    ++k;
    const int c = k % 3;
    const uint4* crow = sm.rows + (int64_t)ib * nch;
    uint64_t lmin = PAD;
    int li = -1;
    for (int base = warp * Ln::CPW; base < L; base += NW * Ln::CPW) {  // warp-uniform
      const int e = cl[min(base + g, L - 1)];
      uint4 y[Ln::VL][K];
      load_slots_smem<G, K>(sm.rows + (int64_t)e * nch, nch, j, y);
      const float dd = slots_dist<METRIC, G, K>(crow, y, nch, a.d, j);
      const uint64_t ek = sm.skey[e];
      const bool keep = j == 0 && base + g < L && ek != bk && dd > key_dist(ek);
      const uint32_t pos = warp_append(keep, scnt + c);
      if (keep) {
        nl[pos] = e;
        if (ek < lmin) {
          lmin = ek;
          li = e;
        }
      }
    }
    if (threadIdx.x == 0 && k - 1 < sm.ls) sm.krow[k - 1] = ib;
    bk = block_argmin64<NW>(lmin, li, rk, ri, parity);
    parity ^= 1;
    ib = li;
    L = (int)scnt[c];
    int32_t* t = cl;
    cl = nl;
    nl = t;
    if (threadIdx.x == 0) scnt[(k + 2) % 3] = 0;
  }
  return k;
}

// Assignment phase shared by both kernels: every item of [t0, t1) of the
// node gets its closest child by (delta, id) among the k children
// kid[start .. start+k), children staged kc at a time in kvec; children
// themselves get -1.  Called by all threads of the CTA.
template <int METRIC, int G, int K, int NW>
__device__ void sat_assign(const SatSegArgs& a, int64_t start, int t0, int t1, int k,
                           int64_t tbase, uint4* kvec, int32_t* kids) {
  using L = Lanes<G, K>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane / L::P, j = lane % L::P;
  const int NG = NW * L::CPW;
  const int gid = warp * L::CPW + g;
  const int nch = a.nchunks;
  for (int c0 = 0; c0 < k; c0 += a.kc) {
    const int kn = min(a.kc, k - c0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < kn * nch; idx += NW * 32) {
      const int t = idx / nch, ch = idx - t * nch;
      kvec[idx] = __ldg(reinterpret_cast<const uint4*>(
                            a.X + (int64_t)a.kid[start + c0 + t] * a.ld_bytes) + ch);
    }
    for (int t = threadIdx.x; t < kn; t += NW * 32) kids[t] = a.kid[start + c0 + t];
    __syncthreads();
    for (int base = t0; base < t1; base += NG) {
      const int64_t it = start + min(base + gid, t1 - 1);
      const int32_t pt = a.item_pt[it];
      uint4 xq[L::VL][K];
      load_slots<G, K>(a.X + (int64_t)pt * a.ld_bytes, nch, j, xq);
      uint64_t bk = PAD & ~1ull;
      bool self = false;
      for (int t = 0; t < kn; ++t) {
        uint4 y[L::VL][K];
        load_slots_smem<G, K>(kvec + (int64_t)t * nch, nch, j, y);
        const float dd = regs_dist<METRIC, G, K>(xq, y, nch, a.d, j, FULL);
        bk = umin64(bk, make_key(dd, kids[t]));
        self |= kids[t] == pt;
      }
      if (base + gid < t1 && j == 0) {
        const uint64_t prev = c0 == 0 ? (PAD & ~1ull) : a.best[it];
        a.best[it] = umin64(prev & ~1ull, bk) | (prev & 1ull) | (self ? 1ull : 0ull);
      }
    }
  }
  __syncthreads();
  for (int i = t0 + threadIdx.x; i < t1; i += NW * 32) {
    const int64_t it = start + i;
    const uint64_t bk = a.best[it];
    a.node_of[tbase + a.item_pt[it]] = (bk & 1ull) ? -1 : key_id(bk);
  }
}

__device__ __forceinline__ void sat_count(const SatSegArgs& a, int m, int k) {
  const long long mm = m, kk = k;
  atomicAdd(a.ctr, (unsigned long long)(mm + kk * (kk - 1) / 2 + (mm - kk) * kk));
}

// Dynamic shared memory of the SAT kernels: one row (the node's point, then
// each new child), then a region used first by the selection (SelSmem) and
// then by the assignment (kc staged children and their ids).
__device__ __forceinline__ SelSmem sel_smem(const SatSegArgs& a, unsigned char* base) {
  SelSmem sm;
  const int64_t nch = a.nchunks;
  sm.rows = reinterpret_cast<uint4*>(base) + nch;
  sm.skey = reinterpret_cast<uint64_t*>(sm.rows + (int64_t)a.ls * nch);
  sm.sl0 = reinterpret_cast<int32_t*>(sm.skey + a.ls);
  sm.sl1 = sm.sl0 + a.ls;
  sm.krow = sm.sl1 + a.ls;
  sm.ls = a.ls;
  return sm;
}

// Assignment of a node whose m points were all staged, in item order, when
// its selection began (m <= ls): point i is staged row i and the t-th child
// staged row krow[t], so no global memory is read.
template <int METRIC, int G, int K, int NW>
__device__ void sat_assign_staged(const SatSegArgs& a, const SelSmem& sm, int m, int k,
                                  int64_t tbase) {
  using L = Lanes<G, K>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane / L::P, j = lane % L::P;
  const int nch = a.nchunks;
  __syncthreads();  // krow of the last step
  for (int base = warp * L::CPW; base < m; base += NW * L::CPW) {  // warp-uniform
    const int i = min(base + g, m - 1);
    uint4 xq[L::VL][K];
    load_slots_smem<G, K>(sm.rows + (int64_t)i * nch, nch, j, xq);
    uint64_t best = PAD;
    bool self = false;
    for (int t = 0; t < k; ++t) {
      const int r = sm.krow[t];
      uint4 y[L::VL][K];
      load_slots_smem<G, K>(sm.rows + (int64_t)r * nch, nch, j, y);
      const float dd = regs_dist<METRIC, G, K>(xq, y, nch, a.d, j, FULL);
      best = umin64(best, make_key(dd, key_id(sm.skey[r])));
      self |= r == i;
    }
    if (base + g < m && j == 0) a.node_of[tbase + key_id(sm.skey[i])] = self ? -1 : key_id(best);
  }
}

// A node with fewer points: one CTA runs the whole construction of its
// children.
template <int METRIC, int G, int K, int NW>
__global__ void __launch_bounds__(NW * 32) sat_segment_kernel(const SatSegArgs a) {
  __shared__ uint64_t rk[2][NW];
  __shared__ int ri[2][NW];
  __shared__ uint32_t scnt[3];
  extern __shared__ __align__(16) unsigned char ssat[];
  uint4* cvec = reinterpret_cast<uint4*>(ssat);  // the node's point, then each new child
  uint4* kvec = cvec + a.nchunks;               // children staged for the assignment
  int32_t* kids = reinterpret_cast<int32_t*>(kvec + (int64_t)a.kc * a.nchunks);
  const SelSmem sm = sel_smem(a, ssat);
  const int64_t s = a.seg_off + blockIdx.x;
  const int64_t start = a.seg_start[s];
  const int m = a.seg_len[s];
  const int32_t anode = a.seg_node[s];
  const int64_t tbase = (int64_t)a.seg_tree[s] * a.n;
  if (threadIdx.x == 0) scnt[0] = scnt[1] = scnt[2] = 0;
  stage_row_cta(cvec, a.X + (int64_t)anode * a.ld_bytes, a.nchunks);
  __syncthreads();
  uint64_t* l0 = a.lst0 + start;
  const uint64_t lmin = sat_first<METRIC, G, K, NW>(a, start, 0, m, cvec, l0);
  const uint64_t bk = block_min64<NW>(lmin, rk, 0);
  const int k = sat_select<METRIC, G, K, NW>(a, start, anode, tbase, l0, a.lst1 + start, m, bk,
                                             0, cvec, sm, rk, ri, scnt);
  if (m <= sm.ls) {  // staged whole from the start
    sat_assign_staged<METRIC, G, K, NW>(a, sm, m, k, tbase);
    if (threadIdx.x == 0) {
      sat_count(a, m, k);
      if (a.seg_k) a.seg_k[s] = -1;  // nothing left for the assignment launch
    }
    return;
  }
  if (a.seg_k) {
    if (threadIdx.x == 0) a.seg_k[s] = k;
    return;
  }
  sat_assign<METRIC, G, K, NW>(a, start, 0, m, k, tbase, kvec, kids);
  if (threadIdx.x == 0) sat_count(a, m, k);
}

// The assignment as its own launch, tiles of ASSIGN_TILE points of a node per
// CTA: segment segs[y] (or seg_off + y without a list), its children counted
// in seg_k.
constexpr int ASSIGN_TILE = 256;
constexpr int ASSIGN_NW = 8;

template <int METRIC, int G, int K>
__global__ void __launch_bounds__(ASSIGN_NW * 32)
    sat_assign_kernel(const SatSegArgs a, const int32_t* segs, int32_t y_off) {
  extern __shared__ __align__(16) unsigned char sasg[];
  uint4* kvec = reinterpret_cast<uint4*>(sasg) + a.nchunks;
  int32_t* kids = reinterpret_cast<int32_t*>(kvec + (int64_t)a.kc * a.nchunks);
  const int y = blockIdx.y + y_off;
  const int64_t s = segs ? (int64_t)segs[y] : a.seg_off + y;
  const int m = a.seg_len[s];
  const int t0 = blockIdx.x * ASSIGN_TILE;
  const int k = a.seg_k[s];
  if (t0 >= m || k < 0) return;  // k < 0: assigned by the node's own CTA
  sat_assign<METRIC, G, K, ASSIGN_NW>(a, a.seg_start[s], t0, min(m, t0 + ASSIGN_TILE), k,
                                      (int64_t)a.seg_tree[s] * a.n, kvec, kids);
  if (blockIdx.x == 0 && threadIdx.x == 0) sat_count(a, m, k);
}

// The assignment on the tensor cores (float32 metrics).  A CTA takes 128
// points of a node (A) and the node's children 128 at a time (B), both staged
// in the canonical operand layout, and computes their Gram tile with
// kind::tf32 MMAs into 128 TMEM columns.  Thread i reads its point's row
// twice: first the bound ub = min over children of (approx + eps), then the
// candidates, the children with approx - eps <= ub; the canonical distance
// of the closest child is at most ub and every other child's at least its
// approx - eps, so the closest by (delta, id) is among the candidates, and
// only they are evaluated in canonical float32 (bound: tcdist.cuh).
constexpr int AT_M = 128;
struct AtSmem {
  int nq;
  __host__ __device__ int b_off() const { return AT_M * nq * 16; }
  __host__ __device__ int kid_off() const { return 2 * AT_M * nq * 16; }
  __host__ __device__ int na_off() const { return kid_off() + 4 * AT_M; }
  __host__ __device__ int nb_off() const { return na_off() + 4 * AT_M; }
  __host__ __device__ int bar_off() const { return nb_off() + 4 * AT_M; }
  __host__ __device__ int bytes() const { return bar_off() + 16; }
};

template <int METRIC, int G, int K>
__global__ void __launch_bounds__(AT_M)
    sat_assign_tc_kernel(const SatSegArgs a, const int32_t* segs, int32_t y_off, float e1,
                         float e0, uint32_t* err) {
  extern __shared__ __align__(128) unsigned char atsm[];
  const int y = blockIdx.y + y_off;
  const int64_t s = segs ? (int64_t)segs[y] : a.seg_off + y;
  const int m = a.seg_len[s];
  const int t0 = blockIdx.x * AT_M;
  const int k = a.seg_k[s];
  if (t0 >= m || k < 0) return;  // before any tensor memory is taken; k < 0: assigned
  const int na = min(AT_M, m - t0);
  const int64_t start = a.seg_start[s];
  const int64_t tbase = (int64_t)a.seg_tree[s] * a.n;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int nch = a.nchunks;
  const AtSmem L{tcp_nq(nch)};
  const int NQ = L.nq;
  uint4* As = reinterpret_cast<uint4*>(atsm);
  uint4* Bs = reinterpret_cast<uint4*>(atsm + L.b_off());
  int32_t* kids = reinterpret_cast<int32_t*>(atsm + L.kid_off());
  float* nra = reinterpret_cast<float*>(atsm + L.na_off());
  float* nrb = reinterpret_cast<float*>(atsm + L.nb_off());
  uint64_t* bar = reinterpret_cast<uint64_t*>(atsm + L.bar_off());
  uint32_t* tslot = reinterpret_cast<uint32_t*>(atsm + L.bar_off() + 8);
  // stage the points (rows past na zero), one row per thread
  tc_stage_row(As, tid,
               tid < na ? a.X + (int64_t)a.item_pt[start + t0 + tid] * a.ld_bytes : nullptr, NQ,
               nch, a.d);
  if (warp == 0) {
    tmem_alloc(tslot, AT_M);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
  const int i = tid;
  const float ni = i < na ? tc_norm2(As, i, NQ, nch) : 0.0f;
  const int32_t pt = i < na ? a.item_pt[start + t0 + i] : -1;
  uint64_t best = PAD;
  bool self = false, ok = true;
  uint32_t phase = 0;
  const uint32_t idesc = idesc_tf32(AT_M, AT_M);
  const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs), sbo = (uint32_t)NQ * 128u;
  for (int c0 = 0; c0 < k; c0 += AT_M) {
    const int kn = min(AT_M, k - c0);
    if (c0 > 0) {  // the previous chunk's MMAs and TMEM reads are done
      tc_fence_before();
      __syncthreads();
    }
    const int32_t kc = tid < kn ? a.kid[start + c0 + tid] : -1;
    tc_stage_row(Bs, tid, kc >= 0 ? a.X + (int64_t)kc * a.ld_bytes : nullptr, NQ, nch, a.d);
    if (tid < kn) kids[tid] = kc;
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      for (int kk = 0; kk < NQ / 2; ++kk)
        mma_tf32(tmem, smem_desc(a0 + kk * 256, 128, sbo), smem_desc(b0 + kk * 256, 128, sbo),
                 idesc, kk > 0 ? 1u : 0u);
      mma_commit(bar);
    }
    if (tid < kn) nrb[tid] = tc_norm2(Bs, tid, NQ, nch);
    bool done = false;
    for (int it = 0; it < a.wait_polls && !done; ++it) done = mbar_try_wait(bar, phase);
    done = __syncthreads_and(done);  // also publishes nrb
    if (!done) {
      ok = false;
      if (tid == 0) atomicOr(err, 1u);
      break;
    }
    phase ^= 1u;
    tc_fence_after();
    const int nb = (kn + 31) / 32;
    float ub = INFINITY;
    for (int cb = 0; cb < nb; ++cb) {  // uniform
      uint32_t v[32];
      tmem_ld32(trow + (uint32_t)(32 * cb), v);
#pragma unroll
      for (int t = 0; t < 32; ++t) {
        const int c = 32 * cb + t;
        float dt, eps;
        tc_approx<METRIC>(__uint_as_float(v[t]), ni, nrb[min(c, kn - 1)], e1, e0, &dt, &eps);
        if (c < kn) ub = fminf(ub, dt + eps);
      }
    }
    for (int cb = 0; cb < nb; ++cb) {
      uint32_t v[32];
      tmem_ld32(trow + (uint32_t)(32 * cb), v);
      uint32_t cand = 0;
#pragma unroll
      for (int t = 0; t < 32; ++t) {
        const int c = 32 * cb + t;
        float dt, eps;
        tc_approx<METRIC>(__uint_as_float(v[t]), ni, nrb[min(c, kn - 1)], e1, e0, &dt, &eps);
        if (c < kn && dt - eps <= ub) cand |= 1u << t;
      }
      if (i < na) {
        while (cand) {
          const int t = __ffs(cand) - 1;
          cand &= cand - 1u;
          const int c = 32 * cb + t;
          const float dd = canon_dist_thread<METRIC, G, K>(As, i, Bs, c, NQ, nch, a.d);
          best = umin64(best, make_key(dd, kids[c]));
        }
        for (int t = 0; t < 32 && 32 * cb + t < kn; ++t) self |= kids[32 * cb + t] == pt;
      }
    }
  }
  if (ok && i < na) a.node_of[tbase + pt] = self ? -1 : key_id(best);
  if (!ok) {
    for (int it = 0; it < kDrainPolls; ++it)
      if (mbar_try_wait(bar, phase)) break;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, AT_M);
  if (blockIdx.x == 0 && tid == 0) sat_count(a, m, k);
}

// ---------------------------------------------------------------------------
// Nodes with many points.  While a node's open list is long, every CTA of a
// launch owns a tile of it and one launch performs one child selection for
// all such nodes: survivors are appended to the other list through a global
// counter, and the minimum is reduced with a 64-bit atomicMin, both into one
// of three rotating per-node buffers (read, write, clear), so no CTA ever
// waits for another.  Once the lists are short, one CTA per node finishes
// the selection, and the assignment is again split into tiles.
// ---------------------------------------------------------------------------
constexpr int BIG_TILE = 512;   // points per CTA (modes 0 and 2)
constexpr int STEP_TILE = 256;  // open entries per CTA (mode 1)
constexpr int BIG_NW = 8;

struct SatBigArgs {
  SatSegArgs s;
  const int32_t* big;  // segment index of each big node
  uint64_t* cur;       // current minimum key per big node (the next child)
  uint64_t* nxt;       // receives the minimum of this pass
  uint64_t* clr;       // reset to PAD for the pass after
  uint32_t* curlen;    // open list length per big node, same rotation
  uint32_t* nxtlen;
  uint32_t* clrlen;
  uint64_t* lin;       // open lists read by this pass (offset by the item range)
  uint64_t* lout;      // and written
  uint32_t* kcount;    // children chosen so far per big node
  int32_t y_off;       // first big node of this launch (grid.y is limited to 65535)
};

// mode 0: keys of every point to the node's point, first minimum.
// mode 1: one child selection, tiles of the open list across CTAs.
// mode 3: the remaining selections, one CTA per node; the assignment follows
// as sat_assign_kernel.
template <int METRIC, int G, int K>
__global__ void __launch_bounds__(BIG_NW * 32) sat_big_kernel(const SatBigArgs A, int mode) {
  __shared__ uint64_t rk[2][BIG_NW];
  __shared__ int ri[2][BIG_NW];
  __shared__ uint32_t scnt[3];
  extern __shared__ __align__(16) unsigned char sbig[];
  const SatSegArgs& a = A.s;
  uint4* cvec = reinterpret_cast<uint4*>(sbig);
  const int y = blockIdx.y + A.y_off;
  const int sidx = A.big[y];
  const int64_t start = a.seg_start[sidx];
  const int m = a.seg_len[sidx];
  const int32_t anode = a.seg_node[sidx];
  const int64_t tbase = (int64_t)a.seg_tree[sidx] * a.n;
  if (mode == 3) {
    if (threadIdx.x == 0) scnt[0] = scnt[1] = scnt[2] = 0;
    __syncthreads();
    const uint64_t bk = A.cur[y];
    int k = (int)A.kcount[y];
    if (bk != PAD)
      k = sat_select<METRIC, G, K, BIG_NW>(a, start, anode, tbase, A.lin + start,
                                           A.lout + start, (int)A.curlen[y], bk, k, cvec,
                                           sel_smem(a, sbig), rk, ri, scnt);
    if (threadIdx.x == 0) a.seg_k[sidx] = k;
    return;
  }
  if (mode == 0) {
    const int t0 = blockIdx.x * BIG_TILE;
    if (t0 >= m) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) A.curlen[y] = (uint32_t)m;
    stage_row_cta(cvec, a.X + (int64_t)anode * a.ld_bytes, a.nchunks);
    __syncthreads();
    uint64_t lmin = sat_first<METRIC, G, K, BIG_NW>(a, start, t0, min(m, t0 + BIG_TILE), cvec,
                                                    A.lin + start);
    lmin = warp_min64(lmin);
    if ((threadIdx.x & 31) == 0 && lmin != PAD)
      atomicMin(reinterpret_cast<unsigned long long*>(A.cur + y), (unsigned long long)lmin);
    return;
  }
  // mode 1
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    A.clr[y] = PAD;
    A.clrlen[y] = 0;
  }
  const uint64_t bk = A.cur[y];
  if (bk == PAD) return;
  const int32_t b = key_id(bk);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const uint32_t k = A.kcount[y];
    a.kid[start + k] = b;
    a.parent[tbase + b] = anode;
    A.kcount[y] = k + 1;
  }
  const int L = (int)A.curlen[y];
  const int e0 = blockIdx.x * STEP_TILE;
  if (e0 >= L) return;
  stage_row_cta(cvec, a.X + (int64_t)b * a.ld_bytes, a.nchunks);
  __syncthreads();
  uint64_t lmin = sat_step<METRIC, G, K, BIG_NW>(a, A.lin + start, A.lout + start, e0,
                                                 min(L, e0 + STEP_TILE), bk, cvec, A.nxtlen + y);
  lmin = warp_min64(lmin);
  if ((threadIdx.x & 31) == 0 && lmin != PAD)
    atomicMin(reinterpret_cast<unsigned long long*>(A.nxt + y), (unsigned long long)lmin);
}

using SatBigFn = void (*)(const SatBigArgs, int);

using SatKernelFn = void (*)(const SatSegArgs);
int g_sat_tc = 1;  // closest-child assignment on the tensor cores where possible
constexpr int SAT_NW = 8;           // warps per CTA: nodes of more points, the big path
constexpr int TINY_NW = 1;          // warps per CTA: nodes that fit in shared memory
constexpr int SAT_SMEM = 96 * 1024; // dynamic shared memory per CTA, by CTA width
constexpr int TINY_SMEM = 12 * 1024;

template <int NW>
static SatKernelFn sat_kernel_for(int metric, int G, int K) {
#define SATX(M, GG, KK) \
  if (metric == M && G == GG && K == KK) return sat_segment_kernel<M, GG, KK, NW>;
#define SATF(M) SATX(M, 4, 1) SATX(M, 8, 1) SATX(M, 16, 1) SATX(M, 32, 1) SATX(M, 32, 2) \
  SATX(M, 32, 4) SATX(M, 32, 8)
  SATF(0)
  SATF(1)
  SATX(2, 4, 1) SATX(2, 8, 1) SATX(2, 16, 1)
#undef SATF
#undef SATX
  return nullptr;
}

// Shared-memory split for a CTA with `budget` bytes: open points staged by
// the selection (a.ls) and children staged per assignment chunk (a.kc).
// Returns the dynamic shared memory size.
static size_t sat_smem_plan(SatSegArgs& a, int budget) {
  const int row16 = a.nchunks * 16;
  a.ls = std::max(1, std::min(4096, (budget - row16) / (row16 + 20)));
  a.kc = std::max(1, std::min(256, (budget - row16) / (row16 + 4)));
  return (size_t)row16 + std::max((size_t)a.ls * (row16 + 20), (size_t)a.kc * (row16 + 4));
}

using SatAssignFn = void (*)(const SatSegArgs, const int32_t*, int32_t);

static SatAssignFn sat_assign_for(int metric, int G, int K) {
#define SATX(M, GG, KK) \
  if (metric == M && G == GG && K == KK) return sat_assign_kernel<M, GG, KK>;
#define SATF(M) SATX(M, 4, 1) SATX(M, 8, 1) SATX(M, 16, 1) SATX(M, 32, 1) SATX(M, 32, 2) \
  SATX(M, 32, 4) SATX(M, 32, 8)
  SATF(0)
  SATF(1)
  SATX(2, 4, 1) SATX(2, 8, 1) SATX(2, 16, 1)
#undef SATF
#undef SATX
  return nullptr;
}

using SatAssignTcFn = void (*)(const SatSegArgs, const int32_t*, int32_t, float, float,
                              uint32_t*);

static SatAssignTcFn sat_assign_tc_for(int metric, int G, int K) {
#define SATX(M, GG, KK) \
  if (metric == M && G == GG && K == KK) return sat_assign_tc_kernel<M, GG, KK>;
#define SATF(M) SATX(M, 4, 1) SATX(M, 8, 1) SATX(M, 16, 1) SATX(M, 32, 1) SATX(M, 32, 2) \
  SATX(M, 32, 4) SATX(M, 32, 8)
  SATF(0)
  SATF(1)
#undef SATF
#undef SATX
  return nullptr;
}

static SatBigFn sat_big_for(int metric, int G, int K) {
#define SATX(M, GG, KK) \
  if (metric == M && G == GG && K == KK) return sat_big_kernel<M, GG, KK>;
#define SATF(M) SATX(M, 4, 1) SATX(M, 8, 1) SATX(M, 16, 1) SATX(M, 32, 1) SATX(M, 32, 2) \
  SATX(M, 32, 4) SATX(M, 32, 8)
  SATF(0)
  SATF(1)
  SATX(2, 4, 1) SATX(2, 8, 1) SATX(2, 16, 1)
#undef SATF
#undef SATX
  return nullptr;
}

__global__ void sat_init_kernel(int64_t n, int T, const int32_t* roots, int32_t* node_of,
                                int32_t* parent) {
  const int64_t tot = (int64_t)T * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(i / n);
    const int32_t x = (int32_t)(i - (int64_t)t * n);
    node_of[i] = (x == roots[t]) ? -1 : roots[t];
    parent[i] = -1;
  }
}

__global__ void sat_count_kernel(int64_t n, int64_t tot, const int32_t* node_of, uint32_t* kcnt,
                                 uint32_t* err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = node_of[i];
    if (a >= n) {
      atomicOr(err, 1u);  // an invalid node id: recorded, never used as an index
      continue;
    }
    if (a >= 0) {
      const int64_t t = i / n;
      atomicAdd(&kcnt[t * n + a], 1u);
    }
  }
}

// Segment lists of a level: nodes of at most tiny_max points fill the list
// from the front (count nseg[0]), nodes of at least big_min points from
// big_base on (nseg[1], with their indices in big_list, most points in
// nseg[6]), the others from the top of the small-node region down (nseg[3],
// most points in nseg[5]).
__global__ void sat_segments_kernel(int64_t n, int64_t tot, const uint32_t* kcnt,
                                    const int64_t* kstart, int64_t* seg_start, int32_t* seg_len,
                                    int32_t* seg_node, int32_t* seg_tree, uint32_t* nseg,
                                    int32_t tiny_max, int32_t big_min, int32_t* big_list,
                                    int64_t big_base) {
  for (int64_t key = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; key < tot;
       key += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t c = kcnt[key];
    if (c) {
      int64_t s;
      if ((int32_t)c >= big_min) {
        const uint32_t j = atomicAdd(nseg + 1, 1u);
        s = big_base + j;
        big_list[j] = (int32_t)s;
        atomicMax(nseg + 6, c);
      } else if ((int32_t)c <= tiny_max) {
        s = atomicAdd(nseg, 1u);
      } else {
        s = tot - 1 - (int64_t)atomicAdd(nseg + 3, 1u);
        atomicMax(nseg + 5, c);
      }
      seg_start[s] = kstart[key];
      seg_len[s] = (int32_t)c;
      seg_node[s] = (int32_t)(key % n);
      seg_tree[s] = (int32_t)(key / n);
    }
  }
}

__global__ void sat_scatter_kernel(int64_t n, int64_t tot, const int32_t* node_of,
                                   uint32_t* kcnt, const int64_t* kstart, int32_t* item_pt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = node_of[i];
    if (a >= 0 && a < n) {
      const int64_t t = i / n;
      const int64_t key = t * n + a;
      const uint32_t r = atomicSub(&kcnt[key], 1u) - 1u;
      item_pt[kstart[key] + r] = (int32_t)(i - t * n);
    }
  }
}

static int grid_for(int64_t tot) {
  int64_t g = (tot + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)device_sms() * 32));
}

int sat_forest(const VecLayout& L, int T, const int32_t* roots_d, int32_t* parents,
               SatScratch& S, unsigned long long* ctr_sat, cudaStream_t s) {
  SatKernelFn kern = sat_kernel_for<SAT_NW>(L.metric, L.G, L.K);
  SatKernelFn tinyk = sat_kernel_for<TINY_NW>(L.metric, L.G, L.K);
  SatBigFn bigk = sat_big_for(L.metric, L.G, L.K);
  SatAssignFn asgk = sat_assign_for(L.metric, L.G, L.K);
  if (!kern || !tinyk || !bigk || !asgk) {
    set_error(1, "no SAT kernel for this metric and dimension");
    return 1;
  }
  const int64_t n = L.n, tot = (int64_t)T * n;
  FG_CUDA(cudaMemsetAsync(S.nseg + 4, 0, sizeof(uint32_t), s));
  sat_init_kernel<<<grid_for(tot), 256, 0, s>>>(n, T, roots_d, S.node_of, parents);
  note_launch();
  FG_CUDA(cudaGetLastError());
  SatSegArgs a;
  a.X = L.X;
  a.ld_bytes = L.ld_bytes;
  a.d = L.d;
  a.nchunks = L.nchunks;
  a.n = n;
  a.item_pt = S.item_pt;
  a.seg_start = S.seg_start;
  a.seg_len = S.seg_len;
  a.seg_node = S.seg_node;
  a.seg_tree = S.seg_tree;
  a.lst0 = S.lst;
  a.lst1 = S.lst + tot;
  a.best = S.best;
  a.kid = S.kid;
  a.node_of = S.node_of;
  a.parent = parents;
  a.ctr = ctr_sat;
  a.seg_off = 0;
  a.seg_k = nullptr;
  a.wait_polls = g_mma_wait_polls;
  SatSegArgs at = a;
  a.seg_k = S.seg_k;
  const size_t smem = sat_smem_plan(a, SAT_SMEM);
  const size_t smem_t = sat_smem_plan(at, TINY_SMEM);
  FG_CUDA(raise_smem_limit(reinterpret_cast<const void*>(kern), (int)smem));
  FG_CUDA(raise_smem_limit(reinterpret_cast<const void*>(bigk), (int)smem));
  FG_CUDA(raise_smem_limit(reinterpret_cast<const void*>(tinyk), (int)smem_t));
  FG_CUDA(raise_smem_limit(reinterpret_cast<const void*>(asgk), (int)smem));
  // the assignment launches: tiles of one node per grid column, nodes in rows
  // (grid.y is limited to 65535, so rows are covered in chunks)
  // on the tensor cores where the metric and the shared memory allow
  SatAssignTcFn asgtc = g_sat_tc ? sat_assign_tc_for(L.metric, L.G, L.K) : nullptr;
  size_t smem_tc = 0;
  float tc_e1 = 0.0f, tc_e0 = 0.0f;
  if (asgtc) {
    int dev = 0, optin = 0, sm_bytes = 0;
    FG_CUDA(cudaGetDevice(&dev));
    FG_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    FG_CUDA(cudaDeviceGetAttribute(&sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    // at most 512 / 128 CTAs on an SM (its tensor memory columns)
    smem_tc = std::max<size_t>(AtSmem{tcp_nq(L.nchunks)}.bytes(), sm_bytes / 5);
    if (smem_tc > (size_t)optin) {
      asgtc = nullptr;
    } else {
      FG_CUDA(raise_smem_limit(reinterpret_cast<const void*>(asgtc), (int)smem_tc));
      tc_error_bound(L.metric, L.nchunks, &tc_e1, &tc_e0);
    }
  }
  auto assign_all = [&](const int32_t* segs, uint32_t nrows, int64_t max_m) {
    const int tile = asgtc ? AT_M : ASSIGN_TILE;
    const unsigned gxa = (unsigned)((max_m + tile - 1) / tile);
    for (uint32_t y0 = 0; y0 < nrows; y0 += 65535u) {
      const dim3 grid(gxa, std::min<uint32_t>(65535u, nrows - y0));
      if (asgtc)
        asgtc<<<grid, AT_M, smem_tc, s>>>(a, segs, (int32_t)y0, tc_e1, tc_e0, S.nseg + 4);
      else
        asgk<<<grid, ASSIGN_NW * 32, smem, s>>>(a, segs, (int32_t)y0);
      note_launch();
    }
  };
  const int32_t tiny_max = at.ls;  // such nodes are staged in shared memory whole
  std::vector<uint64_t> hkeys;
  std::vector<uint32_t> hlens;
  for (int64_t level = 0; level <= n; ++level) {
    FG_CUDA(cudaMemsetAsync(S.nseg, 0, 4 * sizeof(uint32_t), s));
    FG_CUDA(cudaMemsetAsync(S.nseg + 5, 0, 2 * sizeof(uint32_t), s));
    sat_count_kernel<<<grid_for(tot), 256, 0, s>>>(n, tot, S.node_of, S.kcnt, S.nseg + 2);
    note_launch();
    int rc = scan_u32(S.kcnt, S.kstart, tot, S.scan_tmp, s);
    if (rc) return rc;
    sat_segments_kernel<<<grid_for(tot), 256, 0, s>>>(n, tot, S.kcnt, S.kstart, S.seg_start,
                                                      S.seg_len, S.seg_node, S.seg_tree, S.nseg,
                                                      tiny_max, S.big_min, S.big_list, tot);
    note_launch();
    sat_scatter_kernel<<<grid_for(tot), 256, 0, s>>>(n, tot, S.node_of, S.kcnt, S.kstart,
                                                     S.item_pt);
    note_launch();
    FG_CUDA(cudaGetLastError());
    uint32_t cnts[7] = {0, 0, 0, 0, 0, 0, 0};
    FG_CUDA(cudaMemcpyAsync(cnts, S.nseg, sizeof(cnts), cudaMemcpyDeviceToHost, s));
    FG_CUDA(cudaStreamSynchronize(s));
    if (cnts[2]) {
      set_error(3, "SAT: a point was assigned to an invalid node");
      return 3;
    }
    if (cnts[4]) {
      set_error(5, "SAT: a tensor-core assignment timed out waiting for its products");
      return 5;
    }
    const uint32_t ntiny = cnts[0], nbig = cnts[1], nsmall = cnts[3];
    if (ntiny == 0 && nsmall == 0 && nbig == 0) return 0;
    if (nsmall) {
      a.seg_off = tot - nsmall;
      kern<<<nsmall, SAT_NW * 32, smem, s>>>(a);
      note_launch();
      assign_all(nullptr, nsmall, cnts[5]);
      FG_CUDA(cudaGetLastError());
    }
    if (ntiny) {
      tinyk<<<ntiny, TINY_NW * 32, smem_t, s>>>(at);
      note_launch();
      FG_CUDA(cudaGetLastError());
    }
    if (nbig) {
      SatBigArgs B;
      B.s = a;
      B.big = S.big_list;
      B.kcount = S.big_kcount;
      uint64_t* kb[3] = {S.big_keys, S.big_keys + nbig, S.big_keys + 2 * nbig};
      uint32_t* lb[3] = {S.big_lens, S.big_lens + nbig, S.big_lens + 2 * nbig};
      uint64_t* lists[2] = {a.lst0, a.lst1};
      FG_CUDA(cudaMemsetAsync(S.big_keys, 0xFF, 3 * nbig * sizeof(uint64_t), s));
      FG_CUDA(cudaMemsetAsync(S.big_lens, 0, 3 * nbig * sizeof(uint32_t), s));
      FG_CUDA(cudaMemsetAsync(S.big_kcount, 0, nbig * sizeof(uint32_t), s));
      const unsigned gx = (unsigned)((n + BIG_TILE - 1) / BIG_TILE);
      unsigned gx1 = (unsigned)((n + STEP_TILE - 1) / STEP_TILE);  // open lists only shrink
      int r = 0, par = 0;  // kb[r], lb[r], lists[par]: the current step's state
      // grid.y is limited to 65535: big nodes are covered in chunks
      auto launch_all = [&](int mode, unsigned gxm) {
        B.cur = kb[r];
        B.nxt = kb[(r + 1) % 3];
        B.clr = kb[(r + 2) % 3];
        B.curlen = lb[r];
        B.nxtlen = lb[(r + 1) % 3];
        B.clrlen = lb[(r + 2) % 3];
        B.lin = lists[par];
        B.lout = lists[par ^ 1];
        for (uint32_t y0 = 0; y0 < nbig; y0 += 65535u) {
          B.y_off = (int32_t)y0;
          const dim3 grid(gxm, std::min<uint32_t>(65535u, nbig - y0));
          bigk<<<grid, BIG_NW * 32, smem, s>>>(B, mode);
          note_launch();
        }
      };
      launch_all(0, gx);
      FG_CUDA(cudaGetLastError());
      hkeys.resize(nbig);
      hlens.resize(nbig);
      // tiled selection steps while some open list is long
      bool short_lists = false;
      for (int64_t it = 0; it <= n && !short_lists;) {
        for (int j = 0; j < 4; ++j, ++it) {
          launch_all(1, gx1);
          r = (r + 1) % 3;
          par ^= 1;
        }
        FG_CUDA(cudaGetLastError());
        FG_CUDA(cudaMemcpyAsync(hkeys.data(), kb[r], nbig * sizeof(uint64_t),
                                cudaMemcpyDeviceToHost, s));
        FG_CUDA(cudaMemcpyAsync(hlens.data(), lb[r], nbig * sizeof(uint32_t),
                                cudaMemcpyDeviceToHost, s));
        FG_CUDA(cudaStreamSynchronize(s));
        short_lists = true;
        uint32_t max_len = 1;
        for (uint32_t i = 0; i < nbig; ++i) {
          short_lists &= (hkeys[i] == PAD || hlens[i] <= (uint32_t)S.finish_len);
          if (hkeys[i] != PAD) max_len = std::max(max_len, hlens[i]);
        }
        gx1 = (max_len + STEP_TILE - 1) / STEP_TILE;
      }
      if (!short_lists) {
        set_error(1, "SAT child selection did not terminate");
        return 1;
      }
      launch_all(3, 1);
      assign_all(S.big_list, nbig, cnts[6]);
      FG_CUDA(cudaGetLastError());
    }
  }
  set_error(1, "SAT construction did not terminate");
  return 1;
}

}  // namespace fg
