// Warp-level row operations shared by the final-graph and list-prune
// kernels: evaluate a candidate list into (delta, id) keys, sort and
// de-duplicate it, and run the occlusion prune of Section 3 on the sorted
// keys.  A row works in one key buffer (shared memory, or a global scratch
// slice for rows too long for shared memory).
#pragma once
#include "common.cuh"

namespace fg {

__device__ __forceinline__ int pow2_dev(int v) {
  int p = 32;
  while (p < v) p <<= 1;
  return p;
}

struct RowVec {
  const char* X;
  int64_t ld_bytes;
  int32_t d;
  int32_t nchunks;
};

// keys[at + i] = key(delta(u, c_i), c_i) for the candidates c_0.. of two id
// segments (seg0[0..len0) then seg1[0..len1)); us = u's vector staged in
// shared memory.
template <int METRIC, int G, int K>
__device__ void eval_keys(const RowVec& V, const uint4* us, const int32_t* seg0, int len0,
                          const int32_t* seg1, int len1, uint64_t* keys, int at, int lane) {
  using L = Lanes<G, K>;
  const int g = lane / L::P, j = lane % L::P;
  const int len = len0 + len1;
  for (int base = 0; base < len; base += L::CPW * L::U) {
    uint4 y[L::U][L::VL][K];
    int32_t id[L::U];
#pragma unroll
    for (int u = 0; u < L::U; ++u) {
      const int i = base + u * L::CPW + g;
      id[u] = i < len0 ? seg0[i] : (i < len ? seg1[i - len0] : -1);
      const int32_t ld_id = id[u] >= 0 ? id[u] : (len0 > 0 ? seg0[0] : seg1[0]);
      load_slots<G, K>(V.X + (int64_t)ld_id * V.ld_bytes, V.nchunks, j, y[u]);
    }
#pragma unroll
    for (int u = 0; u < L::U; ++u) {
      const float dd = slots_dist<METRIC, G, K>(us, y[u], V.nchunks, V.d, j);
      const int i = base + u * L::CPW + g;
      if (i < len && j == 0) keys[at + i] = make_key(dd, id[u]);
    }
  }
  __syncwarp();
}

// keys[0..m) hold distinct ids (id << 1); each becomes the key
// (delta(us, id), id), two candidates per lane group in flight.
template <int METRIC, int G, int K>
__device__ void eval_keys_inplace(const RowVec& V, const uint4* us, uint64_t* keys, int m,
                                  int lane) {
  using L = Lanes<G, K>;
  constexpr int NU = 2;
  const int g = lane / L::P, j = lane % L::P;
  for (int base = 0; base < m; base += L::CPW * NU) {
    uint4 y[NU][L::VL][K];
    int32_t id[NU];
#pragma unroll
    for (int u = 0; u < NU; ++u) {
      const int i = min(base + u * L::CPW + g, m - 1);
      id[u] = key_id(keys[i]);
      load_slots<G, K>(V.X + (int64_t)id[u] * V.ld_bytes, V.nchunks, j, y[u]);
    }
#pragma unroll
    for (int u = 0; u < NU; ++u) {
      const float dd = slots_dist<METRIC, G, K>(us, y[u], V.nchunks, V.d, j);
      const int i = base + u * L::CPW + g;
      if (i < m && j == 0) keys[i] = make_key(dd, id[u]);
    }
  }
  __syncwarp();
}

// Sorts keys[0..len) (padding to a power of two >= 32 with PAD, which must
// fit the buffer) and removes repeated keys; returns the distinct count.
__device__ inline int sort_unique(uint64_t* keys, int len, int lane) {
  int N2 = 32;
  while (N2 < len) N2 <<= 1;
  for (int i = len + lane; i < N2; i += 32) keys[i] = PAD;
  __syncwarp();
  warp_sort_mem(keys, N2, lane);
  int outn = 0;
  for (int base = 0; base < len; base += 32) {
    int i = base + lane;
    uint64_t k = i < len ? keys[i] : PAD;
    uint64_t prev = (i > 0 && i - 1 < len) ? keys[i - 1] : PAD;
    bool keep = i < len && (i == 0 || k != prev);
    unsigned m = __ballot_sync(FULL, keep);
    __syncwarp();
    if (keep) keys[outn + __popc(m & ((1u << lane) - 1u))] = k;
    outn += __popc(m);
    __syncwarp();
  }
  return outn;
}

// Occlusion prune of keys[0..m) (sorted by (delta(p,.), id), p excluded):
// keep the first alive c*, remove every alive c after it with
// fl(alpha2 * delta(c*, c)) <= delta(p, c); stop at R kept.  On return
// keys[0..kept) hold the kept keys in keep order.  alive: (m+31)/32 words of
// scratch.  *evals accumulates the alive candidates examined.
template <int METRIC, int G, int K>
__device__ int prune_sorted(const RowVec& V, uint64_t* keys, int m, float alpha2, int R,
                            uint32_t* alive, uint4* cs, unsigned long long* evals, int lane) {
  using L = Lanes<G, K>;
  const int g = lane / L::P, j = lane % L::P;
  const int nw = (m + 31) / 32;
  for (int w = lane; w < nw; w += 32) alive[w] = (w * 32 + 32 <= m) ? FULL : ((1u << (m - w * 32)) - 1u);
  __syncwarp();
  int kept = 0, cur = -1;
  unsigned long long ev = 0;
  // kept positions are recorded by clearing alive and setting bit in the high
  // half of the scratch (alive + nw)
  uint32_t* keptm = alive + nw;
  for (int w = lane; w < nw; w += 32) keptm[w] = 0u;
  __syncwarp();
  while (kept < R) {
    int nxt = -1;
    for (int w = (cur + 1) / 32; w < nw && nxt < 0; ++w) {
      uint32_t bits = alive[w];
      if (w == (cur + 1) / 32) bits &= ~((1u << ((cur + 1) % 32)) - 1u);
      if (bits) nxt = w * 32 + __ffs(bits) - 1;
    }
    if (nxt < 0) break;
    cur = nxt;
    if (lane == 0) {
      alive[cur / 32] &= ~(1u << (cur % 32));
      keptm[cur / 32] |= 1u << (cur % 32);
    }
    ++kept;
    __syncwarp();
    if (kept == R) break;
    stage_row(cs, V.X + (int64_t)key_id(keys[cur]) * V.ld_bytes, V.nchunks, lane);
    for (int w = cur / 32; w < nw; ++w) {
      uint32_t bits = alive[w];
      if (w == cur / 32) bits &= ~((2u << (cur % 32)) - 1u);
      ev += (unsigned long long)__popc(bits);
      uint32_t kill = 0;
      while (bits) {
        const int nb = __popc(bits);
        uint4 y[L::UW][L::VL][K];
        int jj[L::UW];
#pragma unroll
        for (int u = 0; u < L::UW; ++u) {
          const int r = u * L::CPW + g;
          jj[u] = r < nb ? nth_set_bit(bits, r) : -1;
          const int e = w * 32 + (jj[u] >= 0 ? jj[u] : 0);
          load_slots<G, K>(V.X + (int64_t)key_id(keys[e]) * V.ld_bytes, V.nchunks, j, y[u]);
        }
#pragma unroll
        for (int u = 0; u < L::UW; ++u) {
          const float dd = slots_dist<METRIC, G, K>(cs, y[u], V.nchunks, V.d, j);
          if (jj[u] >= 0 && j == 0) {
            const float dp = key_dist(keys[w * 32 + jj[u]]);
            if (__fmul_rn(alpha2, dd) <= dp) kill |= 1u << jj[u];
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
      if (lane == 0) alive[w] &= ~kill;
      __syncwarp();
    }
  }
  // compact the kept keys to the front, in order
  int outn = 0;
  for (int base = 0; base < m; base += 32) {
    int i = base + lane;
    bool keep = i < m && ((keptm[i / 32] >> (i % 32)) & 1u);
    uint64_t k = keep ? keys[i] : PAD;
    unsigned msk = __ballot_sync(FULL, keep);
    __syncwarp();
    if (keep) keys[outn + __popc(msk & ((1u << lane) - 1u))] = k;
    outn += __popc(msk);
    __syncwarp();
  }
  *evals += ev;
  return outn;
}

// True (on every lane) when some keys[0..len) carries id v.
__device__ inline bool keys_contain(const uint64_t* keys, int len, int32_t v, int lane) {
  bool f = false;
  for (int base = 0; base < len; base += 32) {
    int i = base + lane;
    f |= __any_sync(FULL, i < len && key_id(keys[i]) == v);
  }
  return f;
}

}  // namespace fg
