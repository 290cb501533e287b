// Device helpers shared by the FGraft kernels (sm_103a).
//
// Canonical distance.  The paper computes Euclidean distances on float32
// vectors, angular data being L2-normalised (Section 2).  Bit-exact results
// need one summation order; the library fixes it as 32 virtual lanes, lane l
// owning elements j = 128k + 4l + c (k = 0,1,..; c = 0..3) in that order with
// acc = fma(t, t, acc), t = x_j - y_j rounded first (acc = fma(x_j, y_j, acc)
// for the angular inner product), followed by the xor butterfly
// +16, +8, +4, +2, +1.  A group of G lanes (G a power of two covering the
// non-empty virtual lanes) reproduces it bit for bit, because the virtual
// lanes it drops hold +0.0 and adding +0.0 to a non-negative-zero partial is
// exact.  uint8 vectors use exact integer arithmetic.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace fg {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr uint32_t EMPTY = 0xFFFFFFFFu;
constexpr uint64_t PAD = ~0ull;

enum Metric : int { L2_F32 = 0, ANGULAR_F32 = 1, L2_U8 = 2 };

// Monotone map of a float onto uint32 (total order for finite values and inf).
__device__ __forceinline__ uint32_t fkey(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(uint32_t k) {
  uint32_t u = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
  return __uint_as_float(u);
}
// (delta, id) packed so that integer order is the (delta, id) order; bit 0 is
// free for a flag (an entry is never compared with itself).
__device__ __forceinline__ uint64_t make_key(float d, int32_t id) {
  return ((uint64_t)fkey(d) << 32) | ((uint64_t)(uint32_t)id << 1);
}
__device__ __forceinline__ int32_t key_id(uint64_t k) { return (int32_t)((uint32_t)k >> 1); }
__device__ __forceinline__ float key_dist(uint64_t k) { return fkey_inv((uint32_t)(k >> 32)); }

__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }
__device__ __forceinline__ uint64_t umax64(uint64_t a, uint64_t b) { return a < b ? b : a; }

// ---------------------------------------------------------------------------
// Vector access.  A row is cut into 16-byte chunks; lane gl of a G-lane group
// holds chunks k*G + gl, k < K.  For float32 with G < 32, K is 1, so the lane
// holds elements 4gl..4gl+3 exactly as virtual lane gl does; for G = 32 the
// chunk k*32 + l covers elements 128k + 4l + c.
// ---------------------------------------------------------------------------
template <int METRIC>
struct ElemBytes {
  static constexpr int value = METRIC == L2_U8 ? 1 : 4;
};

template <int METRIC, int G, int K>
__device__ __forceinline__ void load_chunks(const char* __restrict__ row, int nchunks, int gl,
                                            uint4 (&v)[K]) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
    int c = k * G + gl;
    if (c < nchunks) {
      v[k] = __ldg(reinterpret_cast<const uint4*>(row) + c);
    } else {
      v[k] = make_uint4(0u, 0u, 0u, 0u);
    }
  }
}

// Per-lane partial of the canonical distance.  d = vector length.
template <int METRIC, int G, int K>
__device__ __forceinline__ float partial(const uint4 (&q)[K], const uint4 (&v)[K], int d, int gl) {
  if constexpr (METRIC == L2_U8) {
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      int c = k * G + gl;
      int nb = d - 16 * c;  // valid bytes in this chunk
      uint32_t a[4] = {q[k].x, q[k].y, q[k].z, q[k].w};
      uint32_t b[4] = {v[k].x, v[k].y, v[k].z, v[k].w};
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        int vb = nb - 4 * w;
        uint32_t m = vb >= 4 ? 0xFFFFFFFFu : (vb <= 0 ? 0u : (0xFFFFFFFFu >> (8 * (4 - vb))));
        uint32_t diff = __vabsdiffu4(a[w] & m, b[w] & m);
        s = __dp4a(diff, diff, s);
      }
    }
    return __uint_as_float(s);  // carried as raw bits; reduced as integers
  } else {
    float acc = 0.0f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      int c = k * G + gl;
      int nv = d - 4 * c;  // valid elements in this chunk
      float x[4] = {__uint_as_float(q[k].x), __uint_as_float(q[k].y), __uint_as_float(q[k].z),
                    __uint_as_float(q[k].w)};
      float y[4] = {__uint_as_float(v[k].x), __uint_as_float(v[k].y), __uint_as_float(v[k].z),
                    __uint_as_float(v[k].w)};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (nv > e) {
          if constexpr (METRIC == ANGULAR_F32) {
            acc = __fmaf_rn(x[e], y[e], acc);
          } else {
            float t = __fsub_rn(x[e], y[e]);
            acc = __fmaf_rn(t, t, acc);
          }
        }
      }
    }
    return acc;
  }
}

// Combine the partials of a G-lane group; every lane of the group gets the
// distance.
template <int METRIC, int G>
__device__ __forceinline__ float group_reduce(float p) {
  if constexpr (METRIC == L2_U8) {
    uint32_t s = __float_as_uint(p);
#pragma unroll
    for (int off = G / 2; off >= 1; off >>= 1) s += __shfl_xor_sync(FULL, s, off);
    return __uint2float_rn(s);
  } else {
    float v = p;
#pragma unroll
    for (int off = G / 2; off >= 1; off >>= 1) v = __fadd_rn(v, __shfl_xor_sync(FULL, v, off));
    if constexpr (METRIC == ANGULAR_F32) return __fsub_rn(1.0f, v);
    return v;
  }
}

// ---------------------------------------------------------------------------
// Lane-group distance.  A vector is evaluated by P physical lanes; lane j of
// the group holds the virtual lanes l = j, j+P, j+2P, .. (V/P of them, V = G
// the virtual lanes in use) and, of each, the chunks 32k + l, k < K.  The
// per-virtual-lane sums are exactly the canonical ones; the butterfly levels
// s >= P combine virtual lanes held by the same physical lane (in registers,
// v[i] + v[i + s/P], the operand order of the canonical tree) and the levels
// s < P use shuffles inside the group.  Result: bit-identical to the
// canonical order at a fraction of the shuffles.
// ---------------------------------------------------------------------------
// One 16-byte chunk of two float32 rows into a virtual lane's accumulator,
// elements in order by fused multiply-adds (L2: of the rounded difference
// squared).  The partial form takes only the first nv < 4 elements.
template <int METRIC>
__device__ __forceinline__ float chunk_acc(const uint4 a, const uint4 b, float acc) {
  const float x[4] = {__uint_as_float(a.x), __uint_as_float(a.y), __uint_as_float(a.z),
                      __uint_as_float(a.w)};
  const float y[4] = {__uint_as_float(b.x), __uint_as_float(b.y), __uint_as_float(b.z),
                      __uint_as_float(b.w)};
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    if constexpr (METRIC == ANGULAR_F32) {
      acc = __fmaf_rn(x[e], y[e], acc);
    } else {
      const float t = __fsub_rn(x[e], y[e]);
      acc = __fmaf_rn(t, t, acc);
    }
  }
  return acc;
}
template <int METRIC>
__device__ __forceinline__ float chunk_acc_partial(const uint4 a, const uint4 b, float acc,
                                                  int nv) {
  const float x[4] = {__uint_as_float(a.x), __uint_as_float(a.y), __uint_as_float(a.z),
                      __uint_as_float(a.w)};
  const float y[4] = {__uint_as_float(b.x), __uint_as_float(b.y), __uint_as_float(b.z),
                      __uint_as_float(b.w)};
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    if (e >= nv) break;
    if constexpr (METRIC == ANGULAR_F32) {
      acc = __fmaf_rn(x[e], y[e], acc);
    } else {
      const float t = __fsub_rn(x[e], y[e]);
      acc = __fmaf_rn(t, t, acc);
    }
  }
  return acc;
}

template <int G, int K>
struct Lanes {
  static constexpr int P = G <= 8 ? 1 : (G == 16 ? 2 : 4 * K);  // lanes per vector
  static constexpr int VL = G / P;                               // virtual lanes per lane
  static constexpr int CPW = 32 / P;                             // vectors per warp step
  static constexpr int SLOTS = VL * K;                           // 16-byte chunks per lane
  static constexpr int U = SLOTS >= 8 ? 1 : 8 / SLOTS;           // vectors in flight per group
  static constexpr int UW = CPW * U > 32 ? 32 / CPW : U;          // same, for at most 32 vectors
};

// Copy a row's chunks into shared memory (whole warp), then sync the warp.
__device__ __forceinline__ void stage_row(uint4* dst, const char* __restrict__ row, int nchunks,
                                          int lane) {
  for (int c = lane; c < nchunks; c += 32) dst[c] = __ldg(reinterpret_cast<const uint4*>(row) + c);
  __syncwarp();
}

// One 16-byte chunk of a candidate row.  Normally through the read-only
// path, so that a row one search of an SM has just loaded is served from L1
// to the others (the SM's resident searches share repeated targets).  A
// measurement build with -DFGRAFT_GATHER_NO_L1 caches the rows in L2 only,
// to measure what that sharing is worth.
__device__ __forceinline__ uint4 load_row_chunk(const uint4* p) {
#ifdef FGRAFT_GATHER_NO_L1
  uint4 v;
  // not volatile: the rows are read-only, the loads may be scheduled freely
  asm("ld.global.cg.v4.u32 {%0, %1, %2, %3}, [%4];"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
      : "l"(p));
  return v;
#else
  return __ldg(p);
#endif
}

// The chunks lane j of a group needs from row; indices past the row are
// clamped to its last chunk (the values are masked out later), so every load
// is issued without a branch.
template <int G, int K>
__device__ __forceinline__ void load_slots(const char* __restrict__ row, int nchunks, int j,
                                           uint4 (&y)[Lanes<G, K>::VL][K]) {
  using L = Lanes<G, K>;
#pragma unroll
  for (int i = 0; i < L::VL; ++i) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int c = min(32 * k + j + L::P * i, nchunks - 1);
      y[i][k] = load_row_chunk(reinterpret_cast<const uint4*>(row) + c);
    }
  }
}

// The same chunks from a row staged in shared memory.
template <int G, int K>
__device__ __forceinline__ void load_slots_smem(const uint4* row, int nchunks, int j,
                                                uint4 (&y)[Lanes<G, K>::VL][K]) {
  using L = Lanes<G, K>;
#pragma unroll
  for (int i = 0; i < L::VL; ++i) {
#pragma unroll
    for (int k = 0; k < K; ++k) y[i][k] = row[min(32 * k + j + L::P * i, nchunks - 1)];
  }
}

// Canonical distance between the staged vector qs (shared memory) and the
// chunks y of one group member; every lane of the group returns it.
// The same distance with the first vector's chunks in registers too (loaded
// by load_slots / load_slots_smem with the same lane mapping).
template <int METRIC, int G, int K>
__device__ __forceinline__ float regs_dist(const uint4 (&xq)[Lanes<G, K>::VL][K],
                                           const uint4 (&y)[Lanes<G, K>::VL][K], int nchunks,
                                           int d, int j, unsigned mask) {
  using L = Lanes<G, K>;
  if constexpr (METRIC == L2_U8) {
    uint32_t t = 0;
#pragma unroll
    for (int i = 0; i < L::VL; ++i) {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int c = 32 * k + j + L::P * i;
        if (c < nchunks) {
          const int nb = d - 16 * c;
          const uint32_t a[4] = {xq[i][k].x, xq[i][k].y, xq[i][k].z, xq[i][k].w};
          const uint32_t b[4] = {y[i][k].x, y[i][k].y, y[i][k].z, y[i][k].w};
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            const int vb = nb - 4 * w;
            const uint32_t m =
                vb >= 4 ? 0xFFFFFFFFu : (vb <= 0 ? 0u : (0xFFFFFFFFu >> (8 * (4 - vb))));
            const uint32_t df = __vabsdiffu4(a[w] & m, b[w] & m);
            t = __dp4a(df, df, t);
          }
        }
      }
    }
#pragma unroll
    for (int off = L::P / 2; off >= 1; off >>= 1) t += __shfl_xor_sync(mask, t, off);
    return __uint2float_rn(t);
  } else {
    const int nfull = d >> 2;
    float v[L::VL];
#pragma unroll
    for (int i = 0; i < L::VL; ++i) {
      float acc = 0.0f;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int c = 32 * k + j + L::P * i;
        if (c < nfull)
          acc = chunk_acc<METRIC>(xq[i][k], y[i][k], acc);
        else if (c < nchunks)
          acc = chunk_acc_partial<METRIC>(xq[i][k], y[i][k], acc, d - 4 * c);
      }
      v[i] = acc;
    }
#pragma unroll
    for (int s = G / 2; s >= L::P; s >>= 1) {
#pragma unroll
      for (int i = 0; i < s / L::P; ++i) v[i] = __fadd_rn(v[i], v[i + s / L::P]);
    }
    float r = v[0];
#pragma unroll
    for (int off = L::P / 2; off >= 1; off >>= 1) r = __fadd_rn(r, __shfl_xor_sync(mask, r, off));
    if constexpr (METRIC == ANGULAR_F32) return __fsub_rn(1.0f, r);
    return r;
  }
}

// `mask` names the lanes that execute the call together: the whole warp, or
// only the calling P-lane group when groups run different trip counts.
template <int METRIC, int G, int K>
__device__ __forceinline__ float slots_dist(const uint4* qs, const uint4 (&y)[Lanes<G, K>::VL][K],
                                            int nchunks, int d, int j, unsigned mask = FULL) {
  using L = Lanes<G, K>;
  if constexpr (METRIC == L2_U8) {
    uint32_t v[L::VL];
#pragma unroll
    for (int i = 0; i < L::VL; ++i) {
      uint32_t acc = 0;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int c = 32 * k + j + L::P * i;
        if (c < nchunks) {
          const uint4 x = qs[c];
          const int nb = d - 16 * c;
          const uint32_t a[4] = {x.x, x.y, x.z, x.w};
          const uint32_t b[4] = {y[i][k].x, y[i][k].y, y[i][k].z, y[i][k].w};
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            const int vb = nb - 4 * w;
            const uint32_t m =
                vb >= 4 ? 0xFFFFFFFFu : (vb <= 0 ? 0u : (0xFFFFFFFFu >> (8 * (4 - vb))));
            const uint32_t df = __vabsdiffu4(a[w] & m, b[w] & m);
            acc = __dp4a(df, df, acc);
          }
        }
      }
      v[i] = acc;
    }
    uint32_t t = 0;
#pragma unroll
    for (int i = 0; i < L::VL; ++i) t += v[i];
#pragma unroll
    for (int off = L::P / 2; off >= 1; off >>= 1) t += __shfl_xor_sync(mask, t, off);
    return __uint2float_rn(t);
  } else {
    // full chunks (4 elements inside the row) need no element test; a row
    // whose d is not a multiple of 4 has one partial chunk, the last chunk of
    // its virtual lane, handled apart
    const int nfull = d >> 2;
    float v[L::VL];
#pragma unroll
    for (int i = 0; i < L::VL; ++i) {
      float acc = 0.0f;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int c = 32 * k + j + L::P * i;
        if (c < nfull) {
          const uint4 xq = qs[c];
          acc = chunk_acc<METRIC>(xq, y[i][k], acc);
        } else if (c < nchunks) {
          acc = chunk_acc_partial<METRIC>(qs[c], y[i][k], acc, d - 4 * c);
        }
      }
      v[i] = acc;
    }
    // butterfly levels inside the lane: virtual lanes j + P*i and j + P*i + s
#pragma unroll
    for (int s = G / 2; s >= L::P; s >>= 1) {
#pragma unroll
      for (int i = 0; i < s / L::P; ++i) v[i] = __fadd_rn(v[i], v[i + s / L::P]);
    }
    float r = v[0];
#pragma unroll
    for (int off = L::P / 2; off >= 1; off >>= 1) r = __fadd_rn(r, __shfl_xor_sync(mask, r, off));
    if constexpr (METRIC == ANGULAR_F32) return __fsub_rn(1.0f, r);
    return r;
  }
}

// ---------------------------------------------------------------------------
// Warp bitonic networks on 64-bit keys.
// ---------------------------------------------------------------------------
// Sort one key per lane ascending across the warp.
__device__ __forceinline__ uint64_t warp_sort32(uint64_t x, int lane) {
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      uint64_t o = __shfl_xor_sync(FULL, x, j);
      bool up = (lane & k) == 0;
      bool lower = (lane & j) == 0;
      x = (lower == up) ? umin64(x, o) : umax64(x, o);
    }
  }
  return x;
}

// A register list of N = 32*S keys, entry i at slot i/32 of lane i%32, that
// is bitonic, is sorted ascending.
template <int S>
__device__ __forceinline__ void bitonic_merge_regs(uint64_t (&a)[S], int lane) {
#pragma unroll
  for (int sj = S / 2; sj >= 1; sj >>= 1) {
#pragma unroll
    for (int s = 0; s < S; ++s) {
      if ((s & sj) == 0) {
        uint64_t x = a[s], y = a[s + sj];
        a[s] = umin64(x, y);
        a[s + sj] = umax64(x, y);
      }
    }
  }
#pragma unroll
  for (int j = 16; j >= 1; j >>= 1) {
#pragma unroll
    for (int s = 0; s < S; ++s) {
      uint64_t o = __shfl_xor_sync(FULL, a[s], j);
      a[s] = (lane & j) ? umax64(a[s], o) : umin64(a[s], o);
    }
  }
}

// pool := the ef smallest of pool U {cand}, pool sorted ascending in a list of
// N = 32*S >= ef slots (entries past ef are PAD), cand one key per lane
// (PAD = none).  Keys must be distinct.
template <int S>
__device__ __forceinline__ void merge_into_pool(uint64_t (&pool)[S], uint64_t cand, int ef,
                                                int lane) {
  uint64_t worst = PAD;
#pragma unroll
  for (int s = 0; s < S; ++s)
    if (s == (ef - 1) / 32) worst = __shfl_sync(FULL, pool[s], (ef - 1) % 32);
  if (cand >= worst) cand = PAD;
  unsigned bal = __ballot_sync(FULL, cand != PAD);
  if (bal == 0) return;
  if (__popc(bal) <= 4) {
    // few survivors: insert one at a time (rank by ballots, shift by one)
    while (bal) {
      const int src = __ffs(bal) - 1;
      bal &= bal - 1u;
      const uint64_t c = __shfl_sync(FULL, cand, src);
      int rank = 0;
#pragma unroll
      for (int s = 0; s < S; ++s) rank += __popc(__ballot_sync(FULL, pool[s] < c));
      uint64_t prevlast = PAD;
#pragma unroll
      for (int s = 0; s < S; ++s) {
        uint64_t up = __shfl_up_sync(FULL, pool[s], 1);
        const uint64_t last = __shfl_sync(FULL, pool[s], 31);
        if (lane == 0) up = prevlast;
        const int i = s * 32 + lane;
        pool[s] = i < rank ? pool[s] : (i == rank ? c : up);
        prevlast = last;
      }
    }
#pragma unroll
    for (int s = 0; s < S; ++s)
      if (s * 32 + lane >= ef) pool[s] = PAD;
    return;
  }
  cand = warp_sort32(cand, lane);
  uint64_t rev = __shfl_sync(FULL, cand, 31 - lane);
  pool[S - 1] = umin64(pool[S - 1], rev);
  bitonic_merge_regs<S>(pool, lane);
#pragma unroll
  for (int s = 0; s < S; ++s)
    if (s * 32 + lane >= ef) pool[s] = PAD;
}

// Ascending bitonic sort of N keys (N a power of two) in shared or global
// memory by one warp.
__device__ __forceinline__ void warp_sort_mem(uint64_t* a, int N, int lane) {
  for (int k = 2; k <= N; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < N / 2; i += 32) {
        int lo = ((i & ~(j - 1)) << 1) | (i & (j - 1));
        int hi = lo + j;
        bool asc = (lo & k) == 0;
        uint64_t x = a[lo], y = a[hi];
        if ((x > y) == asc) {
          a[lo] = y;
          a[hi] = x;
        }
      }
      __syncwarp();
    }
  }
}

// Asynchronous prefetch of `bytes` (a multiple of 16, 16-byte aligned) into
// the L2 cache: no registers, no completion to wait for.
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Exact visited set: open addressing over 4-slot buckets, linear probing by
// bucket.  Returns true when id was absent and is now inserted.  Lanes of a
// warp may insert concurrently (a duplicate resolves through atomicCAS).  The
// caller keeps the load below capacity, so an empty slot is always reachable.
__device__ __forceinline__ bool hash_insert(uint32_t* h, uint32_t mask_buckets, uint32_t id) {
  uint32_t bkt = (id * 2654435761u) & mask_buckets;
  for (uint32_t probe = 0; probe <= mask_buckets;) {
    uint32_t* b = h + 4 * bkt;
    uint4 s;
    asm volatile("ld.volatile.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(s.x), "=r"(s.y), "=r"(s.z), "=r"(s.w)
                 : "l"(b));
    if (s.x == id || s.y == id || s.z == id || s.w == id) return false;
    int j = s.x == EMPTY ? 0 : s.y == EMPTY ? 1 : s.z == EMPTY ? 2 : s.w == EMPTY ? 3 : -1;
    if (j < 0) {
      bkt = (bkt + 1) & mask_buckets;
      ++probe;
      continue;
    }
    uint32_t old = atomicCAS(b + j, EMPTY, id);
    if (old == EMPTY) return true;
    if (old == id) return false;
    // the slot went to another id: read the same bucket again
  }
  return false;
}

// Position of the r-th (0-based) set bit of x; r < popc(x).
__device__ __forceinline__ int nth_set_bit(uint32_t x, int r) {
  int base = 0;
#pragma unroll
  for (int w = 16; w >= 1; w >>= 1) {
    int c = __popc((x >> base) & ((1u << w) - 1u));
    if (r >= c) {
      r -= c;
      base += w;
    }
  }
  return base;
}

// Candidates evaluated per lane group per unrolled step: enough independent
// 16-byte loads in flight, at most 32 candidates per warp step.
template <int G, int K>
struct Unroll {
  static constexpr int GPW = 32 / G;
  static constexpr int A = (32 / GPW) < (8 / K) ? (32 / GPW) : (8 / K);
  static constexpr int value = A < 1 ? 1 : A;
};

}  // namespace fg
