// Float32 distances from a Gram matrix computed on the tensor cores, with the
// error bound that says when such a value decides a comparison, and the
// canonical float32 distance of two staged rows for the comparisons it does
// not decide.
//
// Rows are staged as float32 words in the canonical K-major operand layout of
// tcgen05 without swizzle: 16-byte chunk q of row r sits in the core matrix of
// rows r/8 (8 rows x 16 bytes), core matrices 128 bytes apart along K and
// 128 * NQ bytes apart along the rows, NQ the chunk count rounded up to even
// (a kind::tf32 MMA consumes K = 8 elements, two chunks).  The MMA reads the
// same words as TF32 (low mantissa bits ignored).
//
// Error bound.  For rows x, y (d elements, D = 4 NQ after padding) the
// TF32 Gram value G~ differs from the exact dot product by at most
// (2.01 u + D 2^-22) |x||y| with u = 2^-10 (inputs cut to 10 mantissa bits,
// float32 accumulation in any order and rounding mode), and the canonical
// float32 distance from the exact one by at most D 2^-24 times the sum of the
// absolute terms plus its last rounding.  With h = (|x|^2 + |y|^2)/2 >= |x||y|
// and s = |x|^2 + |y|^2 (norms summed in float32 in any order):
//   angular  delta~ = 1 - G~,               |delta~ - delta| <= e1 h + e0,
//            e1 = 2 (2.01 u + (1.25 D + 1) 2^-22),  e0 = 2 * 2^-22;
//   L2       delta~ = s - 2 G~,             |delta~ - delta| <= e1 s,
//            e1 = 2 (2.01 u + (1.75 D + 2) 2^-22);
// the leading 2 is a safety factor that also absorbs the rounding of the
// bound's own arithmetic.
#pragma once

#include <cmath>

#include "common.cuh"
#include "tc.cuh"

namespace fg {

__host__ __device__ inline int tcp_nq(int nchunks) { return (nchunks + 1) & ~1; }

// Index of chunk q of staged row r.
__device__ __forceinline__ int tcp_at(int r, int q, int NQ) {
  return (r >> 3) * 8 * NQ + q * 8 + (r & 7);
}

// Chunk q of a float32 row for staging: zero past the row's d elements.
__device__ __forceinline__ uint4 tc_chunk(const char* __restrict__ row, int q, int nch, int d) {
  uint4 v = make_uint4(0u, 0u, 0u, 0u);
  if (q < nch) {
    v = __ldg(reinterpret_cast<const uint4*>(row) + q);
    const int rem = d - 4 * q;
    if (rem < 4) v.w = 0u;
    if (rem < 3) v.z = 0u;
    if (rem < 2) v.y = 0u;
  }
  return v;
}

// Stage a float32 row as staged row r, one thread, 16 chunks in flight at a
// time (row == nullptr: zeros).
__device__ __forceinline__ void tc_stage_row(uint4* C, int r, const char* __restrict__ row,
                                             int NQ, int nch, int d) {
  for (int q0 = 0; q0 < NQ; q0 += 16) {
    uint4 v[16];
#pragma unroll
    for (int u = 0; u < 16; ++u)
      v[u] = (row && q0 + u < NQ) ? tc_chunk(row, q0 + u, nch, d) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
    for (int u = 0; u < 16; ++u)
      if (q0 + u < NQ) C[tcp_at(r, q0 + u, NQ)] = v[u];
  }
}

// Squared norm of staged row r (float32, any order).
__device__ __forceinline__ float tc_norm2(const uint4* C, int r, int NQ, int nch) {
  float sq = 0.0f;
  for (int q = 0; q < nch; ++q) {
    const uint4 v = C[tcp_at(r, q, NQ)];
    sq = fmaf(__uint_as_float(v.x), __uint_as_float(v.x), sq);
    sq = fmaf(__uint_as_float(v.y), __uint_as_float(v.y), sq);
    sq = fmaf(__uint_as_float(v.z), __uint_as_float(v.z), sq);
    sq = fmaf(__uint_as_float(v.w), __uint_as_float(v.w), sq);
  }
  return sq;
}

// Approximate distance from a Gram value and its error bound.
template <int METRIC>
__device__ __forceinline__ void tc_approx(float g, float ni, float nj, float e1, float e0,
                                          float* dt, float* eps) {
  if constexpr (METRIC == ANGULAR_F32) {
    *dt = 1.0f - g;
    *eps = e1 * 0.5f * (ni + nj) + e0;
  } else {
    *dt = (ni + nj) - 2.0f * g;
    *eps = e1 * (ni + nj) + e0;
  }
}

inline void tc_error_bound(int metric, int nchunks, float* e1, float* e0) {
  const double D = 4.0 * tcp_nq(nchunks);
  const double u = std::ldexp(1.0, -10), u22 = std::ldexp(1.0, -22);
  if (metric == ANGULAR_F32) {
    *e1 = (float)(2.0 * (2.01 * u + (1.25 * D + 1.0) * u22));
    *e0 = (float)(2.0 * u22);
  } else {
    *e1 = (float)(2.0 * (2.01 * u + (1.75 * D + 2.0) * u22));
    *e0 = 0.0f;
  }
}

// Canonical float32 distance of staged rows (A, ra) and (B, rb), one thread:
// virtual lane l (of G) sums elements 128k + 4l + c, k < K, c < 4, by fused
// multiply-adds (L2: of the rounded difference squared), then the lanes are
// added pairwise, lane l with lane l + s for s = G/2 ... 1 -- the order of the
// lane-group kernels, so the value is the same bit for bit.
template <int METRIC, int G, int K>
__device__ float canon_dist_thread(const uint4* A, int ra, const uint4* B, int rb, int NQ,
                                   int nch, int d) {
  float v[G];
#pragma unroll
  for (int l = 0; l < G; ++l) {
    float acc = 0.0f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int c = 32 * k + l;
      if (c < nch) {
        const uint4 xa = A[tcp_at(ra, c, NQ)], ya = B[tcp_at(rb, c, NQ)];
        const float x[4] = {__uint_as_float(xa.x), __uint_as_float(xa.y), __uint_as_float(xa.z),
                            __uint_as_float(xa.w)};
        const float y[4] = {__uint_as_float(ya.x), __uint_as_float(ya.y), __uint_as_float(ya.z),
                            __uint_as_float(ya.w)};
        const int nv = d - 4 * c;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          if (nv > e) {
            if constexpr (METRIC == ANGULAR_F32) {
              acc = __fmaf_rn(x[e], y[e], acc);
            } else {
              const float t = __fsub_rn(x[e], y[e]);
              acc = __fmaf_rn(t, t, acc);
            }
          }
        }
      }
    }
    v[l] = acc;
  }
#pragma unroll
  for (int sh = G / 2; sh >= 1; sh >>= 1) {
#pragma unroll
    for (int l = 0; l < sh; ++l) v[l] = __fadd_rn(v[l], v[l + sh]);
  }
  if constexpr (METRIC == ANGULAR_F32) return __fsub_rn(1.0f, v[0]);
  return v[0];
}

}  // namespace fg
