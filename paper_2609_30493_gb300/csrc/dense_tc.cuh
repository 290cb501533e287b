// Shared layout and error bound of the tensor-core dense kernels: the
// dense-block ceiling (dense_tc.cu) and the exact k nearest neighbours over
// all points (knn_tc.cu).  Rows are rounded to BF16 (or E4M3 with a scale per
// row) by dt_prep_kernel and written as the shared-memory image the tensor
// cores read: K-major core matrices of 8 rows x 16 bytes, one 128 KB image
// per 128-byte K slice of 1024 rows.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "common.cuh"

namespace fg {

constexpr int DT_ROWS = 1024;        // rows of a block after padding
constexpr int DT_M = 128;            // rows per tile (one per TMEM lane)
constexpr int DT_NC = 256;           // columns per chunk (MMA N)
constexpr int DT_KB = 128;           // K bytes per slice (8 core matrices of 16 bytes)
constexpr int DT_STAGES = 3;
constexpr int DT_A_BYTES = DT_M * DT_KB;             // 16 KB
constexpr int DT_B_BYTES = DT_NC * DT_KB;            // 32 KB
constexpr int DT_STAGE_BYTES = DT_A_BYTES + DT_B_BYTES;
constexpr int DT_SLICE_IMG = DT_ROWS * DT_KB;        // 128 KB: one slice of the 1024 rows
constexpr int DT_EPI = 256;          // epilogue threads (warps 0..7)
constexpr int DT_THREADS = DT_EPI + 64;
constexpr int DT_NBIN = 32;
constexpr uint32_t DT_TMEM_COLS = 512;
constexpr uint32_t DT_FALLBACK = 0xFFFFFFFFu;  // candidate count: every valid column

// Byte offset of the 16-byte unit (row r, K byte kb) in a slice image: core
// matrix (r/8, kb/16) at (r/8)*1024 + (kb/16)*128, row r%8 at +16*(r%8).
__host__ __device__ constexpr uint32_t tile_off(int r, int kb) {
  return (uint32_t)((r >> 3) * 1024 + (kb >> 4) * 128 + (r & 7) * 16);
}

struct DtArgs {
  const char* X;
  int64_t ld_bytes;
  int32_t d;
  int32_t metric;
  int32_t fp8;   // 0: BF16, 1: E4M3 with a scale per row
  int32_t dpad;  // d rounded up to a whole slice (64 BF16 or 128 E4M3 elements)
  int32_t rowb;  // bytes of a rounded row
  int32_t nsl;   // slices per row (rowb / 128)
  const int32_t* block_ids;
  int64_t nb;
  int32_t bs;
  int32_t k;
  unsigned char* Xt;  // [nb][nsl][slice image]
  float4* rowA;       // [nb][1024] {|x|^2 centred, (1 - |x|^2)/2 raw (angular), scale, valid}
  float4* rowB;       // [nb][1024] {|x - q|, |q|, |x|^2 raw, 0}
  float* bst;         // [nb][8] {Mx, Rq, Qx, X2max, Cmax}: maxima over the block (>= 0)
  uint32_t* nvalid;   // [nb]
  uint16_t* cand;     // [nb][1024][1024] candidate columns of each row
  uint32_t* ccnt;     // [nb][1024] their number (DT_FALLBACK: every valid column)
  float* cdt;         // optional [nb][1024][1024]: approximate distance of each candidate
  float* reps;        // optional [nb][1024]: eps of each row
  float* rowmin;      // Gram-only mode: [nb * bs] smallest approximate distance per row
  uint32_t* err;      // [0] timeout flag, [8] and [9] error maxima (float bits)
  unsigned long long* pairs;     // valid ordered pairs over all blocks
  unsigned long long* reranked;  // pairs recomputed in the canonical order
  int32_t mode;       // 0: Gram and approximate distances only (per-row minimum), 1: filter
  int32_t errstat;    // keep approximate distances and eps for the float64 error check
  int32_t wait_polls;
  int32_t nocentre;   // 1: the rows are rounded as they are (mean taken as 0)
};


// Centres (unless nocentre), rounds and writes the tile images of every
// block, with the per-row norms and per-block maxima (defined in dense_tc.cu).
__global__ void dt_prep_kernel(const DtArgs a);

// eps of row i: a bound on |approximate - canonical float32| distance for
// every pair (i, j) of the block, from the rows' actual rounding residuals
// (Cauchy-Schwarz on the Gram error: r_i Qx + |x_i| Rq), the FP32
// accumulation over K = dpad products in any order, the float32 norms and
// the canonical distance's own rounding, times a safety factor of 2.
// ni: |x_i - mu|^2; ri = |x_i - q_i|; qi = |q_i|; x2i = |x_i|^2 (raw);
// Mx, Rq, Qx, X2m: the maxima of |x_j - mu|, r_j, |q_j| and |x_j|^2.
__device__ __forceinline__ float dt_row_eps(bool ang, int dpad, int d, float ni, float ri,
                                            float qi, float x2i, float Mx, float Rq, float Qx,
                                            float X2m) {
  const float u = 5.9604645e-8f;  // 2^-24
  const float Ai = sqrtf(ni);
  const float K = (float)dpad, dd = (float)d;
  const float gK = K * u / (1.0f - K * u), gd = (dd + 8.0f) * u;
  const float Eg = ri * Qx + Ai * Rq + (gK + 3.0f * u) * qi * Qx;
  const float Es = 2.0f * Eg + (gd + 2.0f * u) * (ni + Mx * Mx) + 4.0f * u * qi * Qx +
                   2.0f * u * (Ai + Mx) * (Ai + Mx);
  if (ang)
    return 2.0f * (0.5f * Es + 0.5f * gd * (x2i + X2m) + 4.0f * u * (1.0f + X2m) +
                   gd * sqrtf(x2i * X2m) + u);
  return 2.0f * (Es + gd * (Ai + Mx) * (Ai + Mx));
}

}  // namespace fg
