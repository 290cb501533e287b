// Arguments of the occlusion prune kernels of the harvest and of the final
// graph (harvest_prune.cu: lane groups; harvest_prune_tc.cu: tensor cores).
#pragma once
#include <cstdint>

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
  float* D_out;  // optional: delta(p, A_out[p][i]) beside each kept id (harvest)
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

using HPruneFn = void (*)(const HPruneArgs);

// The tensor-core prune for lists of at most nc = 128 or 256 candidates, and
// its shared memory per CTA.
HPruneFn hprune_tc_kernel_for(int metric, int G, int K, int nc);
int harvest_prune_tc_smem(int nchunks, int nc);
// The tensor-core prune runs nc compute threads and this many walker warps.
constexpr int TCP_WALKERS = 2;

}  // namespace fg
