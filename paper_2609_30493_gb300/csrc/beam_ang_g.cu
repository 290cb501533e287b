// Instantiations of the beam kernel for metric ANGULAR_F32 with candidate rows
// gathered by bulk copies into shared memory (rows of at most 64 chunks).
#include "beam.cuh"

namespace fg {

BeamKernelFn beam_kernel_metric1_gather(int G, int K, int S) {
#define X(GG, KK)                                                   \
  if (G == GG && K == KK) {                                         \
    if (S == 1) return beam_kernel<ANGULAR_F32, GG, KK, 1, true>;  \
    if (S == 2) return beam_kernel<ANGULAR_F32, GG, KK, 2, true>;  \
    if (S == 4) return beam_kernel<ANGULAR_F32, GG, KK, 4, true>;  \
  }
  X(4,1) X(8,1) X(16,1) X(32,1) X(32,2)
#undef X
  return nullptr;
}

}  // namespace fg
