// Instantiations of the beam kernel for metric L2_U8 (one file per metric so the
// variants compile in parallel).
#include "beam.cuh"

namespace fg {

BeamKernelFn beam_kernel_metric2(int G, int K, int S) {
#define X(GG, KK)                                              \
  if (G == GG && K == KK) {                                    \
    if (S == 1) return beam_kernel<L2_U8, GG, KK, 1, false>;             \
    if (S == 2) return beam_kernel<L2_U8, GG, KK, 2, false>;             \
    if (S == 4) return beam_kernel<L2_U8, GG, KK, 4, false>;             \
  }
  X(4,1) X(8,1) X(16,1)
#undef X
  return nullptr;
}

}  // namespace fg
