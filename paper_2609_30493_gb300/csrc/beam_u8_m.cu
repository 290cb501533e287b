// Instantiations of the many-builds beam kernel (one launch over the work
// items of several indices) for metric L2_U8.
#include "beam.cuh"

namespace fg {

BeamMultiFn beam_multi_metric2(int G, int K, int S) {
#define X(GG, KK)                                                        \
  if (G == GG && K == KK) {                                              \
    if (S == 1) return beam_multi_kernel<L2_U8, GG, KK, 1, false>;  \
    if (S == 2) return beam_multi_kernel<L2_U8, GG, KK, 2, false>;  \
    if (S == 4) return beam_multi_kernel<L2_U8, GG, KK, 4, false>;  \
  }
  X(4,1) X(8,1) X(16,1)
#undef X
  return nullptr;
}

}  // namespace fg
