// Instantiations of the many-builds beam kernel (one launch over the work
// items of several indices) for metric L2_F32.
#include "beam.cuh"

namespace fg {

BeamMultiFn beam_multi_metric0(int G, int K, int S) {
#define X(GG, KK)                                                        \
  if (G == GG && K == KK) {                                              \
    if (S == 1) return beam_multi_kernel<L2_F32, GG, KK, 1, false>;  \
    if (S == 2) return beam_multi_kernel<L2_F32, GG, KK, 2, false>;  \
    if (S == 4) return beam_multi_kernel<L2_F32, GG, KK, 4, false>;  \
  }
  X(4,1) X(8,1) X(16,1) X(32,1) X(32,2) X(32,4) X(32,8)
#undef X
  return nullptr;
}

}  // namespace fg
