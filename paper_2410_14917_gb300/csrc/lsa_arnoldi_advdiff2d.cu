// Arnoldi kernels instantiated for the advdiff2d operator (one translation unit
// per operator so that the library builds in parallel).
#include "lsa_engine.cuh"

namespace lsa {

cudaError_t launch_arnoldi_advdiff2d(const ArnoldiParams& P, int precision, int G, cudaStream_t s) {
  return launch_arnoldi_op<OpAdvDiff2D>(P, precision, G, s);
}
cudaError_t launch_matvec_advdiff2d(const ArnoldiParams& P, int precision, const void* x, void* y,
                                int G, cudaStream_t s) {
  return launch_matvec_op<OpAdvDiff2D>(P, precision, x, y, G, s);
}
int blocks_per_sm_advdiff2d(int precision) { return blocks_per_sm_op<OpAdvDiff2D>(precision); }

}  // namespace lsa
