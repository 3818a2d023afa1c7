// Arnoldi kernels instantiated for the grayscott2d operator (one translation unit
// per operator so that the library builds in parallel).
#include "lsa_engine.cuh"

namespace lsa {

cudaError_t launch_arnoldi_grayscott2d(const ArnoldiParams& P, int precision, int G, cudaStream_t s) {
  return launch_arnoldi_op<OpGrayScott2D>(P, precision, G, s);
}
cudaError_t launch_matvec_grayscott2d(const ArnoldiParams& P, int precision, const void* x, void* y,
                                int G, cudaStream_t s) {
  return launch_matvec_op<OpGrayScott2D>(P, precision, x, y, G, s);
}
int blocks_per_sm_grayscott2d(int precision) { return blocks_per_sm_op<OpGrayScott2D>(precision); }

}  // namespace lsa
