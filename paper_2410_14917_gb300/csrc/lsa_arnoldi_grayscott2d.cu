// Arnoldi kernels instantiated for the grayscott2d operator (one translation unit
// per operator so that the library builds in parallel).
#include "lsa_batched.cuh"
#include "lsa_tma.cuh"

namespace lsa {

cudaError_t launch_arnoldi_grayscott2d(const ArnoldiParams& P, int precision, int G, cudaStream_t s) {
  return launch_arnoldi_op<OpGrayScott2D>(P, precision, G, s);
}
cudaError_t launch_matvec_grayscott2d(const ArnoldiParams& P, int precision, const void* x, void* y,
                                int G, cudaStream_t s) {
  return launch_matvec_op<OpGrayScott2D>(P, precision, x, y, G, s);
}
int blocks_per_sm_grayscott2d(int precision) { return blocks_per_sm_op<OpGrayScott2D>(precision); }
int flat_blocks_per_sm_grayscott2d(int precision) { return flat_blocks_per_sm_op<OpGrayScott2D>(precision); }
bool tma_applicable_grayscott2d(const DevOp& d, const Tiling& tl, int m, int precision) {
  return precision == LSA_FP32_BASIS ? tma_applicable_op<OpGrayScott2D, float>(d, tl, m)
                                     : tma_applicable_op<OpGrayScott2D, double>(d, tl, m);
}
cudaError_t launch_arnoldi_tma_grayscott2d(const ArnoldiParams& P, int precision, int maxG, cudaStream_t s) {
  return precision == LSA_FP32_BASIS ? launch_arnoldi_tma_op<OpGrayScott2D, float>(P, maxG, s)
                                     : launch_arnoldi_tma_op<OpGrayScott2D, double>(P, maxG, s);
}

cudaError_t launch_batched_grayscott2d(const BatchParams& BP, int precision, int G, cudaStream_t s) {
  return launch_batched_op<OpGrayScott2D>(BP, precision, G, s);
}
int batched_blocks_per_sm_grayscott2d(int precision) { return batched_blocks_per_sm_op<OpGrayScott2D>(precision); }

}  // namespace lsa
