// Arnoldi kernels for the operators of the Gray-Scott gradient (float64 form
// only): the transposed Jacobian and the block operator of the Frechet
// derivative.  One translation unit so that the library builds in parallel.
#include "lsa_engine.cuh"

namespace lsa {

cudaError_t launch_arnoldi_grayscott2d_t(const ArnoldiParams& P, int precision, int G, cudaStream_t s) {
  if (precision != LSA_FP64) return cudaErrorNotSupported;
  return launch_arnoldi_t<OpGrayScott2DT, double>(P, G, s);
}
cudaError_t launch_matvec_grayscott2d_t(const ArnoldiParams& P, int precision, const void* x, void* y,
                                        int G, cudaStream_t s) {
  if (precision != LSA_FP64) return cudaErrorNotSupported;
  return launch_matvec_t<OpGrayScott2DT, double>(P, x, y, G, s);
}
int blocks_per_sm_grayscott2d_t(int precision) {
  return precision == LSA_FP64 ? blocks_per_sm_t<OpGrayScott2DT, double>() : 0;
}

cudaError_t launch_arnoldi_grayscott2d_frechet(const ArnoldiParams& P, int precision, int G, cudaStream_t s) {
  if (precision != LSA_FP64) return cudaErrorNotSupported;
  return launch_arnoldi_t<OpGrayScottFrechet2D, double>(P, G, s);
}
cudaError_t launch_matvec_grayscott2d_frechet(const ArnoldiParams& P, int precision, const void* x,
                                              void* y, int G, cudaStream_t s) {
  if (precision != LSA_FP64) return cudaErrorNotSupported;
  return launch_matvec_t<OpGrayScottFrechet2D, double>(P, x, y, G, s);
}
int blocks_per_sm_grayscott2d_frechet(int precision) {
  return precision == LSA_FP64 ? blocks_per_sm_t<OpGrayScottFrechet2D, double>() : 0;
}

}  // namespace lsa
