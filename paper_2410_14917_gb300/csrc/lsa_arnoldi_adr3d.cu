// Arnoldi kernels instantiated for the adr3d operator (one translation unit
// per operator so that the library builds in parallel).
#include "lsa_engine.cuh"

namespace lsa {

cudaError_t launch_arnoldi_adr3d(const ArnoldiParams& P, int precision, int G, cudaStream_t s) {
  return launch_arnoldi_op<OpADR3D>(P, precision, G, s);
}
cudaError_t launch_matvec_adr3d(const ArnoldiParams& P, int precision, const void* x, void* y,
                                int G, cudaStream_t s) {
  return launch_matvec_op<OpADR3D>(P, precision, x, y, G, s);
}
int blocks_per_sm_adr3d(int precision) { return blocks_per_sm_op<OpADR3D>(precision); }

}  // namespace lsa
