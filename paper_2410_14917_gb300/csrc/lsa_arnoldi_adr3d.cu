// Arnoldi kernels instantiated for the adr3d operator (one translation unit
// per operator so that the library builds in parallel).
#include "lsa_batched.cuh"
#include "lsa_stream.cuh"
#include "lsa_tma.cuh"

namespace lsa {

cudaError_t launch_arnoldi_adr3d(const ArnoldiParams& P, int precision, int G, cudaStream_t s) {
  return launch_arnoldi_op<OpADR3D>(P, precision, G, s);
}
cudaError_t launch_matvec_adr3d(const ArnoldiParams& P, int precision, const void* x, void* y,
                                int G, cudaStream_t s) {
  return launch_matvec_op<OpADR3D>(P, precision, x, y, G, s);
}
int blocks_per_sm_adr3d(int precision) { return blocks_per_sm_op<OpADR3D>(precision); }
int flat_blocks_per_sm_adr3d(int precision) { return flat_blocks_per_sm_op<OpADR3D>(precision); }
bool tma_applicable_adr3d(const DevOp& d, const Tiling& tl, int m, int precision) {
  return precision == LSA_FP32_BASIS ? tma_applicable_op<OpADR3D, float>(d, tl, m)
                                     : tma_applicable_op<OpADR3D, double>(d, tl, m);
}
cudaError_t launch_arnoldi_tma_adr3d(const ArnoldiParams& P, int precision, int maxG, cudaStream_t s) {
  return precision == LSA_FP32_BASIS ? launch_arnoldi_tma_op<OpADR3D, float>(P, maxG, s)
                                     : launch_arnoldi_tma_op<OpADR3D, double>(P, maxG, s);
}

bool stream_applicable_adr3d(const DevOp& d, const Tiling& tl, int m) {
  return stream_applicable_op<OpADR3D>(d, tl, m);
}
cudaError_t launch_arnoldi_stream_adr3d(const ArnoldiParams& P, cudaStream_t s) {
  return launch_arnoldi_stream_op<OpADR3D>(P, s);
}

cudaError_t launch_batched_adr3d(const BatchParams& BP, int precision, int G, cudaStream_t s) {
  return launch_batched_op<OpADR3D>(BP, precision, G, s);
}
int batched_blocks_per_sm_adr3d(int precision) { return batched_blocks_per_sm_op<OpADR3D>(precision); }

}  // namespace lsa
