// Arnoldi kernels instantiated for the advdiff2d operator (one translation unit
// per operator so that the library builds in parallel).
#include "lsa_batched.cuh"
#include "lsa_cluster.cuh"
#include "lsa_stream.cuh"
#include "lsa_tma.cuh"

namespace lsa {

cudaError_t launch_arnoldi_advdiff2d(const ArnoldiParams& P, int precision, int G, cudaStream_t s) {
  return launch_arnoldi_op<OpAdvDiff2D>(P, precision, G, s);
}
cudaError_t launch_matvec_advdiff2d(const ArnoldiParams& P, int precision, const void* x, void* y,
                                int G, cudaStream_t s) {
  return launch_matvec_op<OpAdvDiff2D>(P, precision, x, y, G, s);
}
int blocks_per_sm_advdiff2d(int precision) { return blocks_per_sm_op<OpAdvDiff2D>(precision); }
int flat_blocks_per_sm_advdiff2d(int precision) { return flat_blocks_per_sm_op<OpAdvDiff2D>(precision); }
bool tma_applicable_advdiff2d(const DevOp& d, const Tiling& tl, int m, int precision) {
  return precision == LSA_FP32_BASIS ? tma_applicable_op<OpAdvDiff2D, float>(d, tl, m)
                                     : tma_applicable_op<OpAdvDiff2D, double>(d, tl, m);
}
cudaError_t launch_arnoldi_tma_advdiff2d(const ArnoldiParams& P, int precision, int maxG, cudaStream_t s) {
  return precision == LSA_FP32_BASIS ? launch_arnoldi_tma_op<OpAdvDiff2D, float>(P, maxG, s)
                                     : launch_arnoldi_tma_op<OpAdvDiff2D, double>(P, maxG, s);
}

bool stream_applicable_advdiff2d(const DevOp& d, const Tiling& tl, int m) {
  return stream_applicable_op<OpAdvDiff2D>(d, tl, m);
}
cudaError_t launch_arnoldi_stream_advdiff2d(const ArnoldiParams& P, cudaStream_t s) {
  return launch_arnoldi_stream_op<OpAdvDiff2D>(P, s);
}

bool cluster_applicable_advdiff2d(const DevOp& d, const Tiling& tl, int m) {
  return cluster_applicable_op<OpAdvDiff2D>(d, tl, m);
}
cudaError_t launch_arnoldi_cluster_advdiff2d(const ArnoldiParams& P, const SmallParams* SP, double* y,
                                             cudaStream_t s) {
  return launch_arnoldi_cluster_op<OpAdvDiff2D>(P, SP, y, s);
}

cudaError_t launch_batched_advdiff2d(const BatchParams& BP, int precision, int G, cudaStream_t s) {
  return launch_batched_op<OpAdvDiff2D>(BP, precision, G, s);
}
int batched_blocks_per_sm_advdiff2d(int precision) { return batched_blocks_per_sm_op<OpAdvDiff2D>(precision); }

}  // namespace lsa
