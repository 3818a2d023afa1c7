// Float64 FMA throughput probe: the measured peak the float64 form's roofline
// is reported against.  Every thread runs PROBE_CHAINS independent FMA chains
// (enough independent work to keep the FP64 pipe of each SM busy); the
// checksum store keeps the compiler from removing them.
#include "lsa_internal.cuh"

namespace {

constexpr int PROBE_NT = 256;
constexpr int PROBE_CHAINS = 16;

__global__ void __launch_bounds__(PROBE_NT) k_probe_fp64_fma(int iters, double* out) {
  double a[PROBE_CHAINS];
  const double b = 0.999999999, c = 1e-9 * (1 + threadIdx.x % 7);
#pragma unroll
  for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = 1.0 + 1e-3 * k + 1e-6 * threadIdx.x;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = fma(a[k], b, c);
  }
  double sum = 0.0;
#pragma unroll
  for (int k = 0; k < PROBE_CHAINS; ++k) sum += a[k];
  if (sum == -1.0) out[0] = sum;   // never true for these inputs: keeps the chains live
}

}  // namespace

extern "C" lsa_status lsa_probe_fp64_fma(int iters, double* out, double* flops, void* stream) {
  if (iters < 1 || !out || !flops) return LSA_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LSA_ERR_CUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 4;
  k_probe_fp64_fma<<<blocks, PROBE_NT, 0, (cudaStream_t)stream>>>(iters, out);
  if (cudaGetLastError() != cudaSuccess) return LSA_ERR_CUDA;
  *flops = 2.0 * PROBE_CHAINS * (double)iters * blocks * PROBE_NT;
  return LSA_OK;
}
