// Small kernels: workspace initialisation, the augmented Hessenberg exponential
// (S5), the output combination (S6), basis rescaling for lsa_arnoldi, and the
// barrier-timeout self-test.
#include <math.h>

#include "lsa_expm.cuh"

namespace lsa {

// ---------------------------------------------------------------------------
// Initialisation: zero the control block and H, and (FP32-basis form) make the
// float copies of the coefficient fields used by the stencil.

__global__ void k_init(Ctl* ctl, DevOp op, float* g0, float* g1, int precision, double* H,
                       int hcount, const double* vin, void* vcol0, float* edge0) {
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const int nctl = (int)(sizeof(Ctl) / sizeof(int));
  for (long long i = tid; i < nctl; i += stride) reinterpret_cast<int*>(ctl)[i] = 0;
  for (long long i = tid; i < hcount; i += stride) H[i] = 0.0;
  if (vin && vcol0) {   // basis column 0 holds the start vector (in the basis type)
    if (precision == LSA_FP64)
      for (long long i = tid; i < op.N; i += stride) reinterpret_cast<double*>(vcol0)[i] = vin[i];
    else
      for (long long i = tid; i < op.N; i += stride) reinterpret_cast<float*>(vcol0)[i] = (float)vin[i];
  }
  if (vin && edge0) {   // x-halo edges of column 0 for the streaming kernel
    const int tx = op.nx / TX, ty = op.ny / TY;
    for (long long e = tid; e < op.N / 8; e += stride) {
      const long long t = e / (2 * TY);
      const int r = (int)(e - t * (2 * TY));
      const int side = r / TY, ly = r - side * TY;
      const int bx = (int)(t % tx);
      const long long rest = t / tx;
      const int by = (int)(rest % ty), z = (int)(rest / ty);
      const int x = side ? (bx * TX + TX) % op.nx : (bx * TX - 1 + op.nx) % op.nx;
      const int y = by * TY + ly;
      edge0[e] = (float)vin[x + (long long)op.nx * (y + (long long)op.ny * z)];
    }
  }
  if (precision == LSA_FP32_BASIS) {
    if (op.kind == LSA_OP_GRAYSCOTT2D) {
      long long n = op.nx * (long long)op.ny;
      for (long long i = tid; i < n; i += stride) {
        double u0 = op.f0[i], v0 = op.f1[i];
        g0[i] = (float)(v0 * v0);
        g1[i] = (float)(2.0 * u0 * v0);
      }
    } else if (op.kind == LSA_OP_ADR3D) {
      for (long long i = tid; i < op.npts; i += stride) g0[i] = (float)op.f0[i];
    }
  }
}

cudaError_t launch_init(Ctl* ctl, const DevOp& op, float* g0, float* g1, int precision, double* H,
                        int hcount, const double* vin, void* vcol0, cudaStream_t s, float* edge0) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  k_init<<<sms * 4, 256, 0, s>>>(ctl, op, g0, g1, precision, H, hcount, vin, vcol0, edge0);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(EXPM_NT) k_expm(SmallParams P) {
  __shared__ ExpmShared sh;
  expm_group(P, blockIdx.x, gridDim.x, sh);
}

cudaError_t launch_expm(const SmallParams& P, cudaStream_t s) {
  int dev = 0, sms = 0, nb = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_expm, EXPM_NT, 0);
  int G = sms * (nb > 0 ? (nb < 2 ? nb : 2) : 1);
  // one product entry per thread in the largest phase (X^3 and X^4 together,
  // 2 n^2 entries for n = m + p + 1 at most): more CTAs would only wait at the
  // barrier between the products
  const int n = P.m + P.p + 1;
  const int need = (2 * n * n + EXPM_NT - 1) / EXPM_NT;
  if (need < G) G = need > 0 ? need : 1;
  SmallParams Pc = P;
  void* args[1] = {&Pc};
  return cudaLaunchCooperativeKernel((void*)k_expm, dim3(G), dim3(EXPM_NT), args, 0, s);
}

// ---------------------------------------------------------------------------
// S6: y_k = beta V_m phi_k(h H_m) e_1 = sum_i C[k][i] x_i (beta and the lazy
// scales are already folded into C).

template <class B, int PP>
__global__ void __launch_bounds__(256) k_combine(const B* __restrict__ V, long long N,
                                                 const double* __restrict__ C, int ldc, int p,
                                                 const Ctl* ctl, double* __restrict__ y) {
  combine_group<B, PP>(V, N, C, ldc, p, ctl, y, blockIdx.x, gridDim.x);
}

cudaError_t launch_combine(const void* V, int precision, long long N, const double* C, int ldc,
                           int p, const Ctl* ctl, double* y, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long need = (N + 255) / 256;
  int G = (int)(need < (long long)sms * 8 ? need : (long long)sms * 8);
  if (G < 1) G = 1;
  if (precision == LSA_FP64) {
    if (p <= 3) k_combine<double, 3><<<G, 256, 0, s>>>((const double*)V, N, C, ldc, p, ctl, y);
    else k_combine<double, PMAX><<<G, 256, 0, s>>>((const double*)V, N, C, ldc, p, ctl, y);
  } else {
    if (p <= 3) k_combine<float, 3><<<G, 256, 0, s>>>((const float*)V, N, C, ldc, p, ctl, y);
    else k_combine<float, PMAX><<<G, 256, 0, s>>>((const float*)V, N, C, ldc, p, ctl, y);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// lsa_arnoldi output: copy the workspace basis into the caller's V, columns
// 0..m_eff, scaled by the lazy scales sigma_i of the hybrid variants.

template <class B>
__global__ void k_copy_basis(B* Vd, const B* Vs, long long N, int m, const Ctl* ctl, int apply_sigma) {
  const int me = __ldcg(&ctl->m_eff);
  const int cols = (me < m) ? me + 1 : m + 1;
  const long long total = N * cols;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += stride) {
    const int c = (int)(i / N);
    B v = Vs[i];
    if (apply_sigma) v = (B)((double)v * __ldcg(&ctl->sigma[c]));
    Vd[i] = v;
  }
}

cudaError_t launch_copy_basis(void* Vd, const void* Vs, int precision, long long N, int m,
                              const Ctl* ctl, int apply_sigma, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (precision == LSA_FP64)
    k_copy_basis<double><<<sms * 8, 256, 0, s>>>((double*)Vd, (const double*)Vs, N, m, ctl, apply_sigma);
  else
    k_copy_basis<float><<<sms * 8, 256, 0, s>>>((float*)Vd, (const float*)Vs, N, m, ctl, apply_sigma);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Self-test of the bounded barrier wait: two CTAs wait for a third participant
// that does not exist, so the release flag is never set; each gives up after
// timeout_ns and the kernel ends with status LSA_ERR_TIMEOUT.

__global__ void k_timeout_selftest(Ctl* ctl, long long timeout_ns) {
  __shared__ int flag;
  const BarrierRef br = arnoldi_barrier(ctl);
  int r = barrier_arrive(br, 0u, gridDim.x + 1u, &flag, timeout_ns);
  if (r == 1) barrier_release(br, 0u);   // unreachable: the count is never met
}

cudaError_t launch_timeout_selftest(Ctl* ctl, long long timeout_ns, cudaStream_t s) {
  k_timeout_selftest<<<2, 32, 0, s>>>(ctl, timeout_ns);
  return cudaGetLastError();
}

}  // namespace lsa
