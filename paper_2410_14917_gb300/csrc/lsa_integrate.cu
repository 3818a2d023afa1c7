// Building blocks of the exponential integrators (Sect. 4) other than the phi
// products: the Gray-Scott right-hand side F(u) whose Jacobian is the
// Gray-Scott operator, and the vector update w = a x + b y.
#include <math.h>

#include "lsa_internal.cuh"

namespace lsa {

// F(u, v) = [Du Lap u - u v^2 + F (1 - u);  Dv Lap v + u v^2 - (F + k) v],
// periodic 5-point Laplacian; state and result species-major (u block, v block).
__global__ void k_grayscott_rhs(DevOp d, const double* __restrict__ w, double* __restrict__ f) {
  const long long n = d.npts;
  const double* u = w;
  const double* v = w + n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % d.nx), y = (int)(i / d.nx);
    const long long row = (long long)d.nx * y;
    const long long iW = (x == 0 ? d.nx - 1 : x - 1) + row;
    const long long iE = (x + 1 == d.nx ? 0 : x + 1) + row;
    const long long iS = x + (long long)d.nx * (y == 0 ? d.ny - 1 : y - 1);
    const long long iN = x + (long long)d.nx * (y + 1 == d.ny ? 0 : y + 1);
    const double uc = u[i], vc = v[i];
    const double lu = (u[iW] + u[iE]) + (u[iS] + u[iN]) - 4.0 * uc;
    const double lv = (v[iW] + v[iE]) + (v[iS] + v[iN]) - 4.0 * vc;
    const double uvv = uc * vc * vc;
    f[i] = d.du * lu - uvv + d.F * (1.0 - uc);
    f[n + i] = d.dv * lv + uvv - (d.F + d.k) * vc;
  }
}

__global__ void k_axpby(long long n, double a, const double* x, double b, const double* y, double* w) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    w[i] = a * x[i] + b * y[i];
}

static int grid_for(long long n) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long g = (n + 255) / 256;
  const long long cap = (long long)(sms > 0 ? sms : 1) * 8;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace lsa

using namespace lsa;

extern "C" {

lsa_status lsa_rhs(const lsa_op* op, const double* u, double* f, void* stream) {
  if (!op || !u || !f || op->kind != LSA_OP_GRAYSCOTT2D) return LSA_ERR_ARG;
  DevOp d;
  if (!make_devop(op, &d)) return LSA_ERR_ARG;
  k_grayscott_rhs<<<grid_for(d.npts), 256, 0, (cudaStream_t)stream>>>(d, u, f);
  return cudaGetLastError() == cudaSuccess ? LSA_OK : LSA_ERR_CUDA;
}

lsa_status lsa_axpby(long long n, double a, const double* x, double b, const double* y, double* w,
                     void* stream) {
  if (n < 0 || !isfinite(a) || !isfinite(b)) return LSA_ERR_ARG;
  if (n == 0) return LSA_OK;
  if (!x || !y || !w) return LSA_ERR_ARG;
  k_axpby<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(n, a, x, b, y, w);
  return cudaGetLastError() == cudaSuccess ? LSA_OK : LSA_ERR_CUDA;
}

}  // extern "C"
