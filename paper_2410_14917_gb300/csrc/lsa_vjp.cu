// Vector-Jacobian product of the phi_1 product on the Gray-Scott Jacobian:
// the gradients of a loss L(y), y = phi_1(h A(theta)) v, with respect to v, h
// and theta = (Du, Dv, F, k), given r = dL/dy.  Every term is one more phi
// product through the same Arnoldi engine plus a deterministic dot product:
//   dL/dv     = phi_1(h A^T) r                      (operator LSA_OP_GRAYSCOTT2D_T)
//   dL/dh     = r . (phi_0(hA)v - phi_1(hA)v) / h   (d/dh [h phi_1(hA)] = e^{hA}, Eq. 6)
//   dL/dtheta = r . [phi_1(hK)[0; v]]_top,  K = [[A, dA/dtheta], [0, A]]
//               (LSA_OP_GRAYSCOTT2D_FRECHET: Sect. 2.1's Eq. 7 with the
//               block-triangular augmentation of the Frechet derivative of exp)
//               for Du, Dv and k;
//   dL/dF     = -h r . (phi_1(hA)v - phi_2(hA)v)   (dA/dF = -I commutes with A,
//               and phi_1' = phi_1 - phi_2 by Eq. 6): no product of its own.
// No basis is stored between the forward product and these calls: each call
// rebuilds its Krylov basis from v, r and the operator (recomputation instead
// of keeping V_m).
#include <string.h>

#include "lsa_internal.cuh"

namespace lsa {

constexpr int DOT_NT = 256;
constexpr int DOT_MAXB = 1024;

// part[b] = sum over this block's elements of a_i (b_i - c_i) (c may be null), fixed order
__global__ void __launch_bounds__(DOT_NT) k_dot_partial(const double* __restrict__ a, const double* __restrict__ b,
                                                        const double* __restrict__ c, long long n,
                                                        double* __restrict__ part) {
  __shared__ double sh[DOT_NT];
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)DOT_NT + threadIdx.x; i < n; i += (long long)gridDim.x * DOT_NT)
    acc = fma(a[i], c ? b[i] - c[i] : b[i], acc);
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = DOT_NT / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(DOT_NT) k_dot_final(const double* __restrict__ part, int nb, double scale,
                                                      double* __restrict__ out) {
  __shared__ double sh[DOT_NT];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nb; i += DOT_NT) acc += part[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = DOT_NT / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = scale * sh[0];
}

static cudaError_t launch_dot(const double* a, const double* b, const double* c, long long n, double scale,
                              double* part, double* out, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long need = (n + DOT_NT - 1) / DOT_NT;
  int nb = (int)(need < (long long)sms * 4 ? need : (long long)sms * 4);
  if (nb > DOT_MAXB) nb = DOT_MAXB;
  if (nb < 1) nb = 1;
  k_dot_partial<<<nb, DOT_NT, 0, s>>>(a, b, c, n, part);
  k_dot_final<<<1, DOT_NT, 0, s>>>(part, nb, scale, out);
  return cudaGetLastError();
}

struct VjpLayout {
  size_t phiv, z0, yk, part, total;
};

static bool vjp_layout(const lsa_op* op, int m, VjpLayout* L, long long* Nout) {
  if (!op || op->kind != LSA_OP_GRAYSCOTT2D) return false;
  lsa_op opT = *op, opK = *op;
  opT.kind = LSA_OP_GRAYSCOTT2D_T;
  opK.kind = LSA_OP_GRAYSCOTT2D_FRECHET;
  opK.aux = 0;
  const long long N = lsa_op_dof(op);
  if (N < 1) return false;
  const size_t wT = lsa_workspace_bytes(&opT, m, 1, LSA_FP64);
  const size_t wK = lsa_workspace_bytes(&opK, m, 1, LSA_FP64);
  if (!wT || !wK) return false;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
  L->phiv = take(wT > wK ? wT : wK);
  L->z0 = take((size_t)2 * N * sizeof(double));
  L->yk = take((size_t)4 * N * sizeof(double));
  L->part = take((size_t)DOT_MAXB * sizeof(double));
  L->total = off;
  *Nout = N;
  return true;
}

static void merge_stats(lsa_stats* acc, const lsa_stats& s, bool first) {
  if (first) { *acc = s; acc->arnoldi_kernel = 0; return; }
  if (s.status < 0 || (acc->status >= 0 && s.status > acc->status)) acc->status = s.status;
  if (s.m_eff < acc->m_eff) acc->m_eff = s.m_eff;
  acc->breakdown |= s.breakdown;
  acc->norm_fallbacks += s.norm_fallbacks;
  acc->grid_syncs += s.grid_syncs;
  acc->grid_barriers += s.grid_barriers;
  acc->ms_arnoldi += s.ms_arnoldi;
  acc->ms_expm += s.ms_expm;
  acc->ms_combine += s.ms_combine;
  acc->launches += s.launches;
}

}  // namespace lsa

using namespace lsa;

extern "C" {

size_t lsa_phiv_vjp_workspace_bytes(const lsa_op* op, int m) {
  VjpLayout L;
  long long N = 0;
  if (m < 1 || m > MMAX || !vjp_layout(op, m, &L, &N)) return 0;
  return L.total;
}

lsa_status lsa_phiv_vjp(const lsa_op* op, const double* v, double h, int m, int variant,
                        const double* r, const double* y, double* grad_v, double* grad_s,
                        void* work, size_t work_bytes, lsa_stats* stats, void* stream) {
  if (!v || !r || !y || !grad_v || !grad_s) return LSA_ERR_ARG;
  if (!isfinite(h) || h == 0.0) return LSA_ERR_ARG;
  if (variant < LSA_MGS || variant > LSA_IOCGS || m < 1 || m > MMAX) return LSA_ERR_ARG;
  VjpLayout L;
  long long N = 0;
  if (!vjp_layout(op, m, &L, &N)) return LSA_ERR_ARG;
  if (!work || ((uintptr_t)work & 255u) || work_bytes < L.total) return LSA_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  char* w = (char*)work;
  void* wp = w + L.phiv;
  const size_t wpb = L.z0 - L.phiv;
  double* z0 = (double*)(w + L.z0);
  double* yk = (double*)(w + L.yk);
  double* part = (double*)(w + L.part);
  lsa_stats one, acc;
  memset(&acc, 0, sizeof(acc));
  bool first = true;
  auto phi = [&](const lsa_op* o, const double* x) -> lsa_status {
    lsa_status st = lsa_phiv(o, x, h, 1, m, 0.0, variant, LSA_FP64, yk, wp, wpb, stats ? &one : nullptr, stream);
    if (stats && st >= 0) { merge_stats(&acc, one, first); first = false; }
    return st;
  };
  // dL/dv = phi_1(h A^T) r
  lsa_op opT = *op;
  opT.kind = LSA_OP_GRAYSCOTT2D_T;
  lsa_status st = phi(&opT, r);
  if (st < 0) return st;
  if (cudaMemcpyAsync(grad_v, yk + N, (size_t)N * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return LSA_ERR_CUDA;
  // dL/dh = r . (phi_0 v - phi_1 v) / h
  if (launch_dot(r, y, y + N, N, 1.0 / h, part, grad_s, s) != cudaSuccess) return LSA_ERR_CUDA;
  // dL/dF = -h r . (phi_1 v - phi_2 v): dA/dF = -I commutes with A, so the
  // derivative is -h phi_1'(hA) v, and phi_1'(z) = phi_1(z) - phi_2(z) (Eq. 6)
  if (launch_dot(r, y + N, y + 2 * N, N, -h, part, grad_s + 3, s) != cudaSuccess) return LSA_ERR_CUDA;
  // dL/dtheta_k = r . top half of phi_1(h K_k) [0; v] for Du, Dv and k
  if (cudaMemsetAsync(z0, 0, (size_t)N * sizeof(double), s) != cudaSuccess ||
      cudaMemcpyAsync(z0 + N, v, (size_t)N * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return LSA_ERR_CUDA;
  lsa_op opK = *op;
  opK.kind = LSA_OP_GRAYSCOTT2D_FRECHET;
  for (int k = 0; k < 4; ++k) {
    if (k == 2) continue;   // F: closed form above
    opK.aux = k;
    st = phi(&opK, z0);
    if (st < 0) return st;
    if (launch_dot(r, yk + 2 * N, nullptr, N, 1.0, part, grad_s + 1 + k, s) != cudaSuccess) return LSA_ERR_CUDA;
  }
  if (stats) {
    if (cudaStreamSynchronize(s) != cudaSuccess) return LSA_ERR_CUDA;
    acc.launches += 10;       // five dot products (two kernels each)
    *stats = acc;
    return (lsa_status)acc.status;
  }
  return LSA_OK;
}

}  // extern "C"
