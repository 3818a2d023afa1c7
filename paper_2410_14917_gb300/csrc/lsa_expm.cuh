// Device code of S5 (augmented Hessenberg exponential) and S6 (output
// combination), shared by the standalone kernels and the batched kernel.
#pragma once

#include <math.h>

#include "lsa_internal.cuh"

namespace lsa {

// ---------------------------------------------------------------------------
// S5: phi_k(h H_m) e_1 from one exponential of the augmented matrix
//     Hhat = [[h H_m, e_1, 0], [0, 0, I_p], [0, 0, 0]]   (size n = m + p + 1)
// (the m-sized analogue of Eqs. 7-9): exp(Hhat)[:m, 0] = e^{hH} e_1 and
// exp(Hhat)[:m, m+k-1] = phi_k(hH) e_1 for k = 1..p+1.
//
// Method: scaling and squaring with a degree-18 Taylor polynomial.  With
// ||Hhat 2^-s||_1 <= 1 the truncation error is below sum_{k>=19} 1/k! < 1e-17.
// The polynomial is evaluated by the Paterson-Stockmeyer scheme with blocks of
// four powers (X^2, X^3, X^4, then four Horner steps in X^4), so the whole
// exponential is 7 + s matrix products with no linear solve.  Every product is
// spread over all CTAs of a cooperative launch (one output entry per thread),
// because FP64 arithmetic on this part is ~64x slower than FP32 and a single
// SM would take hundreds of microseconds.

constexpr int EXPM_NT = 64;
constexpr int LD = SMALL_STRIDE;
constexpr int TAYLOR_DEG = 18;

struct ExpmShared {
  int flag;
  int m, n, s;
  double scale;
  double nrm[NT];
};

__device__ __forceinline__ double hhat(const SmallParams& P, int m, double scale, int r, int c) {
  double v = 0.0;
  if (r < m && c < m) v = P.h * __ldcg(P.H + r + (long long)c * P.ldh);
  else if (r == 0 && c == m) v = 1.0;
  else if (r >= m && c == r + 1) v = 1.0;
  return v * scale;
}

// sum_k A[r][k] B[k][c] over k < n (leading dimension LD): eight loads of each
// operand in flight per round trip to L2 (a product entry is one thread's
// chain, so its loads, not its FMAs, set the time), four accumulators
// combined in a fixed order.
__device__ __forceinline__ double dot_rc(const double* A, const double* B, int r, int c, int n) {
  const double* a = A + r * LD;
  const double* b = B + c;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  for (int k = 0; k < n; k += 8) {
    double x[8], y[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const bool in = k + i < n;
      x[i] = in ? __ldcg(a + k + i) : 0.0;
      y[i] = in ? __ldcg(b + (k + i) * LD) : 0.0;
    }
    s0 = fma(x[0], y[0], s0); s1 = fma(x[1], y[1], s1);
    s2 = fma(x[2], y[2], s2); s3 = fma(x[3], y[3], s3);
    s0 = fma(x[4], y[4], s0); s1 = fma(x[5], y[5], s1);
    s2 = fma(x[6], y[6], s2); s3 = fma(x[7], y[7], s3);
  }
  return (s0 + s1) + (s2 + s3);
}

// B_l = sum_{i=0}^{3} a_{4l+i} X^i  (a_k = 1/k!; B_4 = a16 I + a17 X + a18 X^2)
__device__ __forceinline__ double block_coef(const double* X, const double* X2, const double* X3,
                                             int l, int r, int c, const double* a) {
  int k0 = 4 * l;
  double v = (r == c) ? a[k0] : 0.0;
  v = fma(a[k0 + 1], __ldcg(X + r * LD + c), v);
  v = fma(a[k0 + 2], __ldcg(X2 + r * LD + c), v);
  if (k0 + 3 <= TAYLOR_DEG) v = fma(a[k0 + 3], __ldcg(X3 + r * LD + c), v);
  return v;
}

// The exponential, run by a group of gsize CTAs (grank = this CTA's rank):
// the whole grid for the standalone kernel, a slice of it in the batched one,
// the CTAs of one cluster in the single-cluster kernel (kCluster: the group
// barriers are then the hardware cluster barrier instead of the bounded
// global-memory one).  Ends with a group barrier, so its coefficients are
// visible to the group.
template <bool kCluster = false>
static __device__ __noinline__ bool expm_group(const SmallParams& P, int grank, int gsize, ExpmShared& sh) {
  Ctl* ctl = P.ctl;
  const BarrierRef br = expm_barrier(ctl);
  const int tid = threadIdx.x;
  const int nthr = blockDim.x;
  const unsigned G = gsize;
  double a[TAYLOR_DEG + 4];
  a[0] = 1.0;
  for (int k = 1; k < TAYLOR_DEG + 4; ++k) a[k] = a[k - 1] / (double)k;
  for (int k = TAYLOR_DEG + 1; k < TAYLOR_DEG + 4; ++k) a[k] = 0.0;

  if (tid == 0) {
    int m = P.ctl_in ? __ldcg(&P.ctl_in->m_eff) : P.m;
    int st = P.ctl_in ? __ldcg(&P.ctl_in->status) : 0;
    sh.m = (st < 0) ? 0 : m;
    sh.n = sh.m + P.p + 1;
  }
  __syncthreads();
  const int m = sh.m, n = sh.n, p = P.p;
  double* X = P.mats;
  double* X2 = X + LD * LD;
  double* X3 = X2 + LD * LD;
  double* X4 = X3 + LD * LD;
  double* R0 = X4 + LD * LD;
  double* R1 = R0 + LD * LD;

  // the closing group barrier of the early exits (generation 0: no product ran)
  auto close0 = [&]() -> bool {
    if constexpr (kCluster) {
      __syncthreads();
      cluster_barrier();
      return true;
    }
    int r = barrier_arrive(br, 0u, G, &sh.flag, P.timeout_ns);
    if (r < 0) return false;
    if (r == 1) barrier_release(br, 0u);
    return true;
  };

  if (m == 0) {   // zero start vector or failed Arnoldi: all coefficients zero
    for (int i = grank * nthr + tid; i < (p + 2) * P.ldc; i += G * nthr) P.C[i] = 0.0;
    if (grank == 0 && tid == 0) ctl->err_est = 0.0;
    return close0();
  }

  // ||Hhat||_1 = max(1, max_c sum_r |h H_rc|), computed redundantly by every CTA
  {
    double mx = 0.0;
    for (int c = tid; c < m; c += nthr) {
      double s = 0.0;
      for (int r = 0; r < m; ++r) s += fabs(P.h * __ldcg(P.H + r + (long long)c * P.ldh));
      mx = fmax(mx, s);
    }
    sh.nrm[tid] = mx;
    __syncthreads();
    if (tid == 0) {
      double v = 1.0;
      for (int i = 0; i < nthr; ++i) v = fmax(v, sh.nrm[i]);
      int s = 0;
      if (!isfinite(v)) s = -1;
      else while (v > 1.0 && s < 1000) { v *= 0.5; ++s; }
      sh.s = s;
      sh.scale = (s >= 0) ? ldexp(1.0, -s) : 0.0;
    }
    __syncthreads();
  }
  if (sh.s < 0) {
    if (grank == 0 && tid == 0) {
      atomicCAS(&ctl->status, 0, (int)LSA_ERR_NUMERIC);
      ctl->err_est = 0.0;
    }
    return close0();
  }
  const int s = sh.s;
  const double scale = sh.scale;
  unsigned gen = 0;
  const int gtid = grank * nthr + tid;
  const int gstride = G * nthr;
  const int nn = n * n;

#define EXPM_BARRIER()                                                          \
  do {                                                                          \
    if constexpr (kCluster) {                                                   \
      __syncthreads();                                                          \
      cluster_barrier();                                                        \
    } else {                                                                    \
      int _r = barrier_arrive(br, gen, G, &sh.flag, P.timeout_ns);              \
      if (_r < 0) return false;                                                 \
      if (_r == 1) barrier_release(br, gen);                                    \
    }                                                                           \
    ++gen;                                                                      \
  } while (0)

  // X = Hhat * 2^-s
  for (int o = gtid; o < nn; o += gstride) {
    int r = o / n, c = o - r * n;
    X[r * LD + c] = hhat(P, m, scale, r, c);
  }
  EXPM_BARRIER();
  // X2 = X X
  for (int o = gtid; o < nn; o += gstride) {
    int r = o / n, c = o - r * n;
    X2[r * LD + c] = dot_rc(X, X, r, c, n);
  }
  EXPM_BARRIER();
  // X3 = X2 X, X4 = X2 X2
  for (int o = gtid; o < 2 * nn; o += gstride) {
    int which = o >= nn;
    int oo = o - which * nn;
    int r = oo / n, c = oo - r * n;
    (which ? X4 : X3)[r * LD + c] = dot_rc(X2, which ? X2 : X, r, c, n);
  }
  EXPM_BARRIER();
  // Horner in X^4: R = B_4; R = B_l + X^4 R for l = 3, 2, 1, 0
  double* Rin = R0;
  double* Rout = R1;
  for (int l = 3; l >= 0; --l) {
    for (int o = gtid; o < nn; o += gstride) {
      int r = o / n, c = o - r * n;
      double acc;
      if (l < 3) {
        acc = dot_rc(X4, Rin, r, c, n);
      } else {                           // R = B_4 formed on the fly: eight of its entries per round trip
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        for (int k = 0; k < n; k += 8) {
          double x[8], y[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const bool in = k + i < n;
            x[i] = in ? __ldcg(X4 + r * LD + k + i) : 0.0;
            y[i] = in ? block_coef(X, X2, X3, 4, k + i, c, a) : 0.0;
          }
          s0 = fma(x[0], y[0], s0); s1 = fma(x[1], y[1], s1);
          s2 = fma(x[2], y[2], s2); s3 = fma(x[3], y[3], s3);
          s0 = fma(x[4], y[4], s0); s1 = fma(x[5], y[5], s1);
          s2 = fma(x[6], y[6], s2); s3 = fma(x[7], y[7], s3);
        }
        acc = (s0 + s1) + (s2 + s3);
      }
      Rout[r * LD + c] = block_coef(X, X2, X3, l, r, c, a) + acc;
    }
    EXPM_BARRIER();
    double* t = Rin; Rin = Rout; Rout = t;
  }
  // squarings
  for (int q = 0; q < s; ++q) {
    for (int o = gtid; o < nn; o += gstride) {
      int r = o / n, c = o - r * n;
      Rout[r * LD + c] = dot_rc(Rin, Rin, r, c, n);
    }
    EXPM_BARRIER();
    double* t = Rin; Rin = Rout; Rout = t;
  }
  // extract: C[k][i] = E[i][col_k], col_0 = 0, col_k = m + k - 1 (k = 1..p+1)
  const double beta = P.ctl_in ? __ldcg(&P.ctl_in->beta) : 1.0;
  for (int o = gtid; o < (p + 2) * P.ldc; o += gstride) {
    int k = o / P.ldc, i = o - k * P.ldc;
    double v = 0.0;
    if (i < m) {
      int col = (k == 0) ? 0 : m + k - 1;
      v = __ldcg(Rin + i * LD + col);
      if (P.scale_out && k <= p) v *= beta * __ldcg(&P.ctl_in->sigma[i]);
    }
    P.C[o] = v;
  }
  if (grank == 0 && tid == 0) {
    ctl->expm_s = s;
    double err = 0.0;
    if (P.ctl_in && !__ldcg(&P.ctl_in->breakdown)) {
      double phin = __ldcg(Rin + (m - 1) * LD + (m + p));
      err = beta * fabs(P.h) * __ldcg(&P.ctl_in->h_last) * fabs(phin);
    }
    ctl->err_est = err;
    if (P.tol > 0.0 && err > P.tol * beta) atomicCAS(&ctl->status, 0, (int)LSA_NOT_CONVERGED);
  }
  EXPM_BARRIER();
  return true;
}
#undef EXPM_BARRIER


// Run by a group of gsize CTAs (grank = this CTA's rank).  C and V are read
// through L2 (ld.global.cg): in the batched kernel both were written earlier in
// the same launch, where the non-coherent path is not allowed.
template <class B, int PP>
__device__ __forceinline__ void combine_group(const B* __restrict__ V, long long N,
                                              const double* __restrict__ C, int ldc, int p,
                                              const Ctl* ctl, double* __restrict__ y, int grank,
                                              int gsize) {
  __shared__ double cs[(PMAX + 1) * (MMAX + 2)];
  __shared__ float csf[(PMAX + 1) * (MMAX + 2)];   // float copies: no FP64 pipe in the float form
  __shared__ int sm;
  if (threadIdx.x == 0) sm = __ldcg(&ctl->m_eff) * (__ldcg(&ctl->status) >= 0);
  __syncthreads();
  const int m = sm;
  for (int i = threadIdx.x; i < (p + 1) * m; i += blockDim.x) {
    int k = i / m, c = i - k * m;
    const double v = __ldcg(C + (long long)k * ldc + c);
    cs[k * (MMAX + 2) + c] = v;
    csf[k * (MMAX + 2) + c] = (float)v;
  }
  __syncthreads();
  const long long stride = (long long)gsize * blockDim.x;
  for (long long e = grank * (long long)blockDim.x + threadIdx.x; e < N; e += stride) {
    if constexpr (sizeof(B) == 8) {
      double acc[PP + 1];
#pragma unroll
      for (int k = 0; k <= PP; ++k) acc[k] = 0.0;
      for (int i = 0; i < m; ++i) {
        double v = __ldcg(V + (long long)i * N + e);
#pragma unroll
        for (int k = 0; k <= PP; ++k)
          if (k <= p) acc[k] = fma(cs[k * (MMAX + 2) + i], v, acc[k]);
      }
#pragma unroll
      for (int k = 0; k <= PP; ++k)
        if (k <= p) y[(long long)k * N + e] = acc[k];
    } else {
      float acc[PP + 1];
#pragma unroll
      for (int k = 0; k <= PP; ++k) acc[k] = 0.f;
      for (int i = 0; i < m; ++i) {
        float v = __ldcg(V + (long long)i * N + e);
#pragma unroll
        for (int k = 0; k <= PP; ++k)
          if (k <= p) acc[k] = fmaf(csf[k * (MMAX + 2) + i], v, acc[k]);
      }
#pragma unroll
      for (int k = 0; k <= PP; ++k)
        if (k <= p) y[(long long)k * N + e] = (double)acc[k];
    }
  }
}


}  // namespace lsa
