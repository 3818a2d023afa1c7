// Internal declarations shared by the CUDA translation units of liblsarnoldi.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lsarnoldi.h"

namespace lsa {

constexpr int MMAX = 64;                  // largest Krylov dimension of the fused kernels
constexpr int PMAX = 8;                   // largest phi index p
constexpr int SLOTS = 2 * MMAX + 4;       // reduction slots per CTA and pass
constexpr int NT = 256;                   // threads per CTA of the Arnoldi kernels
constexpr int NW = NT / 32;
constexpr int TX = 16, TY = 16;           // tile footprint (grid points) in x and y
constexpr int PW = TX + 2, PH = TY + 2;   // footprint plus a one-point halo
constexpr int PS = PW * PH;               // plane size in shared memory
constexpr int KMAX = (MMAX + NW - 1) / NW; // basis columns per warp in the dot phase
constexpr int NMAX_SMALL = MMAX + PMAX + 1; // largest augmented Hessenberg size
constexpr int SMALL_STRIDE = NMAX_SMALL;    // leading dimension of small dense matrices
constexpr int RG = 32;                    // CTAs per group of the two-level grid reduction
constexpr int RG_MAX = 64;                // groups of the two-level grid reduction (G <= RG * RG_MAX)
constexpr int SMID_CAP = 256;             // SM ids tracked by the SM-aware placement

// Device-side control block, one per workspace.  Written only by the CTA that
// arrives last at a grid barrier (between barriers), read by all after it.
struct Ctl {
  unsigned int arrive;     // grid-barrier arrivals (monotonic within a launch)
  unsigned int release;    // last released barrier generation
  unsigned int e_arrive;   // barrier of the small-exponential kernel
  unsigned int e_release;
  int status;              // device-side lsa_status
  int abort_flag;          // set on a barrier timeout: every CTA leaves
  int m_eff;
  int breakdown;
  int fallbacks;
  int syncs;               // reductions performed
  int barriers;            // grid barriers performed (with or without reduction)
  int done;                // the Arnoldi loop has ended (breakdown)
  int fallback_pending;    // next pass is the explicit-norm fallback pass (Alg. 4)
  int expm_s;              // squarings used by the small exponential
  int finished;            // batched form: the instance ran to its output
  double beta;
  double nrm_est;          // current norm estimate (hybrid)
  double a;                // scale of the source vector in the next projection
  double aw_prev;          // ||A v_j|| of the last completed step (normalised units)
  double h_last;           // H_{m+1,m}
  double err_est;
  double red[SLOTS];       // reduced sums of the last reduction
  unsigned int g_arrive[RG_MAX];  // two-level reduction: arrivals per group of RG CTAs
  unsigned int p_arrive;   // placement barrier of the persistent Arnoldi kernel
  unsigned int p_release;
  int place_off;           // an SM id was out of range: CTA ranks are block indices
  unsigned int sm_ctas[SMID_CAP];  // CTAs resident per SM id
  double coef[MMAX + 2];   // projection coefficients of the next pass
  double sigma[MMAX + 2];  // lazy scales of the stored basis columns
  double hcol[MMAX + 2];
};

// Operator as the kernels see it: geometry, folded stencil coefficients, fields.
struct DevOp {
  int kind;
  int nx, ny, nz;
  int ns;                  // species (2 for Gray-Scott)
  long long npts;          // nx*ny*nz
  long long N;             // ns*npts
  // advdiff2d / adr3d: folded neighbour coefficients; center excludes r
  double cW, cE, cS, cN, cD, cU, cC;
  // grayscott2d (and its transpose and Frechet block operator)
  double du, dv, F, k;     // du = Du/dx^2, dv = Dv/dx^2
  double idx2;             // 1/dx^2
  int dir;                 // Frechet block operator: derivative direction 0..3 = Du, Dv, F, k
  const double* f0;        // fp64 fields (u0 / r)
  const double* f1;        // fp64 field v0
  const float* g0;         // fp32 fields for the FP32-basis form (a=v0^2 / r)
  const float* g1;         // fp32 field b=2 u0 v0
};

struct Tiling {
  int tiles_x, tiles_y, zsegs, ZS;
  int ntiles;
};

struct ArnoldiParams {
  DevOp op;
  Tiling tl;
  const double* vin;       // start vector (fp64)
  void* V;                 // basis, N x (m+1)
  void* W0;                // matvec ping-pong buffers
  void* W1;
  double* H;               // (m+1) x m column-major, leading dimension m+1
  Ctl* ctl;
  double* partials;        // gridDim.x x SLOTS
  double* gsum;            // two-level reduction: per-group sums, RG_MAX x SLOTS (null: one level)
  double* T;               // MMAX x MMAX correction matrix (CWY/NCWY T, GSMGS M^{-1})
  double* L;               // MMAX x MMAX strictly lower part of V^T V (GSMGS)
  int m;
  int variant;
  int write_vlast;         // MGS/CGS2: write v_{m+1} (Arnoldi output only)
  int two_phase;           // hybrid: project, grid barrier, then stencil and inner products
                           // (no halo projection; one more barrier per step)
  double brk_tol;
  long long timeout_ns;
  float* E;                // streaming float32 kernel: edge array, (m+3) columns of N/8 (or null)
  // Augmented operator of Eqs. 8-9 (phi-function linear combinations): every
  // vector carries naug = p extra entries; Aaug [x; xi] = [A x + B xi; K xi]
  // with B = [b_p, ..., b_1] and K the p x p upper shift.  naug = 0: plain A.
  int naug;
  const double* baug;      // b_0..b_p, (p+1) x N (column k of B is b_{p-k})
  double* xaug;            // extra entries of the extended basis columns, (m+3) x PMAX
  double aug_t;            // extra entries of the start vector: exp(aug_t K) e_p
};

// Workspace layout (all offsets 256-byte aligned).
struct Layout {
  size_t ctl, partials, gsum, T, L, H, V, W0, W1, small, coefs, g0, g1, E, xaug, total;
  int G;                   // CTAs of the persistent Arnoldi kernel
};

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// The one-reduce hybrid variants (Alg. 4 with Algs. 5/6/7).
__host__ __device__ inline bool is_hybrid(int variant) {
  return variant >= LSA_HCWY && variant <= LSA_HGSMGS;
}

// Edge array of the streaming float32 kernel.  For every extended-basis
// column and every TX x TY tile (bx, by) of plane z it holds the tile's
// periodic x-halo: the TY values left of the tile (x = x0-1), then the TY
// values right of it (x = x0+TX), 2*TY floats at edge_slot(); a column's
// edges take N/8 floats.  Whoever writes a column also writes its edges.
__host__ __device__ __forceinline__ long long edge_slot(int tiles_x, int tiles_y, int bx, int by, int z) {
  return (((long long)z * tiles_y + by) * tiles_x + bx) * (2 * TY);
}

// Host helpers implemented in lsa_api.cu
bool make_devop(const lsa_op* op, DevOp* d);
Tiling make_tiling(const DevOp& d);

// Launchers implemented per operator translation unit.
cudaError_t launch_arnoldi(const ArnoldiParams& P, int precision, int G, cudaStream_t s);
cudaError_t launch_matvec(const ArnoldiParams& P, int precision, const void* x, void* y, int G,
                          cudaStream_t s);
int arnoldi_blocks_per_sm(const DevOp& d, int precision);

// Small kernels (lsa_small.cu)
struct SmallParams {
  const double* H;         // Hessenberg source, column-major, leading dimension ldh
  int ldh;
  const Ctl* ctl_in;       // when non-null, m_eff / beta / sigma / h_last come from here
  Ctl* ctl;                // expm status/err_est output (may equal ctl_in)
  int m;                   // used when ctl_in is null
  int p;
  double h;
  double* mats;            // 6 scratch matrices of SMALL_STRIDE^2 doubles
  double* C;               // output coefficients: (p+2) x ldc, row k = phi_k(hH)e_1 (scaled)
  int ldc;
  int scale_out;           // 1: fold beta * sigma_i into rows 0..p (for the combine kernel)
  long long timeout_ns;
  double tol;
};
cudaError_t launch_expm(const SmallParams& P, cudaStream_t s);
cudaError_t launch_combine(const void* V, int precision, long long N, const double* C, int ldc,
                           int p, const Ctl* ctl, double* y, cudaStream_t s);
cudaError_t launch_init(Ctl* ctl, const DevOp& op, float* g0, float* g1, int precision,
                        double* H, int ldh_total, const double* vin, void* vcol0, cudaStream_t s,
                        float* edge0 = nullptr);
cudaError_t launch_copy_basis(void* Vdst, const void* Vsrc, int precision, long long N, int m,
                              const Ctl* ctl, int apply_sigma, cudaStream_t s);
cudaError_t launch_timeout_selftest(Ctl* ctl, long long timeout_ns, cudaStream_t s);

// ---------------------------------------------------------------------------
// Device helpers

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int ld_volatile_i32(const int* p) {
  return *(volatile const int*)p;
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// a + b = t + err exactly in float32 arithmetic (Knuth's two-sum; no
// multiplications, so nothing is contracted into an FMA).
__device__ __forceinline__ float two_sum(float a, float b, float& err) {
  const float t = a + b;
  const float bp = t - a;
  const float ap = t - bp;
  err = (a - ap) + (b - bp);
  return t;
}

// Warp sums of NV compensated float32 values (value i = s[i] + e[i]) at once,
// with the recursive halving of warp_sum_many: every stage adds the main parts
// with two_sum and carries the rounding error into the compensation, so the
// sum keeps about twice float32's precision with no float64 instruction.  On
// return lane l holds (s, e) of value l >> (5 - log2 NV) in s[0], e[0].
template <int NV>
__device__ __forceinline__ void warp_sum_many_comp(float (&s)[NV], float (&e)[NV]) {
  static_assert(NV >= 1 && NV <= 32 && (NV & (NV - 1)) == 0, "NV must be a power of two <= 32");
  const unsigned lane = threadIdx.x & 31u;
  int d = 16;
#pragma unroll
  for (int h = NV / 2; h >= 1; h >>= 1, d >>= 1) {
    const bool up = (lane & (unsigned)d) != 0u;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const float ss = up ? s[i] : s[i + h], se = up ? e[i] : e[i + h];
      const float ks = up ? s[i + h] : s[i], ke = up ? e[i + h] : e[i];
      const float os = __shfl_xor_sync(0xffffffffu, ss, d);
      const float oe = __shfl_xor_sync(0xffffffffu, se, d);
      float err;
      s[i] = two_sum(ks, os, err);
      e[i] = (ke + oe) + err;
    }
  }
#pragma unroll
  for (; d >= 1; d >>= 1) {
    const float os = __shfl_xor_sync(0xffffffffu, s[0], d);
    const float oe = __shfl_xor_sync(0xffffffffu, e[0], d);
    float err;
    s[0] = two_sum(s[0], os, err);
    e[0] = (e[0] + oe) + err;
  }
}

// Warp sums of NV per-lane values at once (NV a power of two, at most 32):
// recursive halving, each stage trading half of the values still held with
// the partner lane and adding the other half, so a lane does NV - 1 + (5 -
// log2 NV) additions instead of 5 per value (float64 additions are scarce on
// this GPU).  On return lane l holds the sum of value l >> (5 - log2 NV).
template <int NV>
__device__ __forceinline__ double warp_sum_many(double (&v)[NV]) {
  static_assert(NV >= 1 && NV <= 32 && (NV & (NV - 1)) == 0, "NV must be a power of two <= 32");
  const unsigned lane = threadIdx.x & 31u;
  int s = 16;
#pragma unroll
  for (int h = NV / 2; h >= 1; h >>= 1, s >>= 1) {
    const bool up = (lane & (unsigned)s) != 0u;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const double send = up ? v[i] : v[i + h];
      const double keep = up ? v[i + h] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
  double r = v[0];
#pragma unroll
  for (; s >= 1; s >>= 1) r += __shfl_xor_sync(0xffffffffu, r, s);
  return r;
}

// Grid barrier with a bounded wait.  All `count` participating CTAs call it
// with the same generation number `gen` (0, 1, 2, ...).  Returns 1 in the CTA
// that arrived last (which must later call barrier_release), 0 in the others
// once released, -1 on timeout or abort (the caller must leave the kernel).
// Must be called by all threads of the CTA; `s_flag` is a shared int.
struct BarrierRef {
  unsigned* arrive;
  unsigned* release;
  int* abort_flag;
  int* status;
};

// With `arrive` false the CTA only waits for the release (it is not one of
// the `count` participants).
// Memory ordering: the CTA barrier orders every thread's earlier writes
// before thread 0's fence, and thread 0's fence and atomic publish them at
// device scope (the grid-synchronisation pattern of cooperative groups); the
// waiting side acquires the release flag and fences before the CTA barrier
// that lets the other threads read.
__device__ __forceinline__ int barrier_arrive(const BarrierRef& b, unsigned gen, unsigned count,
                                              int* s_flag, long long timeout_ns, bool arrive = true) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    int last = 0;
    if (arrive) {
      unsigned old = atomicAdd(b.arrive, 1u);
      last = (old == (gen + 1u) * count - 1u);
    }
    int res = last ? 1 : 0;
    if (!last) {
      unsigned long long t0 = global_ns();
      unsigned it = 0;
      while (ld_acquire_u32(b.release) < gen + 1u) {
        if ((++it & 255u) == 0u) {
          if (ld_volatile_i32(b.abort_flag)) { res = -1; break; }
          if ((long long)(global_ns() - t0) > timeout_ns) {
            atomicExch(b.abort_flag, 1);
            atomicCAS(b.status, 0, (int)LSA_ERR_TIMEOUT);
            res = -1;
            break;
          }
          if (it > 4096u) __nanosleep(64);
        }
      }
    }
    __threadfence();
    *s_flag = res;
  }
  __syncthreads();
  return *s_flag;
}

// Arrival at a counter that `count` CTAs reach once per generation, without
// waiting: returns 1 in the CTA that arrived last.  Must be called by all
// threads of the CTA.
__device__ __forceinline__ int counter_arrive(unsigned* ctr, unsigned gen, unsigned count, int* s_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    *s_flag = (atomicAdd(ctr, 1u) == (gen + 1u) * count - 1u);
    __threadfence();
  }
  __syncthreads();
  return *s_flag;
}

__device__ __forceinline__ void barrier_release(const BarrierRef& b, unsigned gen) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    st_release_u32(b.release, gen + 1u);
  }
}

// Barrier of all threads of a thread-block cluster: shared and global writes
// before it are visible to the cluster's threads after it.
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ BarrierRef arnoldi_barrier(Ctl* c) {
  return BarrierRef{&c->arrive, &c->release, &c->abort_flag, &c->status};
}
__device__ __forceinline__ BarrierRef expm_barrier(Ctl* c) {
  return BarrierRef{&c->e_arrive, &c->e_release, &c->abort_flag, &c->status};
}

}  // namespace lsa
