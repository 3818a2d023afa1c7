// Single-cluster hybrid Arnoldi for small single-species 2D grids (float64).
//
// At N of a few thousand (the 64 x 64 advection-diffusion workload: 16 tiles
// of 16 x 16) the grid-wide kernel is bound by latency: its step is a grid
// barrier through global memory, a reduction by the last-arriving CTA and one
// tile of work per CTA.  Here the whole process runs in one thread-block
// cluster, one CTA per tile (at most 16 tiles, a non-portable cluster size):
//
//  * every CTA keeps its tile's slice of the basis -- all m+1 columns and the
//    two matvec buffers -- in its own shared memory (the whole basis never
//    leaves the SMs; each new column is also written through to global memory,
//    where the small exponential, the output combination and lsa_arnoldi read
//    it);
//  * the stencil reads its halo points straight from the neighbouring CTAs'
//    shared memory (distributed shared memory, ld.shared::cluster), so the
//    projection needs no recomputed halo;
//  * the grouped reduction of Alg. 4 is a cluster barrier, then CTA 0 sums the
//    CTAs' partials over DSMEM in a fixed order (deterministic), runs the
//    engine's O(j^2) step (Algs. 5/6/7: the same code as the grid kernel, in
//    its cached mode: T, L and the step's scalars stay in CTA 0's shared
//    memory) and stores the next pass's coefficients and flags straight into
//    every CTA's shared memory; a second cluster barrier releases the others.
//
// Per Alg. 4 step: three cluster barriers (halo ready, partials ready, step
// published) and no global-memory barrier.  The hardware cluster barrier has
// no timeout to bound: every CTA follows the same control flow (its decisions
// come from the published control block), so every barrier is reached by all.
#pragma once

#include "lsa_engine.cuh"
#include "lsa_expm.cuh"

namespace lsa {

constexpr int CL_MAX = 16;            // CTAs of the cluster (tiles), non-portable size
constexpr int CL_TP = TX * TY;        // grid points of a tile

__device__ __forceinline__ unsigned cl_smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned cl_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cl_sync() { cluster_barrier(); }
// the shared-memory address of `local`'s offset in CTA `rank` of the cluster
__device__ __forceinline__ unsigned cl_map(const void* local, unsigned rank) {
  unsigned a;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(cl_smem_u32(local)), "r"(rank));
  return a;
}
// the double at the same shared-memory offset in CTA `rank` of the cluster
__device__ __forceinline__ double cl_ld(const double* local, unsigned rank) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(cl_map(local, rank)) : "memory");
  return v;
}
__device__ __forceinline__ void cl_st(double* local, unsigned rank, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(cl_map(local, rank)), "d"(v) : "memory");
}
__device__ __forceinline__ void cl_st(int* local, unsigned rank, int v) {
  asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(cl_map(local, rank)), "r"(v) : "memory");
}

// Shared-memory layout after the engine's (Smem, then the MMAX x MMAX scratch
// of the O(j^2) step, which holds T between steps in CTA 0): GSMGS's L
// [MMAX][MMAX], the tile's basis [m+3][CL_TP] (columns 0..m, then the two
// matvec buffers m+1, m+2) and the CTA's partial sums [SLOTS].
template <class Op>
struct ClusterLayout {
  using E = Engine<Op, double, double>;
  static __host__ __device__ constexpr size_t l_off() { return (E::smem_bytes() + 127) & ~(size_t)127; }
  static __host__ __device__ constexpr size_t vt_off() { return l_off() + sizeof(double) * MMAX * MMAX; }
  static __host__ __device__ constexpr size_t part_off(int m) {
    return vt_off() + sizeof(double) * (size_t)(m + 3) * CL_TP;
  }
  static __host__ __device__ constexpr size_t expm_off(int m) {
    return (part_off(m) + sizeof(double) * SLOTS + 15) & ~(size_t)15;
  }
  static __host__ __device__ constexpr size_t cs_off(int m) {
    return (expm_off(m) + sizeof(ExpmShared) + 15) & ~(size_t)15;
  }
  static __host__ __device__ constexpr size_t bytes(int m) {
    return cs_off(m) + sizeof(double) * (PMAX + 1) * (MMAX + 2);
  }
};

template <class Op>
struct ClusterEngine {
  using E = Engine<Op, double, double>;
  static_assert(Op::NS == 1 && Op::DIM == 2, "single-species 2D operators");

  E& e;
  double* Vt;      // this tile's basis slice
  double* part;    // this CTA's partial sums
  const int lx, ly, gx, gy, gi;

  __device__ ClusterEngine(E& en, double* vt, double* pt)
      : e(en), Vt(vt), part(pt), lx(en.tid & (TX - 1)), ly(en.tid / TX),
        gx((en.grank % en.P.tl.tiles_x) * TX + (en.tid & (TX - 1))),
        gy((en.grank / en.P.tl.tiles_x) * TY + en.tid / TX),
        gi(gx + en.P.op.nx * gy) {}

  // x of column `col` at grid point (x, y) (periodic): this CTA's shared memory
  // or a neighbouring tile's over DSMEM
  __device__ __forceinline__ double xat(int col, int x, int y) const {
    const DevOp& d = e.P.op;
    x = wrapi(x, d.nx);
    y = wrapi(y, d.ny);
    const int r = (y / TY) * e.P.tl.tiles_x + x / TX;
    const double* p = Vt + (size_t)col * CL_TP + (y & (TY - 1)) * TX + (x & (TX - 1));
    return r == e.grank ? *p : cl_ld(p, (unsigned)r);
  }

  // One pass of the hybrid process over this tile: x = a*src - sum_{c < ncp}
  // coef_c V_c (src < 0: the start vector), stored in column xout (>= 0); with
  // wout >= 0 the stencil w = A x into column wout and the inner products of
  // columns 0..ncp-1 with x and w; the self terms selected by `self`.  Partial
  // sums as the grid kernel lays them out (x dots, w dots, then x.x, x.w,
  // w.w); returns their number.
  __device__ int pass(int ncp, int src, double a, int xout, int wout, int self) {
    const int t = e.tid;
    double x = (src < 0) ? a * __ldg(e.P.vin + gi) : a * Vt[(size_t)src * CL_TP + t];
    double xb = 0.0;   // odd columns in a second chain (half the dependency depth)
    for (int c = 0; c < ncp; ++c) {
      const double cc = e.S.coefc[c];
      const double v = Vt[(size_t)c * CL_TP + t];
      if (c & 1) xb = fma(-cc, v, xb);
      else x = fma(-cc, v, x);
    }
    x += xb;
    if (xout >= 0) {
      Vt[(size_t)xout * CL_TP + t] = x;
      reinterpret_cast<double*>(e.P.V)[(long long)xout * e.P.op.N + gi] = x;   // write-through
    }
    double w = 0.0;
    const bool stencil = wout >= 0;
    if (stencil) {
      cl_sync();   // every tile's x is in its CTA's shared memory
      const Coef<double>& cf = e.cf;
      double r = cf.cC * x;
      r = fma(cf.cW, (lx > 0) ? Vt[(size_t)xout * CL_TP + t - 1] : xat(xout, gx - 1, gy), r);
      r = fma(cf.cE, (lx < TX - 1) ? Vt[(size_t)xout * CL_TP + t + 1] : xat(xout, gx + 1, gy), r);
      r = fma(cf.cS, (ly > 0) ? Vt[(size_t)xout * CL_TP + t - TX] : xat(xout, gx, gy - 1), r);
      r = fma(cf.cN, (ly < TY - 1) ? Vt[(size_t)xout * CL_TP + t + TX] : xat(xout, gx, gy + 1), r);
      w = r;
      Vt[(size_t)wout * CL_TP + t] = w;
    }
    // self terms: block sums
    double s3[4] = {(self & SELF_XX) ? x * x : 0.0, (self & SELF_XW) ? x * w : 0.0,
                    (self & SELF_WW) ? w * w : 0.0, 0.0};
    {
      const double r = warp_sum_many<4>(s3);   // lane l: value l >> 3
      if ((e.lane & 7) == 0 && e.lane < 24) e.S.bred[e.warp][e.lane >> 3] = r;
    }
    __syncthreads();   // x, w and the warp sums are in shared memory
    const int nd = stencil ? ncp : 0;
    // inner products: warp <-> columns c = warp, warp + NW, ...; lane <-> points
    const double* xc = Vt + (size_t)xout * CL_TP;
    const double* wc = Vt + (size_t)wout * CL_TP;
    if (nd <= NW) {              // at most one column per warp
      const int c = e.warp;
      if (c < nd) {
        const double* vc = Vt + (size_t)c * CL_TP;
        double ax = 0.0, aw = 0.0;
#pragma unroll
        for (int k = 0; k < CL_TP / 32; ++k) {
          const int q = e.lane + 32 * k;
          ax = fma(vc[q], xc[q], ax);
          aw = fma(vc[q], wc[q], aw);
        }
        ax = warp_sum(ax);
        aw = warp_sum(aw);
        if (e.lane == 0) {
          part[c] = ax;
          part[nd + c] = aw;
        }
      }
    } else {                     // all the warp's columns, then one transposed warp sum
      double v[2 * KMAX];
#pragma unroll
      for (int kk = 0; kk < KMAX; ++kk) {
        const int c = e.warp + NW * kk;
        double ax = 0.0, aw = 0.0;
        if (c < nd) {
          const double* vc = Vt + (size_t)c * CL_TP;
#pragma unroll
          for (int k = 0; k < CL_TP / 32; ++k) {
            const int q = e.lane + 32 * k;
            ax = fma(vc[q], xc[q], ax);
            aw = fma(vc[q], wc[q], aw);
          }
        }
        v[2 * kk] = ax;
        v[2 * kk + 1] = aw;
      }
      const double r = warp_sum_many<2 * KMAX>(v);   // lanes 2k, 2k+1: value k
      const int k = e.lane >> 1, c = e.warp + NW * (k >> 1);
      if ((e.lane & 1) == 0 && c < nd) part[(k & 1) ? nd + c : c] = r;
    }
    if (e.tid < 3) {
      double acc = 0.0;
      for (int i = 0; i < NW; ++i) acc += e.S.bred[i][e.tid];
      part[2 * nd + e.tid] = acc;
    }
    return 2 * nd + 3;
  }

  // The grouped reduction: CTA 0 sums the CTAs' partials (fixed order), runs
  // fn (the engine's step) and publishes the control block; then every CTA
  // reads the next pass's scalars and ncoef coefficients.
  template <class Fn>
  __device__ void reduce(int nslots, int ncoef, Fn fn) {
    __syncthreads();
    cl_sync();     // every CTA's partials are in its shared memory
    if (e.grank == 0) {
      for (int s = e.tid; s < nslots; s += NT) {
        double v[CL_MAX];   // all the loads first (one DSMEM round trip), then the fixed-order sum
#pragma unroll
        for (int r = 1; r < CL_MAX; ++r) v[r] = (r < e.gsize) ? cl_ld(part + s, (unsigned)r) : 0.0;
        double acc = part[s];
#pragma unroll
        for (int r = 1; r < CL_MAX; ++r) acc += v[r];
        e.S.red[s] = acc;
      }
      __syncthreads();
      fn();
      __syncthreads();
      if (e.tid == 0) e.P.ctl->barriers = e.S.syncs_c;   // one barrier per reduction here
      // the next pass's coefficients and flags into every other CTA's shared memory
      const int per = ncoef + 1;
      for (int i = e.tid; i < (e.gsize - 1) * per; i += NT) {
        const unsigned r = 1u + (unsigned)(i / per);
        const int k = i - (i / per) * per;
        if (k < ncoef) cl_st(&e.S.coefc[k], r, (double)e.S.coefc[k]);
        else {
          cl_st(&e.S.a, r, (double)e.S.a);
          cl_st(&e.S.done, r, e.S.done);
          cl_st(&e.S.fallback_pending, r, e.S.fallback_pending);
        }
      }
      // (the control block in global memory is read only after the kernel)
    }
    cl_sync();     // the step is published; the partials may be overwritten
  }

  // Alg. 4 (the engine's run_hybrid, pass for pass): column j-1 of the basis
  // holds x_j, the matvec buffers alternate in columns m+1 and m+2.
  __device__ void run_hybrid() {
    const int m = e.P.m, wc = m + 1;
    if (e.tid == 0) { e.S.a = 1.0; e.S.done = 0; e.S.fallback_pending = 0; e.S.syncs_c = 0; }
    __syncthreads();
    for (int j = 1; j <= m; ++j) {
      const int ns = pass(j - 1, (j == 1) ? -1 : wc + ((j - 1) & 1), (j == 1) ? 1.0 : (double)e.S.a, j - 1,
                          wc + (j & 1), SELF_XX | SELF_XW | SELF_WW);
      reduce(ns, j, [&] { e.hybrid_step(j); });
      if (e.S.done) return;
      if (e.S.fallback_pending) {   // explicit norm of the projected vector (extra reduction)
        const int nf = pass(j, wc + (j & 1), (double)e.S.a, -1, -1, SELF_XX);
        reduce(nf, j, [&] { e.hybrid_fallback_finish(j); });
        if (e.S.done) return;
      }
    }
    const int nl = pass(m, wc + (m & 1), (double)e.S.a, m, -1, SELF_XX);   // v_{m+1} and its norm
    reduce(nl, 0, [&] { e.hybrid_final_finish(); });
  }
};

// With y non-null (lsa_phiv) the same launch goes on with the small
// exponential (S5, the engine's Taylor / Paterson-Stockmeyer code on the
// cluster's CTAs, cluster barriers between its products) and the output
// combination (S6) of every CTA's own tile from its shared-memory basis.
template <class Op>
__global__ void __launch_bounds__(NT, 1) k_arnoldi_cluster(ArnoldiParams P, SmallParams SP, double* y) {
  extern __shared__ __align__(128) unsigned char smem_cl[];
  using E = Engine<Op, double, double>;
  using LY = ClusterLayout<Op>;
  typename E::Smem& S = *reinterpret_cast<typename E::Smem*>(smem_cl);
  E e(P, S, reinterpret_cast<double*>(smem_cl + E::small_offset()));
  e.grank = (int)cl_rank();
  e.gsize = (int)gridDim.x;   // the grid is the cluster
  e.cached = true;            // CTA 0 runs every step: its state stays in shared memory
  e.smallL = reinterpret_cast<double*>(smem_cl + LY::l_off());
  ClusterEngine<Op> c(e, reinterpret_cast<double*>(smem_cl + LY::vt_off()),
                      reinterpret_cast<double*>(smem_cl + LY::part_off(P.m)));
  c.run_hybrid();
  __threadfence();   // CTA 0's control block, H and scales, for the exponential
  cl_sync();         // ... and no CTA goes on while another may read its shared memory
  if (y == nullptr) return;
  ExpmShared& esh = *reinterpret_cast<ExpmShared*>(smem_cl + LY::expm_off(P.m));
  expm_group<true>(SP, e.grank, e.gsize, esh);
  // y_k = beta V_m phi_k(hH)e_1 on this tile: C (beta and the lazy scales folded
  // in) from the exponential, the basis from shared memory
  double* cs = reinterpret_cast<double*>(smem_cl + LY::cs_off(P.m));
  if (threadIdx.x == 0) S.flag = __ldcg(&P.ctl->m_eff) * (__ldcg(&P.ctl->status) >= 0);
  __syncthreads();
  const int me = S.flag, pp = SP.p;
  for (int i = threadIdx.x; i < (pp + 1) * me; i += NT) {
    const int k = i / me, col = i - k * me;
    cs[k * (MMAX + 2) + col] = __ldcg(SP.C + (long long)k * SP.ldc + col);
  }
  __syncthreads();
  const long long N = P.op.N;
  for (int k = 0; k <= pp; ++k) {
    double acc = 0.0;
    for (int i = 0; i < me; ++i) acc = fma(cs[k * (MMAX + 2) + i], c.Vt[(size_t)i * CL_TP + threadIdx.x], acc);
    y[(long long)k * N + c.gi] = acc;
  }
}

// ---------------------------------------------------------------------------
// Host side

// The cluster form applies to the hybrid variants in float64 on single-species
// 2D grids of whole 16 x 16 tiles, at most CL_MAX of them, whose layout fits
// one CTA's shared memory, when the device can run such a cluster.
template <class Op>
bool cluster_applicable_op(const DevOp& d, const Tiling& tl, int m) {
  if (Op::NS != 1 || Op::DIM != 2) return false;
  if (d.nx % TX != 0 || d.ny % TY != 0 || d.nz != 1) return false;
  const int tiles = tl.tiles_x * tl.tiles_y;
  if (tiles < 1 || tiles > CL_MAX || m < 1 || m > MMAX) return false;
  const size_t sm = ClusterLayout<Op>::bytes(m);
  if (sm > 227 * 1024) return false;
  auto k = k_arnoldi_cluster<Op>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) return false;
  if (tiles > 8 && cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    return false;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)tiles;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(tiles);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = sm;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, (void*)k, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return nclusters >= 1;
}

template <class Op>
cudaError_t launch_arnoldi_cluster_op(const ArnoldiParams& P, const SmallParams* SP, double* y, cudaStream_t s) {
  const int tiles = P.tl.tiles_x * P.tl.tiles_y;
  const size_t sm = ClusterLayout<Op>::bytes(P.m);
  auto k = k_arnoldi_cluster<Op>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e == cudaSuccess && tiles > 8) e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)tiles;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(tiles);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  ArnoldiParams Pc = P;
  SmallParams Sc;
  if (SP) Sc = *SP;
  else memset(&Sc, 0, sizeof(Sc));
  return cudaLaunchKernelEx(&cfg, k, Pc, Sc, SP ? y : (double*)nullptr);
}

}  // namespace lsa
