// Persistent Arnoldi kernels: the tile pass engine and the three Gram-Schmidt
// schemes (MGS, CGS2, hybrid low-synchronisation) built on it.
//
// One cooperative launch runs a whole Arnoldi process.  Each "pass" streams
// the grid tile by tile: it projects a vector (x = a*src - sum_c coef_c V_c),
// optionally applies the stencil (w = A x, needing the projection on a
// one-point halo, recomputed redundantly by each tile -- or, in the two-phase
// forms of the hybrid step, projected once over flat shares and read back
// after a grid barrier, by the tiles or, in the flat form, over flat shares
// of the points again), and accumulates inner products of basis columns with
// x and/or w.  The per-CTA partial sums go to
// global memory, and one grid barrier reduces them in two levels: the last CTA
// of each group of RG CTAs sums its group, the last group sums the group rows
// (both in a fixed order: deterministic) and does the small O(j^2)
// double-precision work of the step (H column, correction matrix T, norm
// estimate) before releasing the others.  (The batched form, whose groups are
// instances, sums all its CTAs' partials in one level.)  A global reduction of the paper
// (an MPI_Allreduce, Sect. 2.3) is therefore one grid barrier here.
#pragma once

#include "lsa_ops.cuh"

namespace lsa {

enum : int { DOT_X = 1, DOT_W = 2 };
enum : int { SELF_XX = 1, SELF_XW = 2, SELF_WW = 4 };

template <class B>
struct PassT {
  int c0, c1;            // projection columns [c0, c1) of V (coefficients in smem coef[c])
  double a;              // scale of the source vector
  const double* src64;   // source: fp64 start vector (first pass) ...
  const B* srcB;         // ... or a basis-typed buffer (may alias xout: in-place update)
  B* xout;               // destination of x (owned interior points), or null
  B* wout;               // stencil output (w = A x), null when the pass has no stencil
  int d0, d1;            // dot columns [d0, d1) of V
  int dmode;             // DOT_X | DOT_W
  int self;              // SELF_* bits
};

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// AUG: the augmented operator of Eqs. 8-9 (phi-function linear combinations;
// float64 only).  A separate instantiation, so that the plain kernels carry
// none of its code.
template <class Op, class Tc, class B, bool AUG = false>
struct Engine {
  static constexpr int NS = Op::NS;
  static constexpr int DIM = Op::DIM;
  static constexpr int RING = (DIM == 3) ? 3 : 1;
  static constexpr int NPL = (NS * TX * TY + 31) / 32;
  static constexpr bool F64 = sizeof(Tc) == 8;

  struct Smem {
    Tc ring[RING * NS * PS];
    Tc wbuf[NS * TX * TY];
    Tc coefc[MMAX + 2];
    double red[SLOTS];
    double tmp[4][MMAX + 2];
    double bred[NW][3];
    double sj, scale, true_nrm, ss;
    double xi[PMAX], xw[PMAX];       // augmented operator: extra entries of the pass's x and w
    int aug_xcol, aug_wcol;          // ... and the columns they belong to (-1: not stored)
    Tc a;
    int flag, done, fallback_pending, stop;
    // cached mode (one CTA runs every step): lazy scales, norm estimate and
    // ||A v_j|| of the last step, kept here instead of re-read from global
    double sig[MMAX + 2];
    double nrm_est_c, aw_prev_c;
    int syncs_c;                     // reductions counted so far (cached mode)
  };

  const ArnoldiParams& P;
  Smem& S;
  double* small;                     // MMAX x MMAX scratch: T (every CTA, CWY/NCWY) or the step's staging
  // Cached mode: the same CTA runs every step (the single-cluster kernel), so T
  // (and GSMGS's L, in smallL) stay in shared memory between steps, the lazy
  // scales and scalars are read from S, and the step also leaves the next
  // pass's coefficients and flags in S (S.coefc, S.a, S.done,
  // S.fallback_pending).  Global copies are written as in the grid kernels.
  bool cached = false;
  double* smallL = nullptr;
  // Grid kernels running Engine::run_hybrid with the CWY or NCWY correction:
  // every CTA keeps T in its `small` scratch, one new row per step read in
  // load_ctl, so that whichever CTA runs the next step need not stage it.
  bool tcache = false;
  Coef<Tc> cf;
  const int tid, lane, warp;
  int grank, gsize;                  // this CTA's rank in its group and the group size
  __host__ __device__ static constexpr size_t small_offset() { return (sizeof(Smem) + 127) & ~(size_t)127; }
  __host__ __device__ static constexpr size_t smem_bytes() { return small_offset() + sizeof(double) * MMAX * MMAX; }
  // dot accumulators (per lane)
  double ax[KMAX], aw[KMAX];
  float axs[KMAX], axc[KMAX], aws[KMAX], awc[KMAX];
  double sxx, sxw, sww;              // self terms (float64 form)
  float fxx[2], fxw[2], fww[2];      // self terms (float32 form): Kahan sum, compensation

  __device__ Engine(const ArnoldiParams& p, Smem& s, double* sm)
      : P(p), S(s), small(sm), tid(threadIdx.x), lane(threadIdx.x & 31), warp(threadIdx.x >> 5),
        grank(blockIdx.x), gsize(gridDim.x) {
    cf.load(P.op);
  }

  __device__ __forceinline__ const B* Vc(int c) const {
    return reinterpret_cast<const B*>(P.V) + (long long)c * P.op.N;
  }

  __device__ void zero_acc() {
#pragma unroll
    for (int k = 0; k < KMAX; ++k) { ax[k] = 0; aw[k] = 0; axs[k] = 0; axc[k] = 0; aws[k] = 0; awc[k] = 0; }
    sxx = sxw = sww = 0;
    fxx[0] = fxx[1] = fxw[0] = fxw[1] = fww[0] = fww[1] = 0.f;
  }

  // self-term accumulation: float64 products in the float64 form; float
  // products with Kahan compensation in the float32 form (no FP64 pipe use)
  __device__ __forceinline__ void self_add(int which, Tc a, Tc b) {
    if constexpr (F64) {
      double p = (double)a * (double)b;
      if (which == 0) sxx += p; else if (which == 1) sxw += p; else sww += p;
    } else {
      float p = (float)a * (float)b;
      if (which == 0) kahan(fxx[0], fxx[1], p);
      else if (which == 1) kahan(fxw[0], fxw[1], p);
      else kahan(fww[0], fww[1], p);
    }
  }

  __device__ __forceinline__ static void kahan(float& s, float& c, float v) {
    float y = v - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
  }

  __device__ __forceinline__ int slot(int z) const { return RING == 1 ? 0 : (z + 3) % 3; }

  // Project plane z (wrapped) of the tile into ring slot `sl`.  With `halo`,
  // the projection also covers the four one-point halo strips.  `own`: the
  // plane's interior belongs to this tile (stores and self terms happen).
  __device__ void project_plane(const PassT<B>& ps, int x0, int y0, int z, int w, int hg, int sl,
                                bool halo, bool own) {
    constexpr int QP = (NS * (TX * TY + 2 * TX + 2 * TY) + NT - 1) / NT;  // points per thread
    const DevOp& d = P.op;
    const int zw = wrapi(z, d.nz);
    const int pint = w * hg;
    const int pall = halo ? pint + 2 * w + 2 * hg : pint;
    const int total = NS * pall;
    const long long N = d.N;
    const B* Vb = reinterpret_cast<const B*>(P.V);
    Tc* ring = S.ring + sl * NS * PS;
    const Tc a = (Tc)ps.a;
    const bool unit = ps.a == 1.0;
    int gi[QP], so[QP];
    Tc x[QP];
#pragma unroll
    for (int u = 0; u < QP; ++u) {
      const int q = tid + u * NT;
      gi[u] = 0;
      so[u] = -1;
      x[u] = (Tc)0;
      if (q < total) {
        int s = q / pall;
        int r = q - s * pall;
        int lx, ly;
        if (r < pint) { ly = r / w; lx = r - ly * w; }
        else {
          int h = r - pint;
          if (h < w) { lx = h; ly = -1; }
          else if (h < 2 * w) { lx = h - w; ly = hg; }
          else if (h < 2 * w + hg) { lx = -1; ly = h - 2 * w; }
          else { lx = w; ly = h - 2 * w - hg; }
        }
        int gx = wrapi(x0 + lx, d.nx), gy = wrapi(y0 + ly, d.ny);
        gi[u] = (int)(s * d.npts + gx + (long long)d.nx * (gy + (long long)d.ny * zw));
        so[u] = s * PS + (ly + 1) * PW + lx + 1;
        if (r < pint && own) so[u] |= (1 << 30);   // owned interior point
        x[u] = ps.src64 ? (Tc)__ldg(ps.src64 + gi[u]) : (Tc)__ldcg(ps.srcB + gi[u]);
        if (!unit) x[u] = a * x[u];        // (a = 1: no float64 instruction)
      }
    }
    // x -= sum_c coef_c V_c : one coefficient load per column, applied to all
    // points; loads are issued in batches of CB columns before their FMAs so
    // that several round trips to L2/HBM overlap.  The float32 form keeps two
    // accumulators per point (halving the FMA dependency chain); the float64
    // form one (its pipe is throughput-bound, and the merge would be one more
    // float64 addition per point).
    constexpr int CB = F64 ? 4 : 8;
    Tc xb[QP];
#pragma unroll
    for (int u = 0; u < QP; ++u) xb[u] = (Tc)0;
    int c = ps.c0;
    for (; c + CB <= ps.c1; c += CB) {
      Tc v[CB][QP];
#pragma unroll
      for (int i = 0; i < CB; ++i) {
        const B* col = Vb + (long long)(c + i) * N;
#pragma unroll
        for (int u = 0; u < QP; ++u) v[i][u] = (Tc)__ldcg(col + gi[u]);
      }
#pragma unroll
      for (int i = 0; i < CB; ++i) {
        const Tc cc = S.coefc[c + i];
#pragma unroll
        for (int u = 0; u < QP; ++u) {
          if (!F64 && (i & 1)) xb[u] = fma(-cc, v[i][u], xb[u]);
          else x[u] = fma(-cc, v[i][u], x[u]);
        }
      }
    }
    for (; c < ps.c1; ++c) {
      const Tc cc = S.coefc[c];
      const B* col = Vb + (long long)c * N;
#pragma unroll
      for (int u = 0; u < QP; ++u) x[u] = fma(-cc, (Tc)__ldcg(col + gi[u]), x[u]);
    }
    if constexpr (!F64) {
#pragma unroll
      for (int u = 0; u < QP; ++u) x[u] += xb[u];
    }
#pragma unroll
    for (int u = 0; u < QP; ++u) {
      if (so[u] < 0) continue;
      Tc xv = x[u];
      if constexpr (!F64) xv = (Tc)(B)xv;   // the stencil sees exactly the stored value
      ring[so[u] & ((1 << 30) - 1)] = xv;
      if (so[u] & (1 << 30)) {
        if (ps.xout) ps.xout[gi[u]] = (B)xv;
        if (!ps.wout && (ps.self & SELF_XX)) self_add(0, xv, xv);
      }
    }
  }

  // First pass of the two-phase step: x = a*src - sum_c coef_c V_c on this
  // CTA's contiguous share of the N values (all species; equal shares, so
  // every CTA has the same work), stored to ps.xout; no halo, no shared
  // memory, no barrier.  Each value goes through the same operations in the
  // same order as in project_plane (CB-column batches, the float32 form's two
  // alternating accumulators, then the tail), so the stored x is bitwise the
  // value the one-pass step stores.
  __device__ void project_flat(const PassT<B>& ps) {
    constexpr int U = 4;                       // values per thread per round
    constexpr int CB = F64 ? 4 : 8;
    const long long N = P.op.N;
    long long per = (N + gsize - 1) / gsize;
    per = (per + 31) & ~31LL;                  // shares start on a 32-value boundary
    const long long e0 = (long long)grank * per;
    const long long e1 = min(N, e0 + per);
    const B* Vb = reinterpret_cast<const B*>(P.V);
    const Tc a = (Tc)ps.a;
    const bool unit = ps.a == 1.0;
    for (long long base = e0; base < e1; base += (long long)U * NT) {
      long long gi[U];
      Tc x[U], xb[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const long long q = base + tid + (long long)u * NT;
        gi[u] = q < e1 ? q : e0;               // out-of-share lanes re-read a valid value
        x[u] = ps.src64 ? (Tc)__ldg(ps.src64 + gi[u]) : (Tc)__ldcg(ps.srcB + gi[u]);
        if (!unit) x[u] = a * x[u];
        xb[u] = (Tc)0;
      }
      int c = ps.c0;
      for (; c + CB <= ps.c1; c += CB) {
        Tc v[CB][U];
#pragma unroll
        for (int i = 0; i < CB; ++i) {
          const B* col = Vb + (long long)(c + i) * N;
#pragma unroll
          for (int u = 0; u < U; ++u) v[i][u] = (Tc)__ldcg(col + gi[u]);
        }
#pragma unroll
        for (int i = 0; i < CB; ++i) {
          const Tc cc = S.coefc[c + i];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            if (!F64 && (i & 1)) xb[u] = fma(-cc, v[i][u], xb[u]);
            else x[u] = fma(-cc, v[i][u], x[u]);
          }
        }
      }
      for (; c < ps.c1; ++c) {
        const Tc cc = S.coefc[c];
        const B* col = Vb + (long long)c * N;
#pragma unroll
        for (int u = 0; u < U; ++u) x[u] = fma(-cc, (Tc)__ldcg(col + gi[u]), x[u]);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const long long q = base + tid + (long long)u * NT;
        if (q < e1) ps.xout[q] = F64 ? (B)x[u] : (B)(x[u] + xb[u]);
      }
    }
  }

  // Second pass of the flat two-phase step: this CTA's equal flat share of
  // the grid points (all species of a point together) in chunks of FCH
  // points.  Each thread forms w = A x at FQ points with the neighbours of x
  // read through L2 (x was stored by the first pass, before the grid barrier;
  // the grid is periodic in every direction, as in the tile passes), stores w
  // and adds the self terms; then the warps form the inner products with basis
  // columns (warp <-> columns, lane <-> points, as in dots_plane) from the
  // chunk's x and w in shared memory (xs, ws: NS*FCH values each).  No halo
  // copy, no tile chain: every CTA has the same number of points.  w is
  // bitwise the tile passes' value (the operator's own arithmetic on the
  // loaded values, staged with a row pitch of 2 and species 5 apart); the
  // inner products sum the points in other groups, so they agree with the
  // tile passes to rounding.
  static constexpr int FQ = 2, FCH = FQ * NT;
  static constexpr bool kFlatOp =
      Op::KIND == LSA_OP_ADR3D || Op::KIND == LSA_OP_ADVDIFF2D || Op::KIND == LSA_OP_GRAYSCOTT2D;
  __device__ int run_pass_flat(const PassT<B>& ps, Tc* xs, Tc* ws) {
    static_assert(kFlatOp, "the flat pass is written for the ADR 3D, advection-diffusion and Gray-Scott operators");
    const DevOp& d = P.op;
    const long long np = d.npts;               // grid points (N = NS * np)
    long long per = (np + gsize - 1) / gsize;
    per = (per + 31) & ~31LL;
    const long long e0 = (long long)grank * per;
    const long long e1 = min(np, e0 + per);
    const B* xg = ps.srcB;
    const int nxy = d.nx * d.ny;
    const bool dx = ps.dmode & DOT_X, dw = ps.dmode & DOT_W;
    zero_acc();
    for (long long base = e0; base < e1; base += FCH) {
#pragma unroll
      for (int u = 0; u < FQ; ++u) {
        const int pl = tid + u * NT;
        Tc xv[NS], wv[NS];
#pragma unroll
        for (int sp = 0; sp < NS; ++sp) { xv[sp] = (Tc)0; wv[sp] = (Tc)0; }
        if (base + pl < e1) {
          // grid indices in 32 bits, as in the tile passes (N < 2^31)
          const int q = (int)base + pl;
          const int r = q / d.nx, ix = q - r * d.nx;
          const int iz = r / d.ny, iy = r - iz * d.ny;
          const int qw = ix == 0 ? q + (d.nx - 1) : q - 1;
          const int qe = ix == d.nx - 1 ? q - (d.nx - 1) : q + 1;
          const int qs = iy == 0 ? q + (d.ny - 1) * d.nx : q - d.nx;
          const int qn = iy == d.ny - 1 ? q - (d.ny - 1) * d.nx : q + d.nx;
          // per species: [south, west, centre, east, north]; below and above at index 2
          Tc c5[5 * NS], zm[3], zp[3];
#pragma unroll
          for (int sp = 0; sp < NS; ++sp) {
            const B* xsp = xg + (long long)sp * np;
            c5[5 * sp + 0] = (Tc)__ldcg(xsp + qs);
            c5[5 * sp + 1] = (Tc)__ldcg(xsp + qw);
            c5[5 * sp + 2] = (Tc)__ldcg(xsp + q);
            c5[5 * sp + 3] = (Tc)__ldcg(xsp + qe);
            c5[5 * sp + 4] = (Tc)__ldcg(xsp + qn);
          }
          zm[0] = zm[1] = zp[0] = zp[1] = (Tc)0;
          if constexpr (DIM == 3) {
            zm[2] = (Tc)__ldcg(xg + (iz == 0 ? q + (d.nz - 1) * nxy : q - nxy));
            zp[2] = (Tc)__ldcg(xg + (iz == d.nz - 1 ? q - (d.nz - 1) * nxy : q + nxy));
          } else {
            zm[2] = zp[2] = (Tc)0;
          }
          Tc out[NS];
          Op::template apply<Tc, 2, 5>(d, cf, zm, c5, zp, 2, (long long)q, out);
#pragma unroll
          for (int sp = 0; sp < NS; ++sp) {
            Tc w = out[sp];
            if constexpr (!F64) w = (Tc)(B)w;
            const Tc x = c5[5 * sp + 2];
            ps.wout[(long long)sp * np + q] = (B)w;
            if (ps.self & SELF_XX) self_add(0, x, x);
            if (ps.self & SELF_XW) self_add(1, x, w);
            if (ps.self & SELF_WW) self_add(2, w, w);
            xv[sp] = x;
            wv[sp] = w;
          }
        }
#pragma unroll
        for (int sp = 0; sp < NS; ++sp) {
          xs[sp * FCH + pl] = xv[sp];
          ws[sp * FCH + pl] = wv[sp];
        }
      }
      __syncthreads();
      if (ps.d1 > ps.d0) {
        // lane l takes points l + 32k of the chunk, k < FCH/32, in groups of
        // 8, one species after the other
        constexpr int NPL = FCH / 32;
        const int nv = (int)min((long long)FCH, e1 - base);   // valid points of the chunk
#pragma unroll 1
        for (int sp = 0; sp < NS; ++sp) {
          const Tc* xsp = xs + sp * FCH;
          const Tc* wsp = ws + sp * FCH;
#pragma unroll
          for (int kk = 0; kk < KMAX; ++kk) {
            const int c = ps.d0 + warp + NW * kk;
            if (c >= ps.d1) break;
            const B* col = Vc(c) + (long long)sp * np + base;
            Tc v[NPL];
#pragma unroll
            for (int k = 0; k < NPL; ++k) {
              const int pl = lane + 32 * k;
              v[k] = (Tc)__ldcg(col + (pl < nv ? pl : 0));   // beyond the share: x = w = 0 there
            }
#pragma unroll
            for (int g = 0; g < NPL / 8; ++g) {
              if constexpr (F64) {
                double a = ax[kk], b = aw[kk];
#pragma unroll
                for (int k = 8 * g; k < 8 * g + 8; ++k) {
                  const int pl = lane + 32 * k;
                  if (dx) a = fma((double)v[k], (double)xsp[pl], a);
                  if (dw) b = fma((double)v[k], (double)wsp[pl], b);
                }
                ax[kk] = a;
                aw[kk] = b;
              } else {
                float px = 0.f, pw = 0.f;
#pragma unroll
                for (int k = 8 * g; k < 8 * g + 8; ++k) {
                  const int pl = lane + 32 * k;
                  px = fmaf((float)v[k], (float)xsp[pl], px);
                  pw = fmaf((float)v[k], (float)wsp[pl], pw);
                }
                if (dx) kahan(axs[kk], axc[kk], px);
                if (dw) kahan(aws[kk], awc[kk], pw);
              }
            }
          }
        }
      }
      __syncthreads();
    }
    return write_partials(ps);
  }

  // Stencil at plane z (interior only) from the ring: w = A x.
  __device__ void stencil_plane(const PassT<B>& ps, int x0, int y0, int z, int w, int hg) {
    const DevOp& d = P.op;
    if (tid >= w * hg) return;
    int ly = tid / w, lx = tid - ly * w;
    const Tc* zm = S.ring + slot(z - 1) * NS * PS;
    const Tc* z0 = S.ring + slot(z) * NS * PS;
    const Tc* zp = S.ring + slot(z + 1) * NS * PS;
    int o = (ly + 1) * PW + lx + 1;
    long long gpt = (x0 + lx) + (long long)d.nx * ((y0 + ly) + (long long)d.ny * z);
    Tc out[NS];
    Op::template apply<Tc>(d, cf, zm, z0, zp, o, gpt, out);
    if constexpr (AUG) {         // + B x_bot (augmented operator)
      const int p = P.naug;
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        double f = (double)out[s];
        for (int k = 0; k < p; ++k)
          f = fma(S.xi[k], __ldg(P.baug + (long long)(p - k) * d.N + s * d.npts + gpt), f);
        out[s] = (Tc)f;
      }
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      Tc wv = out[s];
      if constexpr (!F64) wv = (Tc)(B)wv;
      S.wbuf[s * TX * TY + tid] = wv;
      ps.wout[s * d.npts + gpt] = (B)wv;
      const Tc xs = z0[s * PS + o];
      if (ps.self & SELF_XX) self_add(0, xs, xs);
      if (ps.self & SELF_XW) self_add(1, xs, wv);
      if (ps.self & SELF_WW) self_add(2, wv, wv);
    }
  }

  // Inner products of basis columns [d0, d1) with the plane's x and/or w:
  // warp <-> columns, lane <-> interior points (species one after the other,
  // to bound the registers that hold the point values).
  __device__ void dots_plane(const PassT<B>& ps, int x0, int y0, int z, int w, int hg, int sl) {
    if (ps.d1 <= ps.d0) return;
    constexpr int NPS = (TX * TY + 31) / 32;   // points per lane and species
    const DevOp& d = P.op;
    const int pint = w * hg;
    const bool dx = ps.dmode & DOT_X, dw = ps.dmode & DOT_W;
#pragma unroll 1
    for (int s = 0; s < NS; ++s) {
      const Tc* xr = S.ring + sl * NS * PS + s * PS;
      Tc xv[NPS], wv[NPS];
      int gi[NPS];
#pragma unroll
      for (int k = 0; k < NPS; ++k) {
        int q = lane + 32 * k;
        if (q < pint) {
          int ly = q / w, lx = q - ly * w;
          xv[k] = xr[(ly + 1) * PW + lx + 1];
          wv[k] = dw ? S.wbuf[s * TX * TY + q] : (Tc)0;
          gi[k] = (int)(s * d.npts + (x0 + lx) + (long long)d.nx * ((y0 + ly) + (long long)d.ny * z));
        } else {
          xv[k] = 0; wv[k] = 0; gi[k] = 0;
        }
      }
      // columns of this warp: c = d0 + warp + NW*kk; the next column's values
      // are loaded while the current one is consumed
      Tc vb[2][NPS];
      {
        const int c = ps.d0 + warp;
        const B* base = Vc(c < ps.d1 ? c : ps.d0);
#pragma unroll
        for (int k = 0; k < NPS; ++k) vb[0][k] = (Tc)__ldcg(base + gi[k]);
      }
#pragma unroll
      for (int kk = 0; kk < KMAX; ++kk) {
        const int c = ps.d0 + warp + NW * kk;
        if (c >= ps.d1) break;
        const int cn = c + NW;
        if (kk + 1 < KMAX && cn < ps.d1) {
          const B* nb = Vc(cn);
#pragma unroll
          for (int k = 0; k < NPS; ++k) vb[(kk + 1) & 1][k] = (Tc)__ldcg(nb + gi[k]);
        }
        const Tc* v = vb[kk & 1];
        if constexpr (F64) {
          // straight into the per-column accumulators: every FP64 instruction
          // is a product term (the FP64 pipe is the bound; the independent
          // columns of a warp give the ILP)
          if (dx) {
            double a = ax[kk];
#pragma unroll
            for (int k = 0; k < NPS; ++k) a = fma((double)v[k], (double)xv[k], a);
            ax[kk] = a;
          }
          if (dw) {
            double a = aw[kk];
#pragma unroll
            for (int k = 0; k < NPS; ++k) a = fma((double)v[k], (double)wv[k], a);
            aw[kk] = a;
          }
        } else {
          float px = 0.f, pw = 0.f;
#pragma unroll
          for (int k = 0; k < NPS; ++k) {
            px = fmaf((float)v[k], (float)xv[k], px);
            pw = fmaf((float)v[k], (float)wv[k], pw);
          }
          if (dx) kahan(axs[kk], axc[kk], px);
          if (dw) kahan(aws[kk], awc[kk], pw);
        }
      }
    }
  }

  // -------------------------------------------------------------------------
  // Augmented operator (Eqs. 8-9).  The extra entries of a vector follow the
  // same pass formula as its grid points: x_bot = a*src_bot - sum_c coef_c
  // V_bot,c, and w_bot = K x_bot.  Every CTA forms them at the start of a pass
  // (p <= PMAX entries, O(p j) work) and the stencil adds B x_bot; CTA rank 0
  // adds their share to the inner products; the CTA that completes the pass's
  // reduction stores them (when all CTAs have read the source entries, so an
  // in-place pass is safe).
  __device__ __forceinline__ int col_of(const B* ptr) const {
    return (int)((ptr - reinterpret_cast<const B*>(P.V)) / P.op.N);
  }
  __device__ void aug_begin(const PassT<B>& ps) {
    const int p = P.naug;
    if (tid < p) {
      double x;
      if (ps.src64) {            // the start vector: exp(aug_t K) e_p, entry p-1-i = t^i / i!
        const int i = p - 1 - tid;
        double v = 1.0;
        for (int r = 1; r <= i; ++r) v *= P.aug_t / (double)r;
        x = ps.a * v;
      } else {
        x = ps.a * __ldcg(P.xaug + (long long)col_of(ps.srcB) * PMAX + tid);
      }
      for (int c = ps.c0; c < ps.c1; ++c)
        x = fma(-(double)S.coefc[c], __ldcg(P.xaug + (long long)c * PMAX + tid), x);
      S.xi[tid] = x;
    }
    if (tid == 0) {
      S.aug_xcol = ps.xout ? col_of(ps.xout) : -1;
      S.aug_wcol = ps.wout ? col_of(ps.wout) : -1;
    }
    __syncthreads();
    if (tid < p) S.xw[tid] = (tid + 1 < p) ? S.xi[tid + 1] : 0.0;
    __syncthreads();
  }
  // extra-entry share of (column c) . (x or w)
  __device__ double aug_dot(int c, const double* vec) const {
    double acc = 0.0;
    for (int k = 0; k < P.naug; ++k) {
      const double vc = (c == S.aug_xcol) ? S.xi[k] : __ldcg(P.xaug + (long long)c * PMAX + k);
      acc = fma(vc, vec[k], acc);
    }
    return acc;
  }
  __device__ double aug_self(int which) const {
    const double* a = which == 2 ? S.xw : S.xi;
    const double* b = which == 0 ? S.xi : S.xw;
    double acc = 0.0;
    for (int k = 0; k < P.naug; ++k) acc = fma(a[k], b[k], acc);
    return acc;
  }

  // One pass over all tiles of this CTA; writes the CTA's partial sums.
  // Returns the number of reduction slots used.
  __device__ int run_pass(const PassT<B>& ps) {
    const DevOp& d = P.op;
    const Tiling& tl = P.tl;
    zero_acc();
    if constexpr (AUG) aug_begin(ps);
    const bool stencil = ps.wout != nullptr;
    for (int t = grank; t < tl.ntiles; t += gsize) {
      int bx = t % tl.tiles_x;
      int rr = t / tl.tiles_x;
      int by = rr % tl.tiles_y;
      int bz = rr / tl.tiles_y;
      int x0 = bx * TX, y0 = by * TY, z0 = bz * tl.ZS;
      int w = min(TX, d.nx - x0), hg = min(TY, d.ny - y0), zl = min(tl.ZS, d.nz - z0);
      if (DIM == 3 && stencil) {
        project_plane(ps, x0, y0, z0 - 1, w, hg, slot(z0 - 1), false, false);
        project_plane(ps, x0, y0, z0, w, hg, slot(z0), true, true);
        for (int z = z0; z < z0 + zl; ++z) {
          bool inside = (z + 1 < z0 + zl);
          project_plane(ps, x0, y0, z + 1, w, hg, slot(z + 1), inside, inside);
          __syncthreads();
          stencil_plane(ps, x0, y0, z, w, hg);
          __syncthreads();
          dots_plane(ps, x0, y0, z, w, hg, slot(z));
        }
        __syncthreads();
      } else {
        for (int z = z0; z < z0 + zl; ++z) {
          project_plane(ps, x0, y0, z, w, hg, 0, stencil, true);
          __syncthreads();
          if (stencil) {
            stencil_plane(ps, x0, y0, z, w, hg);
            __syncthreads();
          }
          dots_plane(ps, x0, y0, z, w, hg, 0);
          __syncthreads();
        }
      }
    }
    return write_partials(ps);
  }

  // Per-CTA partial sums of a pass to HBM (dot slots, then the three self terms).
  __device__ int write_partials(const PassT<B>& ps) {
    static_assert(KMAX == 8, "the transposed warp sum below takes 2*KMAX = 16 values");
    const int nd = ps.d1 > ps.d0 ? ps.d1 - ps.d0 : 0;
    double* part = P.partials + (long long)grank * SLOTS;
    {
      // the warp's 2*KMAX column sums at once: value 2kk is x . V_c, 2kk+1 is
      // w . V_c for column c = d0 + warp + NW*kk; lanes 2k and 2k+1 get value k
      // (float32 form: the Kahan pairs reduced as compensated float32 pairs,
      // converted to float64 once)
      double r;
      if constexpr (F64) {
        double v[2 * KMAX];
#pragma unroll
        for (int kk = 0; kk < KMAX; ++kk) { v[2 * kk] = ax[kk]; v[2 * kk + 1] = aw[kk]; }
        r = warp_sum_many<2 * KMAX>(v);
      } else {
        float vs[2 * KMAX], ve[2 * KMAX];   // Kahan keeps sum = s - c: e = -c
#pragma unroll
        for (int kk = 0; kk < KMAX; ++kk) {
          vs[2 * kk] = axs[kk]; ve[2 * kk] = -axc[kk];
          vs[2 * kk + 1] = aws[kk]; ve[2 * kk + 1] = -awc[kk];
        }
        warp_sum_many_comp<2 * KMAX>(vs, ve);
        r = (double)vs[0] + (double)ve[0];
      }
      const int k = lane >> 1, kk = k >> 1, isw = k & 1;
      const int c = ps.d0 + warp + NW * kk;
      if ((lane & 1) == 0 && c < ps.d1) {
        if constexpr (AUG) {
          if (grank == 0) r += isw ? aug_dot(c, S.xw) : aug_dot(c, S.xi);
        }
        if (isw) part[nd + c - ps.d0] = (ps.dmode & DOT_W) ? r : 0.0;
        else part[c - ps.d0] = (ps.dmode & DOT_X) ? r : 0.0;
      }
    }
    {
      double r;                              // lane l: value l >> 3
      if constexpr (F64) {
        double t[4] = {sxx, sxw, sww, 0.0};
        r = warp_sum_many<4>(t);
      } else {
        float ts[4] = {fxx[0], fxw[0], fww[0], 0.f}, te[4] = {-fxx[1], -fxw[1], -fww[1], 0.f};
        warp_sum_many_comp<4>(ts, te);
        r = (double)ts[0] + (double)te[0];
      }
      if ((lane & 7) == 0 && lane < 24) S.bred[warp][lane >> 3] = r;
    }
    __syncthreads();
    if (tid < 3) {
      double acc = 0;
      for (int i = 0; i < NW; ++i) acc += S.bred[i][tid];
      if constexpr (AUG) {
        if (grank == 0 && (ps.self & (1 << tid))) acc += aug_self(tid);
      }
      part[2 * nd + tid] = acc;
    }
    return 2 * nd + 3;
  }

  // Last CTA: fixed-order reduction of all CTAs' partials into S.red.  Warp w
  // takes slots w, w+NW, ...; lane l sums CTAs l, l+32, ... in order (all its
  // loads are independent, so they are in flight together), then a fixed
  // butterfly combines the lanes: the result is deterministic for a given grid.
  __device__ void reduce_partials(int nslots) {
    const int G = gsize;
    for (int s = warp; s < nslots; s += NW) {
      const double* ps = P.partials + s;
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      int c = lane;
      for (; c + 96 < G; c += 128) {
        a0 += __ldcg(ps + (long long)c * SLOTS);
        a1 += __ldcg(ps + (long long)(c + 32) * SLOTS);
        a2 += __ldcg(ps + (long long)(c + 64) * SLOTS);
        a3 += __ldcg(ps + (long long)(c + 96) * SLOTS);
      }
      for (; c < G; c += 32) a0 += __ldcg(ps + (long long)c * SLOTS);
      double v = warp_sum((a0 + a1) + (a2 + a3));
      if (lane == 0) S.red[s] = v;
    }
    __syncthreads();
  }

  // Two-level form.  Level 1: the last CTA of group g (CTAs g*RG .. g*RG+gn-1)
  // sums the group's partials into gsum row g; level 2: the last group to
  // finish sums the group rows into S.red.  One thread per slot, so the loads
  // of a warp are contiguous; each thread adds its rows in index order, so the
  // result is deterministic for a given grid.
  __device__ void sum_rows(const double* src, int nrows, int nslots, double* dst, bool to_smem) {
    for (int s = tid; s < nslots; s += NT) {
      double acc = 0.0;
      int r = 0;
      for (; r < nrows; r += 16) {       // 16 loads in flight, then their sum in row order
        double v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = (r + i < nrows) ? __ldcg(src + (long long)(r + i) * SLOTS + s) : 0.0;
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (r + i < nrows) acc += v[i];
      }
      if (to_smem) dst[s] = acc;
      else __stcg(dst + s, acc);
    }
  }

  // SM-aware ranks.  CTAs that share an SM share its FP64 pipe and shared
  // memory bandwidth, so an SM's time is set by the tiles of all its CTAs.
  // Each CTA records its SM id; after one barrier it takes as rank its place
  // in the order (slot on its SM, SM id), so the CTAs of one SM are about
  // G / #SMs ranks apart and, with tiles dealt cyclically by rank, every SM's
  // tile count is within one of the mean.  The ranks are a permutation of
  // 0..G-1 and tiles and partials follow the rank, so the results do not
  // depend on where the CTAs were placed.  Returns false on a timeout.
  __device__ bool place() {
    if (tid == 0) {
      unsigned sm;
      asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
      unsigned slot = 0;
      if (sm < (unsigned)SMID_CAP) slot = atomicAdd(&P.ctl->sm_ctas[sm], 1u);
      else atomicExch(&P.ctl->place_off, 1);
      S.tmp[0][0] = (double)sm;
      S.tmp[0][1] = (double)slot;
    }
    const BarrierRef br{&P.ctl->p_arrive, &P.ctl->p_release, &P.ctl->abort_flag, &P.ctl->status};
    const int r = barrier_arrive(br, 0u, gsize, &S.flag, P.timeout_ns);
    if (r < 0) return false;
    if (r == 1) barrier_release(br, 0u);
    __syncthreads();
    if (warp == 0) {
      const unsigned sm = (unsigned)S.tmp[0][0], slot = (unsigned)S.tmp[0][1];
      int rank = 0;
      for (int s = lane; s < SMID_CAP; s += 32) {
        const unsigned c = __ldcg(&P.ctl->sm_ctas[s]);
        rank += (int)min(c, slot) + (((unsigned)s < sm && c > slot) ? 1 : 0);
      }
      rank = warp_sum(rank);
      if (lane == 0) S.flag = __ldcg(&P.ctl->place_off) ? (int)blockIdx.x : rank;
    }
    __syncthreads();
    grank = S.flag;
    __syncthreads();
    return true;
  }

  // Read the published control state into shared memory (all threads): the
  // next pass's coefficients and flags, and the hybrid step's lazy scales,
  // norm estimate, ||A v|| and reduction count, so that whichever CTA runs
  // the next step finds them here (no L2 round trip inside the step).
  __device__ void load_ctl(int ncoef, int trow = -1) {
    for (int c = tid; c < ncoef; c += NT) {
      S.coefc[c] = (Tc)__ldcg(&P.ctl->coef[c]);
      S.sig[c] = __ldcg(&P.ctl->sigma[c]);
    }
    if (tcache && trow > 0)
      for (int k = tid; k < trow; k += NT) small[trow * MMAX + k] = __ldcg(&P.T[trow * MMAX + k]);
    if (tid == 0) {
      S.a = (Tc)__ldcg(&P.ctl->a);
      S.done = __ldcg(&P.ctl->done);
      S.fallback_pending = __ldcg(&P.ctl->fallback_pending);
      S.nrm_est_c = __ldcg(&P.ctl->nrm_est);
      S.aw_prev_c = __ldcg(&P.ctl->aw_prev);
      S.syncs_c = __ldcg(&P.ctl->syncs);
    }
    __syncthreads();
  }

  // Barrier + reduction; `fn` runs in the last CTA with S.red filled.
  template <class Fn>
  __device__ bool reduce_step(unsigned& gen, int nslots, int ncoef_after, Fn fn, int trow = -1) {
    const BarrierRef br = arnoldi_barrier(P.ctl);
    int r;
    if (P.gsum == nullptr || gsize > RG * RG_MAX) {
      r = barrier_arrive(br, gen, gsize, &S.flag, P.timeout_ns);
      if (r == 1) reduce_partials(nslots);
    } else {
      const int grp = grank / RG, g0 = grp * RG;
      const int gn = min(RG, gsize - g0), ngr = (gsize + RG - 1) / RG;
      const int lead = counter_arrive(&P.ctl->g_arrive[grp], gen, gn, &S.flag);
      if (lead) sum_rows(P.partials + (long long)g0 * SLOTS, gn, nslots, P.gsum + (long long)grp * SLOTS, false);
      r = barrier_arrive(br, gen, ngr, &S.flag, P.timeout_ns, lead != 0);
      if (r == 1) {
        sum_rows(P.gsum, ngr, nslots, S.red, true);
        __syncthreads();
      }
    }
    if (r < 0) return false;
    if (r == 1) {
      if (AUG && tid < P.naug) {
        if (S.aug_xcol >= 0) P.xaug[(long long)S.aug_xcol * PMAX + tid] = S.xi[tid];
        if (S.aug_wcol >= 0) P.xaug[(long long)S.aug_wcol * PMAX + tid] = S.xw[tid];
      }
      fn();
      __syncthreads();
      if (tid == 0) atomicAdd(&P.ctl->barriers, 1);
      barrier_release(br, gen);
    }
    ++gen;
    load_ctl(ncoef_after, trow);
    return true;
  }

  // Grid barrier without a reduction (between the two passes of the
  // two-phase step), with the arrival structure of reduce_step.
  __device__ bool sync_only(unsigned& gen) {
    const BarrierRef br = arnoldi_barrier(P.ctl);
    int r;
    if (P.gsum == nullptr || gsize > RG * RG_MAX) {
      r = barrier_arrive(br, gen, gsize, &S.flag, P.timeout_ns);
    } else {
      const int grp = grank / RG, g0 = grp * RG;
      const int gn = min(RG, gsize - g0), ngr = (gsize + RG - 1) / RG;
      const int lead = counter_arrive(&P.ctl->g_arrive[grp], gen, gn, &S.flag);
      r = barrier_arrive(br, gen, ngr, &S.flag, P.timeout_ns, lead != 0);
    }
    if (r < 0) return false;
    if (r == 1) {
      if (tid == 0) atomicAdd(&P.ctl->barriers, 1);
      barrier_release(br, gen);
    }
    ++gen;
    return true;
  }

  __device__ __forceinline__ double& Hat(int r, int c) const { return P.H[r + (long long)c * (P.m + 1)]; }

  // -------------------------------------------------------------------------
  // Hybrid low-synchronisation step (Alg. 4 with Alg. 5/6/7), last CTA only.
  // S.red: x_i.x_j (i < j-1), x_i.w_j (i < j-1), x_j.x_j, x_j.w_j, w_j.w_j for the
  // stored (estimate-normalised) x and w = A x.
  __device__ void hybrid_step(int j) {
    Ctl* ctl = P.ctl;
    const int np = j - 1;
    double* temp1 = S.tmp[0];
    double* temp2 = S.tmp[1];
    double* hcol = S.tmp[2];
    double* aux = S.tmp[3];
    if (tid == 0) {
      double Gj = S.red[2 * np], Pj = S.red[2 * np + 1], Q = S.red[2 * np + 2];
      S.flag = 0;
      if (j == 1 && Gj == 0.0) {              // zero start vector: y = 0
        ctl->beta = 0.0;
        ctl->m_eff = 0;
        ctl->done = 1;
        S.flag = 1;
      } else if (!(Gj > 0.0) || !isfinite(Gj) || !isfinite(Pj) || !isfinite(Q)) {
        ctl->status = (int)LSA_ERR_NUMERIC;
        ctl->done = 1;
        ctl->m_eff = j - 1;
        S.flag = 1;
      } else {
        // one reciprocal square root for both 1/||x|| and ||x|| (a float64
        // warp instruction is slow on this GPU, and this thread is the
        // critical path of the step)
        const double sj = rsqrt(Gj);
        const double nx = Gj * sj;
        S.sj = sj;
        if (j == 1) {
          ctl->beta = nx;
        } else {
          const double ne_prev = S.nrm_est_c;
          const double aw_prev = S.aw_prev_c;
          double tn = ne_prev * nx;                        // true norm of the previous vector
          S.true_nrm = tn;
          if (!(tn > P.brk_tol * aw_prev)) {               // lagged breakdown test
            Hat(j - 1, j - 2) = tn;
            ctl->m_eff = j - 1;
            ctl->breakdown = 1;
            ctl->done = 1;
            S.flag = 1;
          }
        }
        ctl->sigma[j - 1] = sj;
        S.sig[j - 1] = sj;
        temp2[np] = sj * sj * Pj;
        temp2[np + 1] = sj * sj * Q;
      }
      ctl->syncs = ++S.syncs_c;
      if (cached && S.flag) S.done = 1;
    }
    __syncthreads();
    if (S.flag) return;
    for (int i = tid; i < np; i += NT) {
      double si = S.sig[i];
      temp1[i] = si * S.sj * S.red[i];
      temp2[i] = si * S.sj * S.red[np + i];
    }
    __syncthreads();
    if (j == 1) {
      if (tid == 0) hcol[0] = temp2[0];
    } else {
      // New row of T (Alg. 5: T_{j,1:j-1} = -temp_{1:j-1,1}^T T_{1:j-1,1:j-1};
      // Alg. 6: T_{j,1:j-1} = -temp_{1:j-1,1}^T; for Alg. 7 this is M^{-1}).
      if (!cached && !tcache) stage(P.T, np);   // else small already holds rows 0..np-1 of T
      if (P.variant != LSA_HNCWY) {
        // T_{j,k} = -temp1_k - sum_{i>k} temp1_i T_{i,k}: the four lanes
        // 4k..4k+3 (all eight warps) take the terms i = k+1+q, k+5+q, ...
        // and combine their sums in a fixed order (deterministic)
        static_assert(MMAX * 4 <= NT, "four lanes per column");
        const int k = tid >> 2, q = tid & 3;
        double a = 0.0;
        if (k < np)
          for (int i = k + 1 + q; i < np; i += 4) a = fma(-temp1[i], small[i * MMAX + k], a);
        a += __shfl_xor_sync(0xffffffffu, a, 1);
        a += __shfl_xor_sync(0xffffffffu, a, 2);
        if (k < np && q == 0) {
          const double acc = -temp1[k] + a;
          small[np * MMAX + k] = acc;
          P.T[np * MMAX + k] = acc;
        }
      } else {
        for (int k = tid; k < np; k += NT) {
          small[np * MMAX + k] = -temp1[k];
          P.T[np * MMAX + k] = -temp1[k];
        }
      }
      __syncthreads();
      if (P.variant != LSA_HGSMGS) {
        apply_unit_lower(temp2, hcol, j);                 // H_{1:j,j} = T_j temp_{1:j,2}
      } else {
        // Alg. 7: y = M^{-1} temp2; p = (I + N M^{-1}) temp2 = temp2 - L^T y;
        // H_{1:j,j} solves (I + L) x = p.
        apply_unit_lower(temp2, aux, j);                  // aux = y
        double* Lm = cached ? smallL : small;             // L (cached: kept between steps)
        if (!cached) stage(P.L, np);
        for (int k = tid; k < np; k += NT) {
          Lm[np * MMAX + k] = temp1[k];
          P.L[np * MMAX + k] = temp1[k];
        }
        __syncthreads();
        for (int r = tid; r < j; r += NT) {
          double acc = 0.0;
          for (int k = r + 1; k < j; ++k) acc = fma(Lm[k * MMAX + r], aux[k], acc);
          hcol[r] = temp2[r] - acc;
        }
        __syncthreads();
        if (warp == 0) {                                   // forward substitution
          for (int r = 0; r < j; ++r) {
            double acc = 0.0;
            for (int k = lane; k < r; k += 32) acc = fma(Lm[r * MMAX + k], hcol[k], acc);
            acc = warp_sum(acc);
            if (lane == 0) hcol[r] = hcol[r] - acc;
            __syncwarp();
          }
        }
      }
    }
    __syncthreads();
    for (int r = tid; r < j; r += NT) Hat(r, j - 1) = hcol[r];
    if (warp == 0) {
      double ss = 0.0;
      for (int i = lane; i < j; i += 32) ss = fma(temp2[i], temp2[i], ss);
      ss = warp_sum(ss);
      if (lane == 0) S.ss = ss;
    }
    __syncthreads();
    if (tid == 0) {
      if (j > 1) Hat(j - 1, j - 2) = S.true_nrm;
      double t = temp2[j];
      double awn = sqrt(t);
      S.scale = 1.0;
      bool done_now = false;
      if (t < S.ss) {                         // Pythagorean radicand negative: explicit norm
        ctl->fallbacks = __ldcg(&ctl->fallbacks) + 1;
        ctl->fallback_pending = 1;
        ctl->nrm_est = 1.0;
        S.nrm_est_c = 1.0;
        if (cached) S.fallback_pending = 1;
      } else {
        const double d = t - S.ss;            // Eq. 18: ne = sqrt(d), scale = 1/ne
        const double rd = (d > 0.0) ? rsqrt(d) : 0.0;
        const double ne = d * rd;
        if (!(ne > P.brk_tol * awn)) {
          Hat(j, j - 1) = ne;
          ctl->m_eff = j;
          ctl->breakdown = 1;
          ctl->done = 1;
          done_now = true;
        }
        ctl->nrm_est = ne;
        S.nrm_est_c = ne;
        S.scale = rd;
      }
      ctl->aw_prev = awn;
      S.aw_prev_c = awn;
      ctl->a = S.sj * S.scale;
      if (cached) {
        S.a = (Tc)(S.sj * S.scale);
        if (done_now) S.done = 1;
      }
      if (j == P.m && !done_now && !__ldcg(&ctl->done)) ctl->m_eff = P.m;
    }
    __syncthreads();
    for (int i = tid; i < j; i += NT) {
      double si = (i == j - 1) ? S.sj : S.sig[i];
      const double c = si * hcol[i] * S.scale;
      ctl->coef[i] = c;
      if (cached) S.coefc[i] = (Tc)c;
    }
  }

  // small[r][k] = M[r][k] for r < rows, k < r (strictly lower part), from global.
  // Eight loads per thread are issued before their stores, so their round trips
  // to L2 overlap (the step runs in one CTA while the others wait).
  __device__ void stage(const double* M, int rows) {
    constexpr int U = 8;
    const int total = rows * MMAX;
    for (int e0 = tid; e0 < total; e0 += U * NT) {
      double v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * NT;
        const int r = e / MMAX, k = e - r * MMAX;
        v[u] = (e < total && k < r) ? __ldcg(M + e) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * NT;
        const int r = e / MMAX, k = e - r * MMAX;
        if (e < total && k < r) small[e] = v[u];
      }
    }
    __syncthreads();
  }

  // out[r] = in[r] + sum_{k<r} small[r][k] in[k]  (unit lower-triangular times
  // vector), r < n: warp w takes rows w, w+NW, ..., then one transposed warp sum.
  __device__ void apply_unit_lower(const double* in, double* out, int n) {
    static_assert(MMAX <= 8 * NW, "eight rows per warp");
    double acc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int r = warp + NW * i;
      double a = 0.0;
      if (r < n)
        for (int k = lane; k < r; k += 32) a = fma(small[r * MMAX + k], in[k], a);
      acc[i] = a;
    }
    const double sum = warp_sum_many<8>(acc);   // lane l: row warp + NW*(l >> 2)
    const int r = warp + NW * (lane >> 2);
    if ((lane & 3) == 0 && r < n) out[r] = in[r] + sum;
    __syncthreads();
  }

  __device__ void hybrid_fallback_finish(int j) {
    Ctl* ctl = P.ctl;
    if (tid == 0) {
      double nrm = sqrt(S.red[0]);
      ctl->syncs = ++S.syncs_c;
      if (!(nrm > P.brk_tol * S.aw_prev_c)) {
        Hat(j, j - 1) = nrm;
        ctl->m_eff = j;
        ctl->breakdown = 1;
        ctl->done = 1;
        if (cached) S.done = 1;
      }
      ctl->nrm_est = nrm;
      S.nrm_est_c = nrm;
      S.scale = (nrm > 0.0) ? 1.0 / nrm : 0.0;
      ctl->a = (cached ? (double)S.a : __ldcg(&ctl->a)) * S.scale;
      ctl->fallback_pending = 0;
      if (cached) { S.a = (Tc)(S.a * S.scale); S.fallback_pending = 0; }
    }
    __syncthreads();
    for (int i = tid; i < j; i += NT) {
      const double c = (cached ? (double)S.coefc[i] : __ldcg(&ctl->coef[i])) * S.scale;
      ctl->coef[i] = c;
      if (cached) S.coefc[i] = (Tc)c;
    }
  }

  __device__ void hybrid_final_finish() {
    Ctl* ctl = P.ctl;
    if (tid == 0) {
      const int m = P.m;
      double nrm = sqrt(S.red[0]);
      double hl = S.nrm_est_c * nrm;   // true norm of the projected v_{m+1}
      Hat(m, m - 1) = hl;
      ctl->h_last = hl;
      ctl->sigma[m] = (nrm > 0.0) ? 1.0 / nrm : 0.0;
      ctl->syncs = ++S.syncs_c;
      if (!(hl > P.brk_tol * S.aw_prev_c)) ctl->breakdown = 1;
    }
  }

  // -------------------------------------------------------------------------
  // Hybrid low-synchronisation Arnoldi (Alg. 4).  Storage: column j-1 holds
  // x_j = u_j / nrm_est_{j-1} (u_j the projected vector); the normalised
  // v_j = sigma_j x_j with sigma_j = 1/||x_j|| known after step j.  All the
  // rescalings of Alg. 4 are folded into the scalars a, coef and sigma.
  // kFlat: the instantiation of k_arnoldi_flat, whose two-phase step runs
  // run_pass_flat after the flat projection (fbuf: 2*NS*FCH values of shared
  // memory); the other kernels carry none of its code.
  template <bool kFlat = false>
  __device__ void run_hybrid(Tc* fbuf = nullptr) {
    B* V = reinterpret_cast<B*>(P.V);
    B* Wb[2] = {reinterpret_cast<B*>(P.W0), reinterpret_cast<B*>(P.W1)};
    const long long N = P.op.N;
    const int m = P.m;
    unsigned gen = 0;
    if (tid == 0) { S.a = (Tc)1; S.done = 0; S.fallback_pending = 0; S.syncs_c = 0; }
    __syncthreads();
    // Two-phase form: a pass over equal flat shares projects x_j (no halo),
    // a grid barrier, then the tile pass reads x_j back with its halo for
    // w_j = A x_j and the inner products.  Every value goes through the same
    // operations in the same order as in the one-pass form.
    const bool two = P.two_phase != 0 && !AUG && !cached;
    tcache = !cached && P.variant != LSA_HGSMGS;
    for (int j = 1; j <= m; ++j) {
      PassT<B> ps;
      ps.c0 = 0; ps.c1 = j - 1;
      ps.a = (j == 1) ? 1.0 : (double)S.a;
      ps.src64 = (j == 1) ? P.vin : nullptr;
      ps.srcB = (j == 1) ? nullptr : Wb[(j - 1) & 1];
      ps.xout = V + (long long)(j - 1) * N;
      ps.wout = Wb[j & 1];
      ps.d0 = 0; ps.d1 = j - 1;
      ps.dmode = DOT_X | DOT_W;
      ps.self = SELF_XX | SELF_XW | SELF_WW;
      if (two) {
        project_flat(ps);                      // x_j (no halo)
        if (!sync_only(gen)) return;
        ps.c0 = ps.c1 = 0;                     // then x_j with its halo, w_j = A x_j, the products
        ps.a = 1.0;
        ps.src64 = nullptr;
        ps.srcB = ps.xout;
        ps.xout = nullptr;
      }
      int ns;
      if constexpr (kFlat) ns = two ? run_pass_flat(ps, fbuf, fbuf + NS * FCH) : run_pass(ps);
      else ns = run_pass(ps);
      if (!reduce_step(gen, ns, j, [&] { hybrid_step(j); }, j - 1)) return;
      if (S.done) return;
      if (S.fallback_pending) {
        // explicit norm of the projected vector (extra reduction of Alg. 4)
        PassT<B> pf;
        pf.c0 = 0; pf.c1 = j; pf.a = (double)S.a;
        pf.src64 = nullptr; pf.srcB = Wb[j & 1];
        pf.xout = nullptr; pf.wout = nullptr;
        pf.d0 = 0; pf.d1 = 0; pf.dmode = 0; pf.self = SELF_XX;
        int nf = run_pass(pf);
        if (!reduce_step(gen, nf, j, [&] { hybrid_fallback_finish(j); })) return;
        if (S.done) return;
      }
    }
    // final projection of v_{m+1} and its norm (one more reduction)
    PassT<B> pl;
    pl.c0 = 0; pl.c1 = m; pl.a = (double)S.a;
    pl.src64 = nullptr; pl.srcB = Wb[m & 1];
    pl.xout = V + (long long)m * N; pl.wout = nullptr;
    pl.d0 = 0; pl.d1 = 0; pl.dmode = 0; pl.self = SELF_XX;
    int nl = run_pass(pl);
    reduce_step(gen, nl, 0, [&] { hybrid_final_finish(); });
  }

  // -------------------------------------------------------------------------
  // Shared pieces of MGS and CGS2: ||v|| and the "next vector" pass.
  __device__ bool norm_of_input(unsigned& gen) {
    PassT<B> ps;
    ps.c0 = ps.c1 = 0; ps.a = 1.0; ps.src64 = P.vin; ps.srcB = nullptr;
    ps.xout = nullptr; ps.wout = nullptr; ps.d0 = ps.d1 = 0; ps.dmode = 0; ps.self = SELF_XX;
    int ns = run_pass(ps);
    return reduce_step(gen, ns, 0, [&] {
      if (tid == 0) {
        double b = sqrt(S.red[0]);
        P.ctl->beta = b;
        P.ctl->syncs = __ldcg(&P.ctl->syncs) + 1;
        if (b == 0.0) { P.ctl->done = 1; P.ctl->m_eff = 0; }     // zero start vector: y = 0
        else if (!isfinite(b)) { P.ctl->done = 1; P.ctl->status = (int)LSA_ERR_NUMERIC; }
        P.ctl->a = (b > 0.0) ? 1.0 / b : 0.0;
        for (int i = 0; i <= P.m; ++i) P.ctl->sigma[i] = 1.0;
      }
    });
  }

  // write v_{m+1} = a * w (no reduction): only for the Arnoldi output
  __device__ void write_last(B* dst, const B* src) {
    PassT<B> ps;
    ps.c0 = ps.c1 = 0; ps.a = (double)S.a; ps.src64 = nullptr; ps.srcB = src;
    ps.xout = dst; ps.wout = nullptr; ps.d0 = ps.d1 = 0; ps.dmode = 0; ps.self = 0;
    run_pass(ps);
  }

  // Alg. 1: Arnoldi with modified Gram-Schmidt (j+1 reductions at step j).
  __device__ void run_mgs(bool write_vlast) {
    B* V = reinterpret_cast<B*>(P.V);
    B* Wb[2] = {reinterpret_cast<B*>(P.W0), reinterpret_cast<B*>(P.W1)};
    const long long N = P.op.N;
    const int m = P.m;
    unsigned gen = 0;
    if (!norm_of_input(gen)) return;
    if (S.done) return;
    for (int j = 1; j <= m; ++j) {
      B* w = Wb[j & 1];
      // v_j = a * (previous w or b); w = A v_j; v_1 . w; ||w||^2
      PassT<B> pa;
      pa.c0 = pa.c1 = 0; pa.a = (double)S.a;
      pa.src64 = (j == 1) ? P.vin : nullptr;
      pa.srcB = (j == 1) ? nullptr : Wb[(j - 1) & 1];
      pa.xout = V + (long long)(j - 1) * N; pa.wout = w;
      pa.d0 = 0; pa.d1 = (j > 1) ? 1 : 0; pa.dmode = DOT_W;
      pa.self = SELF_XW | SELF_WW;
      int ns = run_pass(pa);
      if (!reduce_step(gen, ns, 1, [&] {
            if (tid == 0) {
              const int nd = (j > 1) ? 1 : 0;
              // H_{1,j} = v_1 . w: the W slot of column 0, or x.w when v_1 = x
              double h = (j > 1) ? S.red[nd] : S.red[2 * nd + 1];
              Hat(0, j - 1) = h;
              P.ctl->coef[0] = h;
              P.ctl->aw_prev = sqrt(S.red[2 * nd + 2]);
              P.ctl->syncs = __ldcg(&P.ctl->syncs) + 1;
            }
          })) return;
      for (int i = 1; i < j; ++i) {
        // w -= H_{i,j} v_i ; v_{i+1} . w
        PassT<B> pu;
        pu.c0 = i - 1; pu.c1 = i; pu.a = 1.0; pu.src64 = nullptr; pu.srcB = w;
        pu.xout = w; pu.wout = nullptr;
        pu.d0 = i; pu.d1 = i + 1; pu.dmode = DOT_X; pu.self = 0;
        int nu = run_pass(pu);
        if (!reduce_step(gen, nu, i + 1, [&] {
              if (tid == 0) {
                double h = S.red[0];
                Hat(i, j - 1) = h;
                P.ctl->coef[i] = h;
                P.ctl->syncs = __ldcg(&P.ctl->syncs) + 1;
              }
            })) return;
      }
      // w -= H_{j,j} v_j ; ||w||
      PassT<B> pz;
      pz.c0 = j - 1; pz.c1 = j; pz.a = 1.0; pz.src64 = nullptr; pz.srcB = w;
      pz.xout = w; pz.wout = nullptr; pz.d0 = pz.d1 = 0; pz.dmode = 0; pz.self = SELF_XX;
      int nz = run_pass(pz);
      if (!reduce_step(gen, nz, 0, [&] { finish_norm(j); })) return;
      if (S.done) return;
    }
    if (write_vlast) write_last(V + (long long)m * N, Wb[m & 1]);
  }

  __device__ void finish_norm(int j) {
    if (tid == 0) {
      Ctl* ctl = P.ctl;
      double nrm = sqrt(S.red[0]);
      Hat(j, j - 1) = nrm;
      ctl->syncs = cached ? ++S.syncs_c : __ldcg(&ctl->syncs) + 1;
      if (!(nrm > P.brk_tol * __ldcg(&ctl->aw_prev))) {
        ctl->m_eff = j;
        ctl->breakdown = 1;
        ctl->done = 1;
      }
      if (!isfinite(nrm)) { ctl->status = (int)LSA_ERR_NUMERIC; ctl->done = 1; ctl->m_eff = j - 1; }
      ctl->a = (nrm > 0.0) ? 1.0 / nrm : 0.0;
      ctl->h_last = nrm;
      if (j == P.m && !__ldcg(&ctl->done)) ctl->m_eff = P.m;
    }
  }

  // Classical Gram-Schmidt twice (3 reductions per step).
  __device__ void run_cgs2(bool write_vlast) {
    B* V = reinterpret_cast<B*>(P.V);
    B* Wb[2] = {reinterpret_cast<B*>(P.W0), reinterpret_cast<B*>(P.W1)};
    const long long N = P.op.N;
    const int m = P.m;
    unsigned gen = 0;
    if (!norm_of_input(gen)) return;
    if (S.done) return;
    for (int j = 1; j <= m; ++j) {
      B* w = Wb[j & 1];
      PassT<B> pa;
      pa.c0 = pa.c1 = 0; pa.a = (double)S.a;
      pa.src64 = (j == 1) ? P.vin : nullptr;
      pa.srcB = (j == 1) ? nullptr : Wb[(j - 1) & 1];
      pa.xout = V + (long long)(j - 1) * N; pa.wout = w;
      pa.d0 = 0; pa.d1 = j - 1; pa.dmode = DOT_W;
      pa.self = SELF_XW | SELF_WW;
      int ns = run_pass(pa);
      if (!reduce_step(gen, ns, j, [&] {
            const int nd = j - 1;
            for (int i = tid; i < j; i += NT) {
              double h = (i < nd) ? S.red[nd + i] : S.red[2 * nd + 1];
              P.ctl->hcol[i] = h;
              P.ctl->coef[i] = h;
            }
            if (tid == 0) { P.ctl->aw_prev = sqrt(S.red[2 * nd + 2]); P.ctl->syncs = __ldcg(&P.ctl->syncs) + 1; }
          })) return;
      PassT<B> pb;
      pb.c0 = 0; pb.c1 = j; pb.a = 1.0; pb.src64 = nullptr; pb.srcB = w;
      pb.xout = w; pb.wout = nullptr; pb.d0 = 0; pb.d1 = j; pb.dmode = DOT_X; pb.self = 0;
      int nb = run_pass(pb);
      if (!reduce_step(gen, nb, j, [&] {
            for (int i = tid; i < j; i += NT) {
              double h2 = S.red[i];
              Hat(i, j - 1) = __ldcg(&P.ctl->hcol[i]) + h2;
              P.ctl->coef[i] = h2;
            }
            if (tid == 0) P.ctl->syncs = __ldcg(&P.ctl->syncs) + 1;
          })) return;
      PassT<B> pc;
      pc.c0 = 0; pc.c1 = j; pc.a = 1.0; pc.src64 = nullptr; pc.srcB = w;
      pc.xout = w; pc.wout = nullptr; pc.d0 = pc.d1 = 0; pc.dmode = 0; pc.self = SELF_XX;
      int nc = run_pass(pc);
      if (!reduce_step(gen, nc, 0, [&] { finish_norm(j); })) return;
      if (S.done) return;
    }
    if (write_vlast) write_last(V + (long long)m * N, Wb[m & 1]);
  }

  // Incomplete orthogonalisation (Sect. 2.3.1, the paper's baseline ioCGS):
  // A v_j against v_{j-1} and v_j only, classically -- both inner products in
  // one reduction, then the norm (2 reductions per step).
  __device__ void run_iocgs(bool write_vlast) {
    B* V = reinterpret_cast<B*>(P.V);
    B* Wb[2] = {reinterpret_cast<B*>(P.W0), reinterpret_cast<B*>(P.W1)};
    const long long N = P.op.N;
    const int m = P.m;
    unsigned gen = 0;
    if (!norm_of_input(gen)) return;
    if (S.done) return;
    for (int j = 1; j <= m; ++j) {
      B* w = Wb[j & 1];
      const int lo = j >= 2 ? j - 2 : 0;   // columns lo..j-1: v_{j-1} (if any), v_j
      // v_j = a * (previous w or b); w = A v_j; v_{j-1} . w; v_j . w; ||w||^2
      PassT<B> pa;
      pa.c0 = pa.c1 = 0; pa.a = (double)S.a;
      pa.src64 = (j == 1) ? P.vin : nullptr;
      pa.srcB = (j == 1) ? nullptr : Wb[(j - 1) & 1];
      pa.xout = V + (long long)(j - 1) * N; pa.wout = w;
      pa.d0 = lo; pa.d1 = j - 1; pa.dmode = DOT_W;
      pa.self = SELF_XW | SELF_WW;
      int ns = run_pass(pa);
      if (!reduce_step(gen, ns, j, [&] {
            const int nd = j - 1 - lo;
            for (int i = lo + tid; i < j; i += NT) {
              double h = (i < j - 1) ? S.red[nd + i - lo] : S.red[2 * nd + 1];
              Hat(i, j - 1) = h;
              P.ctl->coef[i] = h;
            }
            if (tid == 0) { P.ctl->aw_prev = sqrt(S.red[2 * nd + 2]); P.ctl->syncs = __ldcg(&P.ctl->syncs) + 1; }
          })) return;
      // w -= H_{lo..j,j} v_{lo..j}; ||w||
      PassT<B> pc;
      pc.c0 = lo; pc.c1 = j; pc.a = 1.0; pc.src64 = nullptr; pc.srcB = w;
      pc.xout = w; pc.wout = nullptr; pc.d0 = pc.d1 = 0; pc.dmode = 0; pc.self = SELF_XX;
      int nc = run_pass(pc);
      if (!reduce_step(gen, nc, 0, [&] { finish_norm(j); })) return;
      if (S.done) return;
    }
    if (write_vlast) write_last(V + (long long)m * N, Wb[m & 1]);
  }
};

#ifndef LSA_MINB_F64
#define LSA_MINB_F64 2
#endif
#ifndef LSA_MINB_F32
#define LSA_MINB_F32 2
#endif

template <class Op, class Tc, class B, bool AUG = false>
__global__ void __launch_bounds__(NT, (sizeof(Tc) == 8) ? LSA_MINB_F64 : LSA_MINB_F32)
    k_arnoldi(ArnoldiParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using E = Engine<Op, Tc, B, AUG>;
  typename E::Smem& S = *reinterpret_cast<typename E::Smem*>(smem_raw);
  E e(P, S, reinterpret_cast<double*>(smem_raw + E::small_offset()));
  if (!e.place()) return;
  if (P.variant == LSA_MGS) e.run_mgs(P.write_vlast != 0);
  else if (P.variant == LSA_CGS2) e.run_cgs2(P.write_vlast != 0);
  else if (P.variant == LSA_IOCGS) e.run_iocgs(P.write_vlast != 0);
  else e.run_hybrid();
}

// The hybrid variants with the flat two-phase step (the ADR 3D,
// advection-diffusion and Gray-Scott operators): a separate instantiation
// with 2*NS*FCH values of extra shared memory.
template <class Op, class Tc>
__global__ void __launch_bounds__(NT, (sizeof(Tc) == 8) ? LSA_MINB_F64 : LSA_MINB_F32)
    k_arnoldi_flat(ArnoldiParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using E = Engine<Op, Tc, Tc>;
  typename E::Smem& S = *reinterpret_cast<typename E::Smem*>(smem_raw);
  E e(P, S, reinterpret_cast<double*>(smem_raw + E::small_offset()));
  if (!e.place()) return;
  e.template run_hybrid<true>(reinterpret_cast<Tc*>(smem_raw + E::smem_bytes()));
}

template <class Op, class Tc>
size_t flat_smem_bytes() {
  return Engine<Op, Tc, Tc>::smem_bytes() + 2 * Op::NS * Engine<Op, Tc, Tc>::FCH * sizeof(Tc);
}

// One stencil pass y = A x with the same tile code (no barrier).
template <class Op, class Tc, class B>
__global__ void __launch_bounds__(NT) k_matvec(ArnoldiParams P, const B* x, B* y) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using E = Engine<Op, Tc, B>;
  typename E::Smem& S = *reinterpret_cast<typename E::Smem*>(smem_raw);
  E e(P, S, reinterpret_cast<double*>(smem_raw + E::small_offset()));
  if (threadIdx.x == 0) S.a = (Tc)1;
  __syncthreads();
  PassT<B> ps;
  ps.c0 = ps.c1 = 0; ps.a = 1.0; ps.src64 = nullptr; ps.srcB = x;
  ps.xout = nullptr; ps.wout = y; ps.d0 = ps.d1 = 0; ps.dmode = 0; ps.self = 0;
  e.run_pass(ps);
}

template <class Op, class Tc>
cudaError_t launch_arnoldi_t(const ArnoldiParams& P, int G, cudaStream_t s) {
  ArnoldiParams Pc = P;
  void* args[1] = {&Pc};
  auto k = k_arnoldi<Op, Tc, Tc>;
  if constexpr (sizeof(Tc) == 8 && Op::KIND <= LSA_OP_ADR3D) {   // the three workload operators
    if (P.naug > 0) k = k_arnoldi<Op, Tc, Tc, true>;
  }
  size_t sm = Engine<Op, Tc, Tc>::smem_bytes();
  if constexpr (Engine<Op, Tc, Tc>::kFlatOp) {
    if (P.two_phase == 2 && P.naug == 0 && is_hybrid(P.variant)) {
      k = k_arnoldi_flat<Op, Tc>;
      sm = flat_smem_bytes<Op, Tc>();
    }
  }
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  return cudaLaunchCooperativeKernel((void*)k, dim3(G), dim3(NT), args, sm, s);
}

template <class Op, class Tc>
cudaError_t launch_matvec_t(const ArnoldiParams& P, const void* x, void* y, int G, cudaStream_t s) {
  auto k = k_matvec<Op, Tc, Tc>;
  size_t sm = Engine<Op, Tc, Tc>::smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k<<<G, NT, sm, s>>>(P, (const Tc*)x, (Tc*)y);
  return cudaGetLastError();
}

template <class Op, class Tc>
int blocks_per_sm_t() {
  int nb = 0;
  auto k = k_arnoldi<Op, Tc, Tc>;
  size_t sm = Engine<Op, Tc, Tc>::smem_bytes();
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, NT, sm);
  return nb;
}

template <class Op>
cudaError_t launch_arnoldi_op(const ArnoldiParams& P, int precision, int G, cudaStream_t s) {
  return precision == LSA_FP64 ? launch_arnoldi_t<Op, double>(P, G, s) : launch_arnoldi_t<Op, float>(P, G, s);
}

template <class Op>
cudaError_t launch_matvec_op(const ArnoldiParams& P, int precision, const void* x, void* y, int G,
                             cudaStream_t s) {
  return precision == LSA_FP64 ? launch_matvec_t<Op, double>(P, x, y, G, s)
                               : launch_matvec_t<Op, float>(P, x, y, G, s);
}

// Resident CTAs per SM of the flat two-phase kernel (0 where it does not exist).
template <class Op, class Tc>
int flat_blocks_per_sm_t() {
  int nb = 0;
  if constexpr (Engine<Op, Tc, Tc>::kFlatOp) {
    auto k = k_arnoldi_flat<Op, Tc>;
    size_t sm = flat_smem_bytes<Op, Tc>();
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, NT, sm);
  }
  return nb;
}

template <class Op>
int flat_blocks_per_sm_op(int precision) {
  return precision == LSA_FP64 ? flat_blocks_per_sm_t<Op, double>() : flat_blocks_per_sm_t<Op, float>();
}

template <class Op>
int blocks_per_sm_op(int precision) {
  return precision == LSA_FP64 ? blocks_per_sm_t<Op, double>() : blocks_per_sm_t<Op, float>();
}

}  // namespace lsa
