// TMA-staged hybrid Arnoldi kernel (float32 basis, whenever the stage
// buffers fit in shared memory and the grid meets the TMA alignment rules).
//
// Same mathematics as the hybrid passes of lsa_engine.cuh (Alg. 4 with the
// corrections of Algs. 5/6/7); what changes is how a pass reads the basis.
// A pass is a sequence of plane tasks per CTA (2D: one per tile; 3D: the
// planes of a z-segment plus one halo plane on each side).  For every task the
// CTA stages all basis columns the task needs into shared memory with a few
// large cp.async.bulk.tensor (TMA) boxes, each covering 8, 4, 2 or 1
// consecutive columns: the 16x16 tile together with its two y-halo rows
// (one 16x18 box), and the two x-halo columns (16-byte-wide boxes; the halo
// value is their last / first element).  Tiles whose y-halo wraps around the
// periodic boundary load the 16x16 interior and the two halo rows separately.
// Completion is counted on one mbarrier per stage.  A ring of three stage
// buffers keeps the next one or two tasks' copies in flight while the current
// task computes.
//
// In 3D the inner products of plane z are formed one task later (after the
// stencil of plane z, which needs the projection of plane z+1); the stage of
// plane z is kept until then, hence three buffers and a prefetch depth of two.
//
// Every wait is bounded (globaltimer); on expiry the CTA sets the abort flag
// and LSA_ERR_TIMEOUT, waits (bounded) for its own copies in flight, and leaves.
#pragma once

#include <cuda.h>
#include <string.h>

#include "lsa_engine.cuh"

namespace lsa {

constexpr int TYH = TY + 2;   // rows of the tile-plus-y-halo box

// Boxes over the extended basis tensor (x, y, zz, col); index q of each array
// covers cbq(q) = 32, 16, 8, 4, 2, 1 columns.
constexpr int NQ = 6;
struct TmaMaps {
  CUtensorMap mA[NQ];   // (TX, TY+2, NZB, cb): tile with both y-halo rows
  CUtensorMap mB[NQ];   // (TX, TY, NZB, cb):   tile only
  CUtensorMap mY[NQ];   // (TX, 1, NZB, cb):    one y-halo row
  CUtensorMap mX[NQ];   // (16 bytes, TY, NZB, cb): x-halo column and its 16-byte neighbourhood
  CUtensorMap mF0;      // operator field 0; box (TX, TY[, 1])
  CUtensorMap mF1;      // operator field 1
};

__host__ __device__ constexpr int cbq(int q) { return 32 >> q; }

struct TmaParams {
  int ncap;          // bulk column slots per stage buffer (even)
  int stage_bytes;
  int wcol;          // column index of the first matvec buffer in the extended basis (m + 1)
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void tma_load_4d(unsigned dst, const CUtensorMap* map, int x, int y,
                                            int z, int c, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(c), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(unsigned dst, const CUtensorMap* map, int x, int y,
                                            int z, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_load_2d(unsigned dst, const CUtensorMap* map, int x, int y,
                                            unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Stage buffer layout (bytes).  Bulk columns 0..ncp-1 occupy region A (and X);
// the source column has its own region S.  Region A per column:
//   full tile  : [NZB][TY+2][TX]        (rows 0 and TY+1 are the y-halo rows)
//   wrap tile  : [NZB][TY][TX] for all columns, then the low halo rows
//                [col][NZB][TX], then the high halo rows [col][NZB][TX]
// Region X per column: low side [NZB][TY][XW], high side likewise (XW = 16 bytes).
template <class Op, class Tc, class B>
struct TmaLayout {
  static constexpr int NS = Op::NS, DIM = Op::DIM, NF = Op::NF;
  static constexpr int NZB = (DIM == 3) ? 1 : NS;     // species ride in the box's z extent (2D)
  static constexpr int ES = sizeof(B);
  static constexpr int XW = 16 / ES;                  // x-halo box width (16 bytes)
  static constexpr int COLA = NZB * TYH * TX * ES;    // full-tile column bytes
  static constexpr int COLB = NZB * TY * TX * ES;     // tile-only column bytes
  static constexpr int COLY = NZB * TX * ES;          // one halo row, per column
  static constexpr int COLX = NZB * TY * XW * ES;     // one x-halo box, per column
  static constexpr int FBOX = TY * TX * ES;
  static constexpr int FB = (FBOX + 127) / 128 * 128;
  static constexpr int SYR = (COLY + 127) / 128 * 128;  // source y-halo row slots (128-aligned)
  static constexpr int SA0 = (COLA + 127) / 128 * 128;
  static constexpr int SA = SA0 > COLB + 2 * SYR ? SA0 : COLB + 2 * SYR;   // source tile slot
  static constexpr int SX = (COLX + 127) / 128 * 128;
  static __host__ __device__ int offX(int ncap) { return ncap * COLA; }
  static __host__ __device__ int offS(int ncap) { return offX(ncap) + 2 * ncap * COLX; }
  static __host__ __device__ int offF(int ncap) { return offS(ncap) + SA + 2 * SX; }
  static __host__ __device__ int stage_bytes(int ncap) { return offF(ncap) + NF * FB; }
  static __host__ __device__ size_t head_bytes() {
    return (Engine<Op, Tc, B>::small_offset() + 128 + 127) & ~(size_t)127;  // Smem + 3 mbarriers
  }
  static __host__ __device__ size_t smem_bytes(int ncap) {
    size_t st = (size_t)3 * stage_bytes(ncap);
    size_t mn = sizeof(double) * MMAX * MMAX;             // the last CTA's scratch aliases the stages
    return head_bytes() + (st > mn ? st : mn);
  }
  static __host__ __device__ int ncap_for(int m) { return (m + 1) & ~1; }   // even, >= m
};

// What one pass of the staged kernel does.
struct TmaPass {
  int ncp;           // projection columns 0..ncp-1
  int src_col;       // column of the source vector in the extended basis
  double a;          // source scale
  int xout_col;      // column written with x (-1: none)
  int wout_col;      // column written with w = A x (-1: no stencil)
  int self;          // SELF_* bits
};

template <class Op, class Tc, class B>
struct TmaEngine {
  using E = Engine<Op, Tc, B>;
  using LY = TmaLayout<Op, Tc, B>;
  static constexpr int NS = Op::NS, DIM = Op::DIM, NF = Op::NF, NZB = LY::NZB, ES = LY::ES;
  static constexpr bool F64 = sizeof(Tc) == 8;

  E& e;
  const TmaMaps& maps;
  const TmaParams tp;
  unsigned char* stages;
  unsigned bar0;         // shared address of the first of three mbarriers
  unsigned phases = 0;   // parity of the next wait, per stage
  int ntask = 0, tpt = 1, lag = 0, depth = 3;

  __device__ TmaEngine(E& en, const TmaMaps& m, const TmaParams& t, unsigned char* st, unsigned b)
      : e(en), maps(m), tp(t), stages(st), bar0(b) {}

  __device__ __forceinline__ unsigned char* stage(int s) const { return stages + (size_t)s * tp.stage_bytes; }

  struct Task {
    int x0, y0, w, hg, z;
    bool main;   // a plane of the segment itself (not a z-halo plane)
  };

  __device__ Task task(int i, bool stencil) const {
    const DevOp& d = e.P.op;
    const Tiling& tl = e.P.tl;
    const int tl_i = i / tpt, k = i - tl_i * tpt;
    const int t = blockIdx.x + tl_i * gridDim.x;
    const int bx = t % tl.tiles_x, rr = t / tl.tiles_x;
    const int by = rr % tl.tiles_y, bz = rr / tl.tiles_y;
    Task T;
    T.x0 = bx * TX;
    T.y0 = by * TY;
    T.w = min(TX, d.nx - T.x0);
    T.hg = min(TY, d.ny - T.y0);
    if (DIM == 3) {
      const int kk = stencil ? k - 1 : k;
      T.z = bz * tl.ZS + kk;
      T.main = kk >= 0 && kk < tl.ZS;
    } else {
      T.z = 0;
      T.main = true;
    }
    return T;
  }

  // How the task's data sits in its stage: strips needed, and whether the
  // tile-plus-halo box applies (no wrap of the y-halo, full-height tile).
  __device__ __forceinline__ bool has_strips(const Task& T, bool stencil) const { return stencil && T.main; }
  __device__ __forceinline__ bool is_full(const Task& T, bool stencil) const {
    return has_strips(T, stencil) && T.y0 >= 1 && T.hg == TY && T.y0 + TY + 1 <= e.P.op.ny;
  }

  // Issue the copies of task i into stage s (all threads call).
  __device__ void issue(int i, int s, const TmaPass& ps) {
    const bool stencil = ps.wout_col >= 0;
    if (i >= ntask) return;
    const DevOp& d = e.P.op;
    const Task T = task(i, stencil);
    const bool strips = has_strips(T, stencil);
    const bool full = is_full(T, stencil);
    const bool fields = stencil && T.main && NF > 0;
    if (e.warp != 0) return;
    const unsigned sbase = smem_u32(stage(s));
    const unsigned bar = bar0 + 8u * s;
    const int zz = (DIM == 3) ? wrapi(T.z, d.nz) : 0;
    const int ylo = wrapi(T.y0 - 1, d.ny), yhi = wrapi(T.y0 + T.hg, d.ny);
    const int xl = wrapi(T.x0 - LY::XW, d.nx), xh = wrapi(T.x0 + T.w, d.nx);
    const int ncap = tp.ncap;
    // column chunks of the bulk columns: 32s, then 16, 8, 4, 2, 1 (odd-sized
    // chunks start at even columns, which keeps every destination 128-byte aligned)
    const int n32 = ps.ncp >> 5, rem = ps.ncp & 31;
    const int nch = n32 + __popc(rem);
    // per chunk: tile box(es) and x-halo boxes; plus the same for the source column
    const int per = strips ? (full ? 3 : 5) : 1;
    const int nops = (nch + 1) * per;
    if (e.lane == 0) {
      const unsigned tile_bytes = full ? (unsigned)LY::COLA
                                       : (unsigned)(LY::COLB + (strips ? 2 * LY::COLY : 0));
      const unsigned halo_bytes = strips ? 2u * LY::COLX : 0u;
      const unsigned bytes = (unsigned)(ps.ncp + 1) * (tile_bytes + halo_bytes) +
                             (fields ? (unsigned)(NF * LY::FBOX) : 0u);
      mbar_expect_tx(bar, bytes);
    }
    __syncwarp();
    for (int o = e.lane; o < nops; o += 32) {
      const int ch = o / per, kind = o - ch * per;
      const bool src = ch == nch;
      int q = NQ - 1, c0 = 0;
      if (!src) {
        if (ch < n32) { q = 0; c0 = ch << 5; }
        else {
          int k = ch - n32;          // k-th set bit of rem among 16, 8, 4, 2, 1
          c0 = n32 << 5;
          for (int b = 4; b >= 0; --b) {
            if ((rem >> b) & 1) {
              if (k == 0) { q = 5 - b; break; }
              c0 += 1 << b;
              --k;
            }
          }
        }
      }
      const int col = src ? ps.src_col : c0;
      const unsigned regA = src ? sbase + LY::offS(ncap) : sbase;
      const unsigned regX = src ? sbase + LY::offS(ncap) + LY::SA : sbase + LY::offX(ncap);
      const int nX = src ? 1 : ncap;    // columns per x region side
      if (kind == 0) {
        if (full) tma_load_4d(regA + c0 * LY::COLA, &maps.mA[q], T.x0, T.y0 - 1, zz, col, bar);
        else tma_load_4d(regA + c0 * LY::COLB, &maps.mB[q], T.x0, T.y0, zz, col, bar);
      } else if (full) {   // kind 1, 2: x-halo boxes
        const int side = kind - 1;
        tma_load_4d(regX + (side * nX + c0) * LY::COLX, &maps.mX[q], side ? xh : xl, T.y0, zz, col, bar);
      } else if (kind <= 2) {   // wrap tile: y-halo rows
        const int side = kind - 1;
        const unsigned dst = src ? regA + LY::COLB + side * LY::SYR
                                 : regA + ncap * LY::COLB + (side * ncap + c0) * LY::COLY;
        tma_load_4d(dst, &maps.mY[q], T.x0, side ? yhi : ylo, zz, col, bar);
      } else {
        const int side = kind - 3;
        tma_load_4d(regX + (side * nX + c0) * LY::COLX, &maps.mX[q], side ? xh : xl, T.y0, zz, col, bar);
      }
    }
    if (fields && e.lane == 0) {
      const unsigned fdst = sbase + LY::offF(ncap);
      if (DIM == 3) {
        tma_load_3d(fdst, &maps.mF0, T.x0, T.y0, zz, bar);
      } else {
        tma_load_2d(fdst, &maps.mF0, T.x0, T.y0, bar);
        if (NF > 1) tma_load_2d(fdst + LY::FB, &maps.mF1, T.x0, T.y0, bar);
      }
    }
  }

  // Bounded wait for stage s; false on timeout or abort.
  __device__ bool wait_stage(int s) {
    const unsigned bar = bar0 + 8u * s;
    const unsigned par = (phases >> s) & 1u;
    if (e.tid == 0) {
      unsigned long long t0 = global_ns();
      unsigned it = 0;
      int res = 1;
      while (!mbar_try_wait(bar, par)) {
        if ((++it & 63u) == 0u) {
          if (ld_volatile_i32(&e.P.ctl->abort_flag)) { res = 0; break; }
          if ((long long)(global_ns() - t0) > e.P.timeout_ns) {
            atomicExch(&e.P.ctl->abort_flag, 1);
            atomicCAS(&e.P.ctl->status, 0, (int)LSA_ERR_TIMEOUT);
            res = 0;
            break;
          }
        }
      }
      e.S.flag = res;
    }
    __syncthreads();
    const bool ok = e.S.flag != 0;
    // every thread observes the completed phase itself (acquire of the TMA writes)
    if (ok) (void)mbar_try_wait(bar, par);
    phases ^= (1u << s);
    return ok;
  }

  // After a failed wait: let this CTA's copies already in flight land (bounded), then leave.
  __device__ void drain() {
    if (e.tid == 0) {
      const long long limit = 100000000LL;   // 0.1 s in total
      unsigned long long t0 = global_ns();
      for (int s = 0; s < 3; ++s) {
        const unsigned bar = bar0 + 8u * s;
        while (!mbar_try_wait(bar, (phases >> s) & 1u)) {
          if ((long long)(global_ns() - t0) > limit) break;
        }
      }
    }
    __syncthreads();
  }

  // Element offsets of a point's value in column 0 of its region and the
  // per-column stride (elements) -- bulk columns (src = false) or the source slot.
  __device__ __forceinline__ void locate(const Task& T, bool stencil, int sp, int lx, int ly,
                                         bool src, int& off, int& stride) const {
    const int ncap = tp.ncap;
    const bool full = is_full(T, stencil);
    const int nA = src ? 1 : ncap;
    const int baseA = src ? LY::offS(ncap) / ES : 0;
    const int baseX = src ? (LY::offS(ncap) + LY::SA) / ES : LY::offX(ncap) / ES;
    if (lx < 0 || lx >= T.w) {            // x-halo
      const int side = lx < 0 ? 0 : 1;
      stride = LY::COLX / ES;
      off = baseX + side * nA * stride + (sp * TY + ly) * LY::XW + (side ? 0 : LY::XW - 1);
    } else if (full) {
      stride = LY::COLA / ES;
      off = baseA + (sp * TYH + ly + 1) * TX + lx;
    } else if (ly < 0 || ly >= T.hg) {    // y-halo row of a wrap tile
      const int side = ly < 0 ? 0 : 1;
      stride = LY::COLY / ES;
      off = src ? baseA + (LY::COLB + side * LY::SYR) / ES + sp * TX + lx
                : baseA + nA * (LY::COLB / ES) + side * nA * stride + sp * TX + lx;
    } else {
      stride = LY::COLB / ES;
      off = baseA + (sp * TY + ly) * TX + lx;
    }
  }

  // Projection of task T from stage s into ring slot sl (and xout / self terms).
  __device__ void project(const Task& T, int s, const TmaPass& ps, int sl) {
    const DevOp& d = e.P.op;
    const bool stencil = ps.wout_col >= 0;
    const bool halo = has_strips(T, stencil);
    const int w = T.w, hg = T.hg;
    const bool fullw = (w == TX);
    const int pint = w * hg;
    const int pall = halo ? pint + 2 * w + 2 * hg : pint;
    const int total = NS * pall;
    const Tc* st = reinterpret_cast<const Tc*>(stage(s));
    const Tc a = (Tc)ps.a;
    Tc* ring = e.S.ring + sl * NS * PS;
    B* xout = ps.xout_col >= 0 ? reinterpret_cast<B*>(e.P.V) + (long long)ps.xout_col * d.N : nullptr;
    const int zz = (DIM == 3) ? wrapi(T.z, d.nz) : 0;
    const int ncp = ps.ncp;
    if (e.warp == 0) return;               // warp 0 is issuing the next task's copies
    for (int q = e.tid - 32; q < total; q += NT - 32) {
      const int sp = (NS == 1) ? 0 : q / pall;
      const int r = q - sp * pall;
      int lx, ly;
      if (r < pint) {
        if (fullw) { ly = r >> 4; lx = r & (TX - 1); }
        else { ly = r / w; lx = r - ly * w; }
      } else {
        const int h = r - pint;
        if (h < w) { lx = h; ly = -1; }
        else if (h < 2 * w) { lx = h - w; ly = hg; }
        else if (h < 2 * w + hg) { ly = h - 2 * w; lx = -1; }
        else { ly = h - 2 * w - hg; lx = w; }
      }
      int off, stride, soff, sstride;
      locate(T, stencil, sp, lx, ly, false, off, stride);
      locate(T, stencil, sp, lx, ly, true, soff, sstride);
      const Tc* p = st + off;
      Tc x0 = a * st[soff], x1 = (Tc)0;
      int c = 0;
      // batches of 8 columns: all shared-memory loads first, then the FMAs
      for (; c + 8 <= ncp; c += 8) {
        Tc v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = p[u * stride];
        p += 8 * stride;
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
          x0 = fma(-e.S.coefc[c + u], v[u], x0);
          x1 = fma(-e.S.coefc[c + u + 1], v[u + 1], x1);
        }
      }
      if (c + 4 <= ncp) {
        Tc v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = p[u * stride];
        p += 4 * stride;
        x0 = fma(-e.S.coefc[c], v[0], x0);
        x1 = fma(-e.S.coefc[c + 1], v[1], x1);
        x0 = fma(-e.S.coefc[c + 2], v[2], x0);
        x1 = fma(-e.S.coefc[c + 3], v[3], x1);
        c += 4;
      }
      for (; c < ncp; ++c, p += stride) x0 = fma(-e.S.coefc[c], *p, x0);
      const Tc x = x0 + x1;
      ring[sp * PS + (ly + 1) * PW + lx + 1] = x;
      if (T.main && r < pint) {
        const long long g = (long long)sp * d.npts + (T.x0 + lx) +
                            (long long)d.nx * ((T.y0 + ly) + (long long)d.ny * zz);
        if (xout) xout[g] = (B)x;
        if (!stencil && (ps.self & SELF_XX)) e.self_add(0, x, x);
      }
    }
  }

  // Stencil of plane zc (the task T's footprint) from the ring; fields from stage fs.
  __device__ void stencil(const Task& T, int zc, int fs, const TmaPass& ps) {
    const DevOp& d = e.P.op;
    const int w = T.w, hg = T.hg;
    if (e.tid >= w * hg) return;
    const int ly = (w == TX) ? (e.tid >> 4) : e.tid / w;
    const int lx = e.tid - ly * w;
    const Tc* zm = e.S.ring + e.slot(zc - 1) * NS * PS;
    const Tc* z0 = e.S.ring + e.slot(zc) * NS * PS;
    const Tc* zp = e.S.ring + e.slot(zc + 1) * NS * PS;
    const int o = (ly + 1) * PW + lx + 1;
    const Tc* F = reinterpret_cast<const Tc*>(stage(fs) + LY::offF(tp.ncap));
    Tc f0 = (Tc)0, f1 = (Tc)0;
    if (NF > 0) f0 = F[ly * TX + lx];
    if (NF > 1) f1 = F[LY::FB / ES + ly * TX + lx];
    Tc out[NS];
    Op::template apply_f<Tc>(e.cf, zm, z0, zp, o, f0, f1, out);
    B* wout = reinterpret_cast<B*>(e.P.V) + (long long)ps.wout_col * d.N;
    const long long gpt = (T.x0 + lx) + (long long)d.nx * ((T.y0 + ly) + (long long)d.ny * zc);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const Tc wv = out[s];
      e.S.wbuf[s * TX * TY + e.tid] = wv;
      wout[s * d.npts + gpt] = (B)wv;
      const Tc xs = z0[s * PS + o];
      if (ps.self & SELF_XX) e.self_add(0, xs, xs);
      if (ps.self & SELF_XW) e.self_add(1, xs, wv);
      if (ps.self & SELF_WW) e.self_add(2, wv, wv);
    }
  }

  // Inner products of columns 0..ncp-1 (stage ds, loaded for task Tds) with
  // plane zc's x and w.
  __device__ void dots(const Task& T, const Task& Tds, int zc, int ds, const TmaPass& ps) {
    if (ps.ncp <= 0) return;
    constexpr int NPS = (TX * TY + 31) / 32;
    const int w = T.w, hg = T.hg, pint = w * hg;
    const Tc* I = reinterpret_cast<const Tc*>(stage(ds));
    const bool full = is_full(Tds, true);
    const int cstride = full ? LY::COLA / ES : LY::COLB / ES;
    const int rows = full ? TYH : TY, row0 = full ? 1 : 0;
    const bool fullw = (w == TX);
#pragma unroll 1
    for (int sp = 0; sp < NS; ++sp) {
      const Tc* xr = e.S.ring + e.slot(zc) * NS * PS + sp * PS;
      Tc xv[NPS], wv[NPS];
      int so[NPS];
      if (fullw) {
        const int lx = e.lane & (TX - 1), ly0 = e.lane >> 4;
#pragma unroll
        for (int k = 0; k < NPS; ++k) {
          const int ly = ly0 + 2 * k;
          const bool ok = ly < hg;
          xv[k] = ok ? xr[(ly + 1) * PW + lx + 1] : (Tc)0;
          wv[k] = ok ? e.S.wbuf[sp * TX * TY + e.lane + 32 * k] : (Tc)0;
          so[k] = ok ? (sp * rows + ly + row0) * TX + lx : 0;
        }
      } else {
#pragma unroll
        for (int k = 0; k < NPS; ++k) {
          const int q = e.lane + 32 * k;
          if (q < pint) {
            const int ly = q / w, lx = q - ly * w;
            xv[k] = xr[(ly + 1) * PW + lx + 1];
            wv[k] = e.S.wbuf[sp * TX * TY + q];
            so[k] = (sp * rows + ly + row0) * TX + lx;
          } else {
            xv[k] = 0; wv[k] = 0; so[k] = 0;
          }
        }
      }
#pragma unroll
      for (int kk = 0; kk < KMAX; ++kk) {
        const int c = e.warp + NW * kk;
        if (c >= ps.ncp) break;
        const Tc* col = I + (size_t)c * cstride;
        if constexpr (F64) {
          double px0 = 0, pw0 = 0, px1 = 0, pw1 = 0;
#pragma unroll
          for (int k = 0; k < NPS; k += 2) {
            const double v0 = col[so[k]], v1 = col[so[k + 1]];
            px0 = fma(v0, (double)xv[k], px0);
            pw0 = fma(v0, (double)wv[k], pw0);
            px1 = fma(v1, (double)xv[k + 1], px1);
            pw1 = fma(v1, (double)wv[k + 1], pw1);
          }
          e.ax[kk] += px0 + px1;
          e.aw[kk] += pw0 + pw1;
        } else {
          float px0 = 0.f, pw0 = 0.f, px1 = 0.f, pw1 = 0.f;
#pragma unroll
          for (int k = 0; k < NPS; k += 2) {
            const float v0 = col[so[k]], v1 = col[so[k + 1]];
            px0 = fmaf(v0, (float)xv[k], px0);
            pw0 = fmaf(v0, (float)wv[k], pw0);
            px1 = fmaf(v1, (float)xv[k + 1], px1);
            pw1 = fmaf(v1, (float)wv[k + 1], pw1);
          }
          E::kahan(e.axs[kk], e.axc[kk], px0 + px1);
          E::kahan(e.aws[kk], e.awc[kk], pw0 + pw1);
        }
      }
    }
  }

  // One pass; returns the number of reduction slots, or -1 after a failed wait.
  __device__ int run(const TmaPass& ps) {
    const Tiling& tl = e.P.tl;
    const bool stencil = ps.wout_col >= 0;
    e.zero_acc();
    lag = (DIM == 3 && stencil) ? 1 : 0;
    depth = 2;
    tpt = (DIM == 3) ? (stencil ? tl.ZS + 2 : tl.ZS) : 1;
    const int ntiles_cta = (blockIdx.x < (unsigned)tl.ntiles)
                               ? (tl.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    ntask = ntiles_cta * tpt;
    fence_proxy_async();   // generic writes to the stage area (last CTA's scratch) before TMA
    __syncthreads();
    issue(0, 0, ps);
    Task Tprev;
    for (int i = 0; i < ntask; ++i) {
      const int s = i % 3;
      if (!wait_stage(s)) { drain(); return -1; }
      // the stage of task i-2 is free (its last reads were before the barrier
      // that closed task i-1): warp 0 refills it with task i+1 while warps 1..7
      // project task i
      issue(i + 1, (i + 1) % 3, ps);
      const Task T = task(i, stencil);
      project(T, s, ps, e.slot(T.z));
      __syncthreads();
      int zc = T.z, ds = s;
      bool compute = stencil;
      if (DIM == 3 && stencil) {
        const int k = i % tpt;            // 0: lower halo plane, 1: first plane, ...
        compute = k >= 2;                 // the stencil of plane z-1 is ready
        zc = T.z - 1;
        ds = (i + 2) % 3;                 // stage of task i-1
      }
      if (compute) {
        stencil_(T, zc, ds, ps);
        __syncthreads();
        dots(T, (DIM == 3 && stencil) ? Tprev : T, zc, ds, ps);
      }
      Tprev = T;
      __syncthreads();       // every thread is done with task i-1's stage before TMA refills it
    }
    PassT<B> pt;
    pt.d0 = 0;
    pt.d1 = stencil ? ps.ncp : 0;
    pt.dmode = DOT_X | DOT_W;
    pt.self = ps.self;
    return e.write_partials(pt);
  }

  __device__ __forceinline__ void stencil_(const Task& T, int zc, int fs, const TmaPass& ps) {
    stencil(T, zc, fs, ps);
  }

  // Alg. 4 with the staged passes; the step math is the engine's.
  __device__ void run_hybrid() {
    const int m = e.P.m;
    const int wc = tp.wcol;
    unsigned gen = 0;
    if (e.tid == 0) { e.S.a = (Tc)1; e.S.done = 0; e.S.fallback_pending = 0; e.S.syncs_c = 0; }
    __syncthreads();
    for (int j = 1; j <= m; ++j) {
      TmaPass ps;
      ps.ncp = j - 1;
      ps.src_col = (j == 1) ? 0 : wc + ((j - 1) & 1);
      ps.a = (j == 1) ? 1.0 : (double)e.S.a;
      ps.xout_col = (j == 1) ? -1 : j - 1;
      ps.wout_col = wc + (j & 1);
      ps.self = SELF_XX | SELF_XW | SELF_WW;
      const int ns = run(ps);
      if (ns < 0) return;
      if (!e.reduce_step(gen, ns, j, [&] { e.hybrid_step(j); })) return;
      if (e.S.done) return;
      if (e.S.fallback_pending) {
        TmaPass pf;
        pf.ncp = j;
        pf.src_col = wc + (j & 1);
        pf.a = (double)e.S.a;
        pf.xout_col = -1;
        pf.wout_col = -1;
        pf.self = SELF_XX;
        const int nf = run(pf);
        if (nf < 0) return;
        if (!e.reduce_step(gen, nf, j, [&] { e.hybrid_fallback_finish(j); })) return;
        if (e.S.done) return;
      }
    }
    TmaPass pl;
    pl.ncp = m;
    pl.src_col = wc + (m & 1);
    pl.a = (double)e.S.a;
    pl.xout_col = m;
    pl.wout_col = -1;
    pl.self = SELF_XX;
    const int nl = run(pl);
    if (nl < 0) return;
    e.reduce_step(gen, nl, 0, [&] { e.hybrid_final_finish(); });
  }
};

template <class Op, class Tc, class B>
__global__ void __launch_bounds__(NT, 1)
    k_arnoldi_tma(ArnoldiParams P, const __grid_constant__ TmaMaps maps, TmaParams tp) {
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  using E = Engine<Op, Tc, B>;
  using LY = TmaLayout<Op, Tc, B>;
  unsigned char* smem_raw = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
  typename E::Smem& S = *reinterpret_cast<typename E::Smem*>(smem_raw);
  unsigned char* stages = smem_raw + LY::head_bytes();
  E e(P, S, reinterpret_cast<double*>(stages));
  const unsigned bar0 = smem_u32(smem_raw + E::small_offset());
  if (threadIdx.x == 0) {
    for (int s = 0; s < 3; ++s) mbar_init(bar0 + 8u * s, 1u);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  TmaEngine<Op, Tc, B> t(e, maps, tp, stages, bar0);
  t.run_hybrid();
}

// ---------------------------------------------------------------------------
// Host side: applicability, tensor maps, launch.

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline EncodeTiledFn encode_tiled_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

constexpr size_t kMaxSmemPerBlock = 227 * 1024;

template <class Op, class Tc>
bool tma_applicable_op(const DevOp& d, const Tiling& tl, int m) {
  using LY = TmaLayout<Op, Tc, Tc>;
  const int es = sizeof(Tc);
  if (!encode_tiled_fn()) return false;
  if ((d.nx * es) % 16 != 0 || d.nx < TX || d.ny < TYH) return false;
  if (Op::DIM == 3 && (d.nz % tl.ZS) != 0) return false;
  return LY::smem_bytes(LY::ncap_for(m)) + 128 <= kMaxSmemPerBlock;
}

inline CUresult encode_box(EncodeTiledFn enc, CUtensorMap* map, CUtensorMapDataType dt, int rank,
                           const void* base, const cuuint64_t* dims, const cuuint64_t* strides,
                           const cuuint32_t* box) {
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  return enc(map, dt, rank, const_cast<void*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

template <class Op, class Tc>
cudaError_t launch_arnoldi_tma_op(const ArnoldiParams& P, int maxG, cudaStream_t s) {
  using LY = TmaLayout<Op, Tc, Tc>;
  const DevOp& d = P.op;
  EncodeTiledFn enc = encode_tiled_fn();
  if (!enc) return cudaErrorNotSupported;
  const int es = sizeof(Tc);
  const CUtensorMapDataType dt = es == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  TmaMaps maps;
  memset(&maps, 0, sizeof(maps));
  const cuuint64_t nzs = (Op::DIM == 3) ? (cuuint64_t)d.nz : (cuuint64_t)d.ns;
  const cuuint64_t dims[4] = {(cuuint64_t)d.nx, (cuuint64_t)d.ny, nzs, (cuuint64_t)(P.m + 3)};
  const cuuint64_t strides[3] = {(cuuint64_t)d.nx * es, (cuuint64_t)d.nx * d.ny * es,
                                 (cuuint64_t)d.N * es};
  CUresult r = CUDA_SUCCESS;
  for (int q = 0; q < NQ && r == CUDA_SUCCESS; ++q) {
    const cuuint32_t cb = (cuuint32_t)cbq(q);
    const cuuint32_t bA[4] = {TX, TYH, (cuuint32_t)LY::NZB, cb};
    const cuuint32_t bB[4] = {TX, TY, (cuuint32_t)LY::NZB, cb};
    const cuuint32_t bY[4] = {TX, 1, (cuuint32_t)LY::NZB, cb};
    const cuuint32_t bX[4] = {(cuuint32_t)LY::XW, TY, (cuuint32_t)LY::NZB, cb};
    r = encode_box(enc, &maps.mA[q], dt, 4, P.V, dims, strides, bA);
    if (r == CUDA_SUCCESS) r = encode_box(enc, &maps.mB[q], dt, 4, P.V, dims, strides, bB);
    if (r == CUDA_SUCCESS) r = encode_box(enc, &maps.mY[q], dt, 4, P.V, dims, strides, bY);
    if (r == CUDA_SUCCESS) r = encode_box(enc, &maps.mX[q], dt, 4, P.V, dims, strides, bX);
  }
  const void* f0 = es == 8 ? (const void*)d.f0 : (const void*)d.g0;
  const void* f1 = es == 8 ? (const void*)d.f1 : (const void*)d.g1;
  if (r == CUDA_SUCCESS && Op::NF > 0) {
    if (Op::DIM == 3) {
      const cuuint64_t fd[3] = {(cuuint64_t)d.nx, (cuuint64_t)d.ny, (cuuint64_t)d.nz};
      const cuuint64_t fs[2] = {(cuuint64_t)d.nx * es, (cuuint64_t)d.nx * d.ny * es};
      const cuuint32_t fb[3] = {TX, TY, 1};
      r = encode_box(enc, &maps.mF0, dt, 3, f0, fd, fs, fb);
    } else {
      const cuuint64_t fd[2] = {(cuuint64_t)d.nx, (cuuint64_t)d.ny};
      const cuuint64_t fs[1] = {(cuuint64_t)d.nx * es};
      const cuuint32_t fb[2] = {TX, TY};
      r = encode_box(enc, &maps.mF0, dt, 2, f0, fd, fs, fb);
      if (r == CUDA_SUCCESS && Op::NF > 1) r = encode_box(enc, &maps.mF1, dt, 2, f1, fd, fs, fb);
    }
  }
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  TmaParams tp;
  tp.ncap = LY::ncap_for(P.m);
  tp.stage_bytes = LY::stage_bytes(tp.ncap);
  tp.wcol = P.m + 1;
  const size_t sm = LY::smem_bytes(tp.ncap) + 128;
  auto k = k_arnoldi_tma<Op, Tc, Tc>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int nb = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, NT, sm);
  if (e != cudaSuccess || nb < 1) return e != cudaSuccess ? e : cudaErrorInvalidConfiguration;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int G = sms * nb;
  if (G > maxG) G = maxG;
  if (G > P.tl.ntiles) G = P.tl.ntiles;
  if (G < 1) G = 1;
  ArnoldiParams Pc = P;
  void* args[3] = {&Pc, &maps, &tp};
  return cudaLaunchCooperativeKernel((void*)k, dim3(G), dim3(NT), args, sm, s);
}

}  // namespace lsa
