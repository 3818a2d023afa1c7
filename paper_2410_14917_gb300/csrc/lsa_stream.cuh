// Streaming hybrid Arnoldi kernel for single-species operators in the float32
// basis form: the hot loop of the 3D advection-diffusion-reaction workload.
//
// Same mathematics as the hybrid passes of lsa_engine.cuh (Alg. 4 with the
// corrections of Algs. 5/6/7); what changes is how a pass moves the basis
// through the SM.
//
//  * A task is one 16x16 plane of a tile.  Its stage holds, for each of the
//    n projection columns and for the source vector: the tile interior with
//    its two y-halo rows, the x-halo (from the edge array -- see edge_slot --
//    where the writers of every column keep a tile's left and right
//    neighbour values contiguous), and the reaction field.  All of it comes
//    by TMA (cp.async.bulk.tensor) in few, large boxes: the TMA unit spends a
//    roughly fixed time per box, so a tile whose y-halo does not wrap takes
//    one 16x18 box per column range (interior and both halo rows), and a
//    column range is at most two boxes (8a + b columns, maps for 1..8 and for
//    multiples of 8).  A non-wrapping task with its field is 7 boxes.
//  * A task's boxes are issued by lane 0 of each warp (one box per warp, the
//    TMA unit then works through them) right after the barrier that frees the
//    stage, `depth` tasks ahead of the one being computed; thread 0 registers
//    the byte count on the stage's mbarrier before that barrier.  The stages
//    form a ring whose depth is chosen per pass from the shared memory left
//    (up to 8 stages), so short passes (small j) keep as many bytes in flight
//    as long ones.
//  * Thread (q, g) owns a 4-point quad q of the tile and the columns
//    c = g, g+4, g+8, ...: 128-bit shared loads, packed float32 pairs
//    (fma.rn.f32x2), and a three-shuffle transpose reduction that leaves point
//    g of the quad in lane group g.  The inner loops are unrolled to 16 column
//    slots with an exit after the pass's count; column slots past n read the
//    source slot with a zero coefficient.  The 64 halo points use the same
//    per-lane column split and the same summation order (a butterfly pairing
//    the same lanes in the same order), so a halo value equals, bit for bit,
//    the value the owning tile stores.
//  * The stencil of plane z needs the projection of plane z+1, so its inner
//    products are formed one task later; the stage of plane z is kept until
//    then.  Projected planes sit in a four-slot ring in shared memory; one
//    __syncthreads per task separates the projection from the stencil.
//  * Values are stored with per-pass column pointers and 32-bit indices; the
//    x-halo copies of a projected plane are written after the barrier by one
//    warp as two coalesced 64-byte rows read back from the ring.
//
// Every wait is bounded (globaltimer); on expiry the CTA sets the abort flag
// and LSA_ERR_TIMEOUT, lets its own copies in flight land (bounded), and leaves.
#pragma once

#include "lsa_tma.cuh"

namespace lsa {

constexpr int SQ_NG = 4;                               // column groups per quad
constexpr int SQ_KC = (MMAX + SQ_NG - 1) / SQ_NG;      // columns per group, at most
constexpr int SQ_RP = 24;                              // ring row pitch (floats); interior from column 4
constexpr int SQ_RS = (TY + 2) * SQ_RP;                // ring slot (floats)
constexpr int SQ_NRING = 4;
constexpr int SQ_NSTMAX = 8;
constexpr int SQ_COL = TX * TY;                        // floats of a column interior
constexpr int SQ_COLH = TX * (TY + 2);                 // ... with both y-halo rows
constexpr int SQ_EW = 2 * TY;                          // floats of a tile's x-halo (edge) record
constexpr int SQ_NB = 15;                              // box sizes: 1..8, 16, 24, ..., 64 columns
static_assert(2 * TX + 2 * TY == NT / 4, "one halo point per quad slot");
static_assert(MMAX <= 64, "column ranges are split as 8a + b with 8a <= 64");

__host__ __device__ constexpr int stream_box_cols(int i) { return i < 8 ? i + 1 : 8 * (i - 6); }
__host__ __device__ constexpr int stream_box_index(int cb) { return cb <= 8 ? cb - 1 : 6 + cb / 8; }

// Stage layout for n projection columns, every TMA destination 128-byte
// aligned.  Region A holds slots 0..n (the source in slot n) either as
// [slot][TY+2][TX] (tile and both y-halo rows; tiles whose halo does not
// wrap) or as [slot][TY][TX] followed by the two y-halo rows, each side
// [nys][TX] with the source row in the even slot ysrc.  Then the edge records
// [n+1][2TY] and the field [TY][TX].
__host__ __device__ constexpr int stream_ysrc(int n) { return n + (n & 1); }
__host__ __device__ constexpr int stream_nys(int n) { return stream_ysrc(n) + 2; }
__host__ __device__ constexpr int stream_regA(int n) { return (n + 1) * SQ_COL + 2 * stream_nys(n) * TX; }
__host__ __device__ constexpr int stream_stage_bytes(int n, int nfield) {
  return ((stream_regA(n) + (n + 1) * SQ_EW + nfield * SQ_COL) * 4 + 127) & ~127;
}

struct StreamMaps {
  CUtensorMap mA[SQ_NB];   // (TX, TY+2, 1, cb): tile and y-halo rows, extended basis (x, y, z, col)
  CUtensorMap mI[SQ_NB];   // (TX, TY, 1, cb):   tile only
  CUtensorMap mY[SQ_NB];   // (TX, 1, 1, cb):    one y-halo row
  CUtensorMap mE[SQ_NB];   // (2TY, 1, 1, cb):   edge records, over (r, bx, by + tiles_y z, col)
  CUtensorMap mF;          // (TX, TY, 1):       float field (x, y, z)
};

struct StreamParams {
  int cap;                 // bytes of shared memory for the stage ring
  int wcol;                // column of the first matvec buffer in the extended basis (m + 1)
};

struct SPass {
  int ncp;                 // projection columns 0..ncp-1
  int src_col;             // column of the source vector
  double a;                // source scale
  int xout_col;            // column written with x (-1: none)
  int wout_col;            // column written with w = A x (-1: no stencil)
  int self;                // SELF_* bits
};

// Per-pass accumulators of one thread, kept in registers by the pass loop:
// inner products of columns c = g + 4k (Kahan sum and compensation) and the
// three self terms x.x, x.w, w.w.
template <int KN>
struct StreamAcc {
  float xs[KN + 1], xc[KN + 1], ws[KN + 1], wc[KN + 1];
  float ss[3], sc[3];
};

template <class Op>
struct StreamLayout {
  using E = Engine<Op, float, float>;
  static __host__ __device__ constexpr size_t ring_off() { return (sizeof(typename E::Smem) + 127) & ~(size_t)127; }
  static __host__ __device__ constexpr size_t bar_off() { return ring_off() + (size_t)SQ_NRING * SQ_RS * 4; }
  static __host__ __device__ constexpr size_t tab_off() { return (bar_off() + 8 * SQ_NSTMAX + 15) & ~(size_t)15; }
  static __host__ __device__ constexpr size_t c2_off() { return (tab_off() + 16 * 3 * NW * 2 + 15) & ~(size_t)15; }
  static __host__ __device__ constexpr size_t stage_off() { return (c2_off() + 8 * (MMAX + 4) + 127) & ~(size_t)127; }
};

template <class Op>
struct StreamEngine {
  using E = Engine<Op, float, float>;
  static constexpr int DIM = Op::DIM, NF = Op::NF;
  static_assert(Op::NS == 1, "single-species operators only");

  E& e;
  const StreamMaps& maps;
  const StreamParams sp;
  float* ring;
  unsigned char* stages;
  unsigned full0;           // shared address of the first stage mbarrier
  unsigned fpar = 0;        // parity of the next wait, per stage
  unsigned pend = 0;        // thread 0: stages with copies not yet waited for
  int* s_stop;              // shared stop flag of this CTA
  int4* itab;               // per pass: each warp's boxes per task kind (see build_issue_table)
  const unsigned long long* coef2;   // per pass: {-coef_c, -coef_c} pairs (0 past n) for the packed FMAs

  // per pass
  int n = 0, kn = 0, nst = 2, depth = 1, lag = 0, tpt = 1, ntask = 0, sbytes = 0;
  bool stencil = false;
  float* vx = nullptr;      // columns the pass writes (x, w) and their edge records
  float* vw = nullptr;
  float* ex = nullptr;
  float* ew = nullptr;

  // thread roles: quad q (4 consecutive x points of a row), column group g
  const int q, g, ly, lx4;
  // this thread's point (lx4 + g, ly): its x-halo copy, if it has one, goes to the
  // record of the tile edx away (left for lx = 0, right for lx = TX-1) at eoff
  const bool edge;
  const int edx, eoff;
  const int hring;          // ring offset of this thread's halo point (halo_ring(q))
  // geometry in 32-bit units (a column has fewer than 2^31 points): row pitch,
  // plane size, tiles per row, edge-record plane size
  const int gnx, gplane, gtx, geplane;

  __device__ StreamEngine(E& en, const StreamMaps& m, const StreamParams& p, float* rg,
                          unsigned char* st, unsigned b, int* stop, int4* tab,
                          const unsigned long long* c2)
      : e(en), maps(m), sp(p), ring(rg), stages(st), full0(b), s_stop(stop), itab(tab), coef2(c2),
        q(en.warp * 8 + (en.lane & 7)), g(en.lane >> 3), ly(q >> 2), lx4((q & 3) * 4),
        edge(lx4 + g == 0 || lx4 + g == TX - 1), edx(lx4 + g == 0 ? -1 : 1),
        eoff((lx4 + g == 0 ? TY : 0) + ly), hring(halo_ring(en.warp * 8 + (en.lane & 7))),
        gnx(en.P.op.nx), gplane(en.P.op.nx * en.P.op.ny),
        gtx(en.P.tl.tiles_x), geplane(en.P.tl.tiles_x * en.P.tl.tiles_y * 2 * TY) {}

  __device__ __forceinline__ const float* stage(int s) const {
    return reinterpret_cast<const float*>(stages + (size_t)s * sbytes);
  }
  // float offsets inside a stage
  __device__ __forceinline__ int offY(int side) const { return (n + 1) * SQ_COL + side * stream_nys(n) * TX; }
  __device__ __forceinline__ int offE() const { return stream_regA(n); }
  __device__ __forceinline__ int offF() const { return stream_regA(n) + (n + 1) * SQ_EW; }

  struct STask {
    int bx, by, z;
    bool main;
  };

  // Incremental walk over this CTA's tasks (divisions only when the tile changes).
  struct Cursor {
    int tl_i, k, bx, by, bz;
  };
  __device__ __forceinline__ void cursor_tile(Cursor& c) const {
    const Tiling& tl = e.P.tl;
    const int t = blockIdx.x + c.tl_i * gridDim.x;
    const int rr = t / tl.tiles_x;
    c.bx = t - rr * tl.tiles_x;
    c.by = rr % tl.tiles_y;
    c.bz = rr / tl.tiles_y;
  }
  __device__ __forceinline__ Cursor cursor_at(int i) const {
    Cursor c;
    c.tl_i = i / tpt;
    c.k = i - c.tl_i * tpt;
    cursor_tile(c);
    return c;
  }
  __device__ __forceinline__ void cursor_next(Cursor& c) const {
    if (++c.k == tpt) { c.k = 0; ++c.tl_i; cursor_tile(c); }
  }
  __device__ __forceinline__ STask task_of(const Cursor& c) const {
    STask T;
    T.bx = c.bx;
    T.by = c.by;
    if (DIM == 3) {
      const int kk = stencil ? c.k - 1 : c.k;
      T.z = c.bz * e.P.tl.ZS + kk;
      T.main = kk >= 0 && kk < e.P.tl.ZS;
    } else {
      T.z = 0;
      T.main = true;
    }
    return T;
  }

  __device__ __forceinline__ bool has_halo(const STask& T) const { return stencil && T.main; }
  // the 16x18 layout: a halo task whose y-halo rows do not wrap around
  __device__ __forceinline__ bool is_full(const STask& T) const {
    return has_halo(T) && T.by >= 1 && T.by + 1 < e.P.tl.tiles_y;
  }

  __device__ bool timed_out(unsigned long long& t0, unsigned& it) const {
    if ((++it & 63u) != 0u) return false;
    if (ld_volatile_i32(s_stop)) return true;
    const unsigned long long now = global_ns();
    if (t0 == 0) { t0 = now; return false; }
    if ((long long)(now - t0) > e.P.timeout_ns) {
      atomicExch(&e.P.ctl->abort_flag, 1);
      atomicCAS(&e.P.ctl->status, 0, (int)LSA_ERR_TIMEOUT);
      *(volatile int*)s_stop = 1;
      return true;
    }
    return false;
  }

  // Thread 0 registers the bytes task T will bring into stage s (before the
  // barrier after which the boxes are issued).
  __device__ __forceinline__ void expect(const STask& T, int s) {
    const bool halo = has_halo(T);
    const bool field = halo && NF > 0;
    const unsigned per = (unsigned)(SQ_COL + (halo ? 2 * TX + SQ_EW : 0)) * 4u;
    mbar_expect_tx(full0 + 8u * s, (unsigned)(n + 1) * per + (field ? (unsigned)SQ_COL * 4u : 0u));
    pend |= 1u << s;
  }

  // Per pass, lane 0 of every warp lists the boxes it issues for each kind of
  // task (0: halo, y-halo not wrapping; 1: halo, wrapping; 2: no halo).  A
  // task's boxes are -- per map family the column ranges [0, 8a) and [8a, n)
  // (when not empty) and the source, then the field -- and warp w takes boxes
  // w and w + 8.  Entry: (family | box index << 3, stage byte offset, column).
  // Families: 0 tile + y-halo rows, 1 tile, 2 / 3 low / high y-halo row,
  // 4 edge records, 5 field.
  __device__ __forceinline__ void build_issue_table(const SPass& ps) {
    if (e.lane != 0) return;
    const int a = n & ~7, b = n & 7;
    const int per_fam = (a ? 1 : 0) + (b ? 1 : 0) + 1;
    for (int kind = 0; kind < 3; ++kind) {
      const bool halo = kind < 2, full = kind == 0;
      const bool field = halo && NF > 0;
      const int nfam = !halo ? 1 : (full ? 2 : 4);
      const int nbox = nfam * per_fam + (field ? 1 : 0);
      for (int slot = 0; slot < 2; ++slot) {
        const int bi = e.warp + NW * slot;
        int4 en = make_int4(-1, 0, 0, 0);
        if (bi == nfam * per_fam && field) {
          en = make_int4(5, offF() * 4, 0, 0);
        } else if (bi < nbox) {
          const int fam = bi / per_fam, r = bi - fam * per_fam;
          const int rk = (a && r == 0) ? 0 : (b && r == (a ? 1 : 0)) ? 1 : 2;   // range, range, source
          const int c0 = rk == 0 ? 0 : a;
          const int col = rk == 2 ? ps.src_col : c0;
          const int bidx = rk == 2 ? 0 : stream_box_index(rk == 0 ? a : b);
          const int sl = rk == 2 ? n : c0;
          const int fk = full ? (fam == 0 ? 0 : 4) : (!halo ? 1 : (fam == 0 ? 1 : fam == 3 ? 4 : fam + 1));
          int dst;
          if (fk == 0) dst = sl * SQ_COLH * 4;
          else if (fk == 1) dst = sl * SQ_COL * 4;
          else if (fk == 4) dst = (offE() + sl * SQ_EW) * 4;
          else dst = (offY(fk - 2) + (rk == 2 ? stream_ysrc(n) : c0) * TX) * 4;
          en = make_int4(fk | (bidx << 3), dst, col, 0);
        }
        itab[(kind * NW + e.warp) * 2 + slot] = en;
      }
    }
  }

  // The copies of task T into stage s (lane 0 of each warp, its table entries).
  __device__ __forceinline__ void issue(const STask& T, int s) {
    if (e.lane != 0) return;
    const bool halo = has_halo(T), full = is_full(T);
    const int kind = full ? 0 : (halo ? 1 : 2);
    const unsigned bar = full0 + 8u * s;
    const unsigned base = smem_u32(stages) + (unsigned)(s * sbytes);
    const DevOp& d = e.P.op;
    const int zz = (DIM == 3) ? wrapi(T.z, d.nz) : 0;
    const int x0 = T.bx * TX, y0 = T.by * TY;
#pragma unroll
    for (int slot = 0; slot < 2; ++slot) {
      const int4 en = itab[(kind * NW + e.warp) * 2 + slot];
      if (en.x < 0) break;
      const int fk = en.x & 7, bidx = en.x >> 3;
      const unsigned dst = base + (unsigned)en.y;
      switch (fk) {
        case 0: tma_load_4d(dst, &maps.mA[bidx], x0, y0 - 1, zz, en.z, bar); break;
        case 1: tma_load_4d(dst, &maps.mI[bidx], x0, y0, zz, en.z, bar); break;
        case 2: tma_load_4d(dst, &maps.mY[bidx], x0, wrapi(y0 - 1, d.ny), zz, en.z, bar); break;
        case 3: tma_load_4d(dst, &maps.mY[bidx], x0, wrapi(y0 + TY, d.ny), zz, en.z, bar); break;
        case 4: tma_load_4d(dst, &maps.mE[bidx], 0, T.bx, T.by + e.P.tl.tiles_y * zz, en.z, bar); break;
        default: tma_load_3d(dst, &maps.mF, x0, y0, zz, bar); break;
      }
    }
  }

  // After a stop: thread 0 lets this CTA's copies in flight land (bounded).
  __device__ void drain() {
    if (e.tid != 0) return;
    const long long limit = 100000000LL;   // 0.1 s in total
    const unsigned long long t0 = global_ns();
    for (int s = 0; s < SQ_NSTMAX; ++s) {
      if (!((pend >> s) & 1u)) continue;
      while (!mbar_try_wait(full0 + 8u * s, (fpar >> s) & 1u))
        if ((long long)(global_ns() - t0) > limit) break;
    }
  }

  // Bounded wait of the calling thread for stage s.
  __device__ __forceinline__ bool wait_full(int s) {
    const unsigned bar = full0 + 8u * s;
    unsigned long long t0 = 0;
    unsigned it = 0;
    while (!mbar_try_wait(bar, (fpar >> s) & 1u))
      if (timed_out(t0, it)) return false;
    fpar ^= 1u << s;
    if (e.tid == 0) pend &= ~(1u << s);
    return true;
  }

  __device__ __forceinline__ static int halo_ring(int h) {
    if (h < TX) return 4 + h;
    if (h < 2 * TX) return (TY + 1) * SQ_RP + 4 + (h - TX);
    if (h < 2 * TX + TY) return (h - 2 * TX + 1) * SQ_RP + 3;
    return (h - 2 * TX - TY + 1) * SQ_RP + 4 + TX;
  }

  __device__ __forceinline__ static float4 lds4(const float* p) {
    return *reinterpret_cast<const float4*>(p);
  }
  // Packed float32 pairs (fma/mul.rn.f32x2: two IEEE float32 operations per
  // instruction, each rounded as the scalar one).
  __device__ __forceinline__ static unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                            unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
  }
  __device__ __forceinline__ static unsigned long long fmul2(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
  }
  __device__ __forceinline__ static unsigned long long pack2(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
  }
  __device__ __forceinline__ static float2 unpack2(unsigned long long r) {
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
  }
  __device__ __forceinline__ static ulonglong2 lds2x2(const float* p) {
    return *reinterpret_cast<const ulonglong2*>(p);
  }
  // Sum of the quad over the four column groups, component g to lane group g,
  // in the butterfly's order (pairs across lane bit 3, then across bit 4), so
  // a point's value equals bit for bit what bfly gives its halo copy.
  __device__ __forceinline__ float quad_sum(const float4& x) const {
    const bool b0 = g & 1, b1 = g & 2;
    // across bit 3: keep the components whose low index bit is g's, send the others
    const float s0 = b0 ? x.x : x.y, s1 = b0 ? x.z : x.w;
    const float k0 = (b0 ? x.y : x.x) + __shfl_xor_sync(0xffffffffu, s0, 8);
    const float k1 = (b0 ? x.w : x.z) + __shfl_xor_sync(0xffffffffu, s1, 8);
    // across bit 4: keep component g
    return (b1 ? k1 : k0) + __shfl_xor_sync(0xffffffffu, b1 ? k0 : k1, 16);
  }
  __device__ __forceinline__ static float bfly(float v) {
    v += __shfl_xor_sync(0xffffffffu, v, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 16);
    return v;
  }

  // store this thread's value x of tile T, plane zz into column vc, with its
  // edge copy into ec (the column's edge records): the left column is the right
  // halo of the tile to the left, the right column the left halo of the next
  __device__ __forceinline__ void store_point(const STask& T, int zz, float* vc, float* ec, float x) const {
    vc[T.bx * TX + lx4 + g + gnx * (T.by * TY + ly) + gplane * zz] = x;
    if (ec && edge) {
      int nb = T.bx + edx;
      nb = nb < 0 ? gtx - 1 : (nb == gtx ? 0 : nb);
      ec[geplane * zz + (T.by * gtx + nb) * (2 * TY) + eoff] = x;   // edge_slot(nb, T.by, zz) + eoff
    }
  }

  // The x-halo copies of a projected plane (ring slot rs), written by one warp
  // after the barrier: lanes 0-15 the tile's left column into the record of the
  // tile to the left (its right halo), lanes 16-31 the right column into the
  // record of the next tile (its left halo) -- two 64-byte rows.
  __device__ __forceinline__ void x_edges(const STask& T, int rs) const {
    const int zz = (DIM == 3) ? wrapi(T.z, e.P.op.nz) : 0;
    const int side = e.lane >> 4, r = e.lane & (TY - 1);
    const float v = ring[rs * SQ_RS + (r + 1) * SQ_RP + 4 + (side ? TX - 1 : 0)];
    int nb = T.bx + (side ? 1 : -1);
    nb = nb < 0 ? gtx - 1 : (nb == gtx ? 0 : nb);
    ex[geplane * zz + (T.by * gtx + nb) * (2 * TY) + (side ? 0 : TY) + r] = v;
  }

  // x (quad) = a*src - sum_c coef_c V_c over this thread's column slots
  // c = g, g+4, ... (p points at slot 0 of the quad, CS is the slot stride);
  // slots below kn-1 are always columns (4(kn-1) + 3 < n + 3); the last one may
  // be past n and then reads the source slot with a zero coefficient.
  // The inner loops for the pass's column count: unrolled to the largest count
  // with an exit after kn slots (one copy of each loop instead of one per count,
  // so the task loop stays small in the instruction cache).
  template <int CS>
  __device__ __forceinline__ float4 proj_quad_n(const float* p, float a) const {
    const unsigned long long* coef = coef2 + g;
    const float* pg = p + g * CS;
    unsigned long long xlo = 0ull, xhi = 0ull;      // (+0, +0) pairs
    if (g == 0) {
      const float4 sv = lds4(p + n * CS);
      xlo = pack2(a * sv.x, a * sv.y);
      xhi = pack2(a * sv.z, a * sv.w);
    }
    // per point the same fma(-c, v, x) sequence as proj_point_n: bit-identical
#pragma unroll
    for (int k = 0; k < SQ_KC; ++k) {
      if (k >= kn) break;
      const float* pk = (k + 1 < kn || g + SQ_NG * k < n) ? pg + SQ_NG * k * CS : p + n * CS;
      const ulonglong2 v = lds2x2(pk);
      const unsigned long long cc = coef[SQ_NG * k];
      xlo = ffma2(cc, v.x, xlo);
      xhi = ffma2(cc, v.y, xhi);
    }
    const float2 lo = unpack2(xlo), hi = unpack2(xhi);
    return make_float4(lo.x, lo.y, hi.x, hi.y);
  }
  template <int CS>
  __device__ __forceinline__ float proj_point_n(const float* p, int sslot, float a) const {
    const float* coef = e.S.coefc + g;
    const float* pg = p + g * CS;
    float x = (g == 0) ? a * p[sslot * CS] : 0.f;
#pragma unroll
    for (int k = 0; k < SQ_KC; ++k) {
      if (k >= kn) break;
      const float* pk = (k + 1 < kn || g + SQ_NG * k < n) ? pg + SQ_NG * k * CS : p + sslot * CS;
      x = fmaf(-coef[SQ_NG * k], *pk, x);
    }
    return x;
  }
  template <int CS>
  __device__ __forceinline__ void dots_quad_n(const float* p, const float4& x4, const float4& w4,
                                              StreamAcc<SQ_KC>& A) const {
    const float* pg = p + g * CS;
    const unsigned long long xlo = pack2(x4.x, x4.y), xhi = pack2(x4.z, x4.w);
    const unsigned long long wlo = pack2(w4.x, w4.y), whi = pack2(w4.z, w4.w);
#pragma unroll
    for (int k = 0; k < SQ_KC; ++k) {
      if (k >= kn) break;
      const float* pk = (k + 1 < kn || g + SQ_NG * k < n) ? pg + SQ_NG * k * CS : p + n * CS;
      const ulonglong2 v = lds2x2(pk);
      const float2 tx = unpack2(ffma2(v.y, xhi, fmul2(v.x, xlo)));   // (v0 x0 + v2 x2, v1 x1 + v3 x3)
      const float2 tw = unpack2(ffma2(v.y, whi, fmul2(v.x, wlo)));
      E::kahan(A.xs[k], A.xc[k], tx.x + tx.y);
      E::kahan(A.ws[k], A.wc[k], tw.x + tw.y);
    }
  }

  // Projection of task T from stage s into ring slot rs: x = a*src - sum_c coef_c V_c.
  __device__ __forceinline__ void project(const STask& T, int s, const SPass& ps, int rs, StreamAcc<SQ_KC>& A) {
    const DevOp& d = e.P.op;
    const float* st = stage(s);
    const float a = (float)ps.a;
    const bool full = is_full(T);
    const float4 x = full ? proj_quad_n<SQ_COLH>(st + (ly + 1) * TX + lx4, a)
                          : proj_quad_n<SQ_COL>(st + ly * TX + lx4, a);
    const float xg = quad_sum(x);
    float* rg = ring + rs * SQ_RS;
    rg[(ly + 1) * SQ_RP + 4 + lx4 + g] = xg;
    if (T.main) {
      const int zz = (DIM == 3) ? wrapi(T.z, d.nz) : 0;
      if (ps.xout_col >= 0) store_point(T, zz, vx, nullptr, xg);   // edges: x_edges
      if (!stencil && (ps.self & SELF_XX)) E::kahan(A.ss[0], A.sc[0], xg * xg);
    }
    if (has_halo(T)) {
      // halo point q, same column split and summation order as its owner
      float hx;
      if (q < 2 * TX) {                    // y-halo rows
        const int side = q >= TX ? 1 : 0, hx0 = q & (TX - 1);
        if (full) hx = proj_point_n<SQ_COLH>(st + side * (TY + 1) * TX + hx0, n, a);
        else hx = proj_point_n<TX>(st + offY(side) + hx0, stream_ysrc(n), a);
      } else {                             // x-halo from the edge records
        hx = proj_point_n<SQ_EW>(st + offE() + (q - 2 * TX), n, a);
      }
      hx = bfly(hx);
      if (g == 0) rg[hring] = hx;
    }
  }

  // Stencil of plane zc (ring slots rm, r0, rp) at this thread's point, the
  // self terms, and the inner products of the columns staged for task Td in ds.
  __device__ __forceinline__ void stencil_dots(const STask& Td, int zc, int ds, int rm, int r0, int rp,
                                               const SPass& ps, const Coef<float>& cf, StreamAcc<SQ_KC>& A) {
    const float* xm = ring + rm * SQ_RS;
    const float* x0 = ring + r0 * SQ_RS;
    const float* xp = ring + rp * SQ_RS;
    const float* sd = stage(ds);
    const int lx = lx4 + g;
    const int o = (ly + 1) * SQ_RP + 4 + lx;
    const float f0 = (NF > 0) ? sd[offF() + ly * TX + lx] : 0.f;
    float out[1];
    Op::template apply_f<float, SQ_RP>(cf, xm, x0, xp, o, f0, 0.f, out);
    const float w = out[0];
    store_point(Td, zc, vw, ew, w);
    const float xs = x0[o];
    if (ps.self & SELF_XX) E::kahan(A.ss[0], A.sc[0], xs * xs);
    if (ps.self & SELF_XW) E::kahan(A.ss[1], A.sc[1], xs * w);
    if (ps.self & SELF_WW) E::kahan(A.ss[2], A.sc[2], w * w);
    const int src = e.lane & 7;
    float4 w4;
    w4.x = __shfl_sync(0xffffffffu, w, src);
    w4.y = __shfl_sync(0xffffffffu, w, src + 8);
    w4.z = __shfl_sync(0xffffffffu, w, src + 16);
    w4.w = __shfl_sync(0xffffffffu, w, src + 24);
    const float4 x4 = lds4(x0 + (ly + 1) * SQ_RP + 4 + lx4);
    const bool full = is_full(Td);
    if (full) dots_quad_n<SQ_COLH>(sd + (ly + 1) * TX + lx4, x4, w4, A);
    else dots_quad_n<SQ_COL>(sd + ly * TX + lx4, x4, w4, A);
  }

  // The task loop of a pass and its per-CTA partial sums (x dots, w dots,
  // then the three self terms); returns the number of reduction slots, or -1
  // after a stop.
  __device__ __forceinline__ int consume(const SPass& ps) {
    StreamAcc<SQ_KC> A;
#pragma unroll
    for (int k = 0; k <= SQ_KC; ++k) A.xs[k] = A.xc[k] = A.ws[k] = A.wc[k] = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) A.ss[k] = A.sc[k] = 0.f;
    const Coef<float> cf = e.cf;
    Cursor cur = cursor_at(0), icur = cursor_at(depth);   // task i, and task i + depth to issue
    int s = 0, si = depth % nst, sprev = 0;
    STask Tp = task_of(cur);
    for (int i = 0; i < ntask; ++i) {
      const STask T = task_of(cur);
      // a warp projects only if all its lanes saw the stage (warp shuffles inside)
      if (__all_sync(0xffffffffu, wait_full(s))) project(T, s, ps, i & (SQ_NRING - 1), A);
      const bool refill = i + depth < ntask;
      const STask Ti = task_of(icur);
      if (refill && e.tid == 0) expect(Ti, si);
      __syncthreads();
      if (ld_volatile_i32(s_stop)) break;
      if (ex && T.main && e.warp == 0) x_edges(T, i & (SQ_NRING - 1));
      // the stage of task i-1-lag is free: refill it with task i+depth
      if (refill) issue(Ti, si);
      bool compute = stencil;
      if (DIM == 3 && stencil) compute = cur.k >= 2;   // the stencil of plane z-1 needs plane z
      if (compute) {
        if (DIM == 3)
          stencil_dots(Tp, T.z - 1, sprev, (i + SQ_NRING - 2) & (SQ_NRING - 1), (i - 1) & (SQ_NRING - 1),
                       i & (SQ_NRING - 1), ps, cf, A);
        else
          stencil_dots(T, 0, s, i & (SQ_NRING - 1), i & (SQ_NRING - 1), i & (SQ_NRING - 1), ps, cf, A);
      }
      Tp = T;
      sprev = s;
      if (++s == nst) s = 0;
      if (++si == nst) si = 0;
      cursor_next(cur);
      cursor_next(icur);
    }
    __syncthreads();   // every read of the stages is done (the partials reuse them)
    if (ld_volatile_i32(s_stop)) {
      drain();
      __syncthreads();
      return -1;
    }
    const int nd = stencil ? n : 0;
    double* part = e.P.partials + (long long)e.grank * SLOTS;
    double* wred = reinterpret_cast<double*>(stages);      // NW x 2 x MMAX (stages are idle)
    // the eight quads of a lane group summed as compensated float32 pairs
    // (Kahan keeps sum = s - c: the pair is (s, -c); two_sum at every stage),
    // converted to float64 once; slots past the pass's count hold nothing
#pragma unroll
    for (int k = 0; k < SQ_KC; ++k) {
      if (k >= kn) break;
      const int c = g + SQ_NG * k;
      float xs = A.xs[k], xe = -A.xc[k], ws = A.ws[k], we = -A.wc[k];
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) {
        const float oxs = __shfl_xor_sync(0xffffffffu, xs, o), oxe = __shfl_xor_sync(0xffffffffu, xe, o);
        const float ows = __shfl_xor_sync(0xffffffffu, ws, o), owe = __shfl_xor_sync(0xffffffffu, we, o);
        float ex, ew;
        xs = two_sum(xs, oxs, ex);
        xe = (xe + oxe) + ex;
        ws = two_sum(ws, ows, ew);
        we = (we + owe) + ew;
      }
      if ((e.lane & 7) == 0 && c < nd) {
        wred[(e.warp * 2) * MMAX + c] = (double)xs + (double)xe;
        wred[(e.warp * 2 + 1) * MMAX + c] = (double)ws + (double)we;
      }
    }
    {
      float ts[4] = {A.ss[0], A.ss[1], A.ss[2], 0.f}, te[4] = {-A.sc[0], -A.sc[1], -A.sc[2], 0.f};
      warp_sum_many_comp<4>(ts, te);           // lane l: value l >> 3
      if ((e.lane & 7) == 0 && e.lane < 24) e.S.bred[e.warp][e.lane >> 3] = (double)ts[0] + (double)te[0];
    }
    __syncthreads();
    for (int t = e.tid; t < 2 * nd; t += NT) {
      const int kind = t / nd, c = t - kind * nd;
      double acc = 0.0;
      for (int w = 0; w < NW; ++w) acc += wred[(w * 2 + kind) * MMAX + c];
      part[kind * nd + c] = acc;
    }
    if (e.tid < 3) {
      double acc = 0;
      for (int i = 0; i < NW; ++i) acc += e.S.bred[i][e.tid];
      part[2 * nd + e.tid] = acc;
    }
    return 2 * nd + 3;
  }

  // One pass; returns the number of reduction slots, or -1 after a stop.
  __device__ __forceinline__ int run(const SPass& ps) {
    const Tiling& tl = e.P.tl;
    n = ps.ncp;
    kn = (n + SQ_NG - 1) / SQ_NG;
    stencil = ps.wout_col >= 0;
    {
      const long long N = e.P.op.N;
      float* V = reinterpret_cast<float*>(e.P.V);
      vx = ps.xout_col >= 0 ? V + (long long)ps.xout_col * N : nullptr;
      ex = ps.xout_col >= 0 ? e.P.E + (long long)ps.xout_col * (N / 8) : nullptr;
      vw = stencil ? V + (long long)ps.wout_col * N : nullptr;
      ew = stencil ? e.P.E + (long long)ps.wout_col * (N / 8) : nullptr;
    }
    lag = (DIM == 3 && stencil) ? 1 : 0;
    tpt = (DIM == 3) ? (stencil ? tl.ZS + 2 : tl.ZS) : 1;
    const int ntiles_cta = ((int)blockIdx.x < tl.ntiles) ? (tl.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    ntask = ntiles_cta * tpt;
    sbytes = stream_stage_bytes(n, (stencil && NF > 0) ? 1 : 0);
    nst = sp.cap / sbytes;
    if (nst > SQ_NSTMAX) nst = SQ_NSTMAX;
    depth = nst - 1 - lag;                // the host guarantees depth >= 1
    // column slots n..4kn-1 of the last group get a zero coefficient
    if (e.tid >= n && e.tid < SQ_NG * kn) e.S.coefc[e.tid] = 0.f;
    if (e.tid < SQ_NG * kn) {
      const float c = (e.tid < n) ? -e.S.coefc[e.tid] : 0.f;
      const_cast<unsigned long long*>(coef2)[e.tid] = pack2(c, c);
    }
    // generic writes to the stage area (partials scratch, the last CTA's small
    // matrices) are ordered before this pass's TMA writes into it
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (e.tid == 0) {
      Cursor c = cursor_at(0);
      for (int t = 0; t < depth && t < ntask; ++t) {
        expect(task_of(c), t);
        cursor_next(c);
      }
    }
    build_issue_table(ps);
    __syncthreads();
    if (e.lane == 0) {
      asm volatile("fence.proxy.async;" ::: "memory");   // and global writes before the TMA reads
      Cursor c = cursor_at(0);
      for (int t = 0; t < depth && t < ntask; ++t) {
        issue(task_of(c), t);
        cursor_next(c);
      }
    }
    return consume(ps);
  }

  // Alg. 4 with the streamed passes; the step mathematics is the engine's.
  // One call site of run() (its per-column-count variants are inlined once):
  // kind 0 = the step's pass, 1 = the explicit-norm fallback pass, 2 = the
  // final projection and norm.
  __device__ void run_hybrid() {
    const int m = e.P.m;
    const int wc = sp.wcol;
    unsigned gen = 0;
    if (e.tid == 0) { e.S.a = 1.f; e.S.done = 0; e.S.fallback_pending = 0; e.S.syncs_c = 0; *s_stop = 0; }
    __syncthreads();
    int j = 1, kind = 0;
    for (;;) {
      SPass ps;
      if (kind == 0) {
        ps.ncp = j - 1;
        ps.src_col = (j == 1) ? 0 : wc + ((j - 1) & 1);
        ps.a = (j == 1) ? 1.0 : (double)e.S.a;
        ps.xout_col = (j == 1) ? -1 : j - 1;
        ps.wout_col = wc + (j & 1);
        ps.self = SELF_XX | SELF_XW | SELF_WW;
      } else {
        ps.ncp = (kind == 1) ? j : m;
        ps.src_col = wc + (((kind == 1) ? j : m) & 1);
        ps.a = (double)e.S.a;
        ps.xout_col = (kind == 1) ? -1 : m;
        ps.wout_col = -1;
        ps.self = SELF_XX;
      }
      const int ns = run(ps);
      if (ns < 0) return;
      if (kind == 0) {
        if (!e.reduce_step(gen, ns, j, [&] { e.hybrid_step(j); })) return;
        if (e.S.done) return;
        if (e.S.fallback_pending) kind = 1;
        else if (j == m) kind = 2;
        else ++j;
      } else if (kind == 1) {
        if (!e.reduce_step(gen, ns, j, [&] { e.hybrid_fallback_finish(j); })) return;
        if (e.S.done) return;
        if (j == m) kind = 2;
        else { ++j; kind = 0; }
      } else {
        e.reduce_step(gen, ns, 0, [&] { e.hybrid_final_finish(); });
        return;
      }
    }
  }
};

template <class Op>
__global__ void __launch_bounds__(NT, 1)
    k_arnoldi_stream(ArnoldiParams P, const __grid_constant__ StreamMaps maps, StreamParams sp) {
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  using E = Engine<Op, float, float>;
  using LY = StreamLayout<Op>;
  unsigned char* smem_raw = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
  typename E::Smem& S = *reinterpret_cast<typename E::Smem*>(smem_raw);
  unsigned char* stages = smem_raw + LY::stage_off();
  E e(P, S, reinterpret_cast<double*>(stages));
  const unsigned bar0 = smem_u32(smem_raw + LY::bar_off());
  if (threadIdx.x == 0) {
    for (int s = 0; s < SQ_NSTMAX; ++s) mbar_init(bar0 + 8u * s, 1u);   // thread 0's expect_tx
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  StreamEngine<Op> t(e, maps, sp, reinterpret_cast<float*>(smem_raw + LY::ring_off()), stages, bar0,
                     &S.stop, reinterpret_cast<int4*>(smem_raw + LY::tab_off()),
                     reinterpret_cast<const unsigned long long*>(smem_raw + LY::c2_off()));
  t.run_hybrid();
}

// ---------------------------------------------------------------------------
// Host side: applicability, tensor maps, launch.

template <class Op>
int stream_cap_bytes() {
  using LY = StreamLayout<Op>;
  return (int)(kMaxSmemPerBlock - 128 - LY::stage_off());
}

template <class Op>
bool stream_applicable_op(const DevOp& d, const Tiling& tl, int m) {
  if (Op::NS != 1) return false;
  if (!encode_tiled_fn()) return false;
  if (d.nx % TX != 0 || d.ny % TY != 0) return false;
  if (Op::DIM == 3 && (d.nz % tl.ZS) != 0) return false;
  const int cap = stream_cap_bytes<Op>();
  const int lag = (Op::DIM == 3) ? 1 : 0;
  // hybrid passes (n <= m - 1, stencil) and the final / fallback passes (n <= m)
  const int s_hyb = stream_stage_bytes(m - 1, Op::NF > 0 ? 1 : 0);
  const int s_fin = stream_stage_bytes(m, 0);
  if (cap / s_hyb < 2 + lag || cap / s_fin < 2) return false;
  return cap >= (int)(sizeof(double) * MMAX * MMAX) && cap >= (int)(sizeof(double) * 2 * NW * MMAX);
}

template <class Op>
cudaError_t launch_arnoldi_stream_op(const ArnoldiParams& P, cudaStream_t s) {
  const DevOp& d = P.op;
  const Tiling& tl = P.tl;
  EncodeTiledFn enc = encode_tiled_fn();
  if (!enc || !P.E) return cudaErrorNotSupported;
  StreamMaps maps;
  memset(&maps, 0, sizeof(maps));
  const cuuint64_t nzs = (Op::DIM == 3) ? (cuuint64_t)d.nz : 1;
  const cuuint64_t dims[4] = {(cuuint64_t)d.nx, (cuuint64_t)d.ny, nzs, (cuuint64_t)(P.m + 3)};
  const cuuint64_t strides[3] = {(cuuint64_t)d.nx * 4, (cuuint64_t)d.nx * d.ny * 4, (cuuint64_t)d.N * 4};
  const cuuint64_t edims[4] = {(cuuint64_t)SQ_EW, (cuuint64_t)tl.tiles_x, (cuuint64_t)tl.tiles_y * nzs,
                               (cuuint64_t)(P.m + 3)};
  const cuuint64_t estrides[3] = {(cuuint64_t)SQ_EW * 4, (cuuint64_t)tl.tiles_x * SQ_EW * 4,
                                  (cuuint64_t)(d.N / 8) * 4};
  const CUtensorMapDataType f32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  CUresult r = CUDA_SUCCESS;
  for (int i = 0; i < SQ_NB && r == CUDA_SUCCESS; ++i) {
    const cuuint32_t cb = (cuuint32_t)stream_box_cols(i);
    const cuuint32_t bA[4] = {TX, TY + 2, 1, cb};
    const cuuint32_t bI[4] = {TX, TY, 1, cb};
    const cuuint32_t bY[4] = {TX, 1, 1, cb};
    const cuuint32_t bE[4] = {SQ_EW, 1, 1, cb};
    r = encode_box(enc, &maps.mA[i], f32, 4, P.V, dims, strides, bA);
    if (r == CUDA_SUCCESS) r = encode_box(enc, &maps.mI[i], f32, 4, P.V, dims, strides, bI);
    if (r == CUDA_SUCCESS) r = encode_box(enc, &maps.mY[i], f32, 4, P.V, dims, strides, bY);
    if (r == CUDA_SUCCESS) r = encode_box(enc, &maps.mE[i], f32, 4, P.E, edims, estrides, bE);
  }
  if (r == CUDA_SUCCESS && Op::NF > 0) {
    const cuuint64_t fd[3] = {(cuuint64_t)d.nx, (cuuint64_t)d.ny, nzs};
    const cuuint64_t fs[2] = {(cuuint64_t)d.nx * 4, (cuuint64_t)d.nx * d.ny * 4};
    const cuuint32_t fb[3] = {TX, TY, 1};
    r = encode_box(enc, &maps.mF, f32, 3, d.g0, fd, fs, fb);
  }
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  StreamParams sp;
  sp.cap = stream_cap_bytes<Op>();
  sp.wcol = P.m + 1;
  const size_t sm = kMaxSmemPerBlock;
  auto k = k_arnoldi_stream<Op>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int nb = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, NT, sm);
  if (e != cudaSuccess || nb < 1) return e != cudaSuccess ? e : cudaErrorInvalidConfiguration;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int G = sms * nb;
  if (G > P.tl.ntiles) G = P.tl.ntiles;
  if (G < 1) G = 1;
  ArnoldiParams Pc = P;
  void* args[3] = {&Pc, &maps, &sp};
  return cudaLaunchCooperativeKernel((void*)k, dim3(G), dim3(NT), args, sm, s);
}

}  // namespace lsa
