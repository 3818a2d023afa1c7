// C-ABI entry points of liblsarnoldi: argument checks, workspace layout and
// the launch sequence of each call.  See include/lsarnoldi.h for the contract.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>

#include "lsa_internal.cuh"

namespace lsa {

cudaError_t launch_arnoldi_advdiff2d(const ArnoldiParams&, int, int, cudaStream_t);
cudaError_t launch_arnoldi_grayscott2d(const ArnoldiParams&, int, int, cudaStream_t);
cudaError_t launch_arnoldi_adr3d(const ArnoldiParams&, int, int, cudaStream_t);
cudaError_t launch_matvec_advdiff2d(const ArnoldiParams&, int, const void*, void*, int, cudaStream_t);
cudaError_t launch_matvec_grayscott2d(const ArnoldiParams&, int, const void*, void*, int, cudaStream_t);
cudaError_t launch_matvec_adr3d(const ArnoldiParams&, int, const void*, void*, int, cudaStream_t);
int blocks_per_sm_advdiff2d(int);
int blocks_per_sm_grayscott2d(int);
int blocks_per_sm_adr3d(int);
int flat_blocks_per_sm_adr3d(int);
int flat_blocks_per_sm_advdiff2d(int);
int flat_blocks_per_sm_grayscott2d(int);
bool tma_applicable_advdiff2d(const DevOp&, const Tiling&, int, int);
bool tma_applicable_grayscott2d(const DevOp&, const Tiling&, int, int);
bool tma_applicable_adr3d(const DevOp&, const Tiling&, int, int);
cudaError_t launch_arnoldi_tma_advdiff2d(const ArnoldiParams&, int, int, cudaStream_t);
cudaError_t launch_arnoldi_tma_grayscott2d(const ArnoldiParams&, int, int, cudaStream_t);
cudaError_t launch_arnoldi_tma_adr3d(const ArnoldiParams&, int, int, cudaStream_t);
bool stream_applicable_advdiff2d(const DevOp&, const Tiling&, int);
bool stream_applicable_adr3d(const DevOp&, const Tiling&, int);
cudaError_t launch_arnoldi_stream_advdiff2d(const ArnoldiParams&, cudaStream_t);
bool cluster_applicable_advdiff2d(const DevOp&, const Tiling&, int);
cudaError_t launch_arnoldi_cluster_advdiff2d(const ArnoldiParams&, const SmallParams*, double*, cudaStream_t);
cudaError_t launch_arnoldi_stream_adr3d(const ArnoldiParams&, cudaStream_t);

cudaError_t launch_arnoldi_grayscott2d_t(const ArnoldiParams&, int, int, cudaStream_t);
cudaError_t launch_matvec_grayscott2d_t(const ArnoldiParams&, int, const void*, void*, int, cudaStream_t);
int blocks_per_sm_grayscott2d_t(int);
cudaError_t launch_arnoldi_grayscott2d_frechet(const ArnoldiParams&, int, int, cudaStream_t);
cudaError_t launch_matvec_grayscott2d_frechet(const ArnoldiParams&, int, const void*, void*, int, cudaStream_t);
int blocks_per_sm_grayscott2d_frechet(int);

static const long long kTimeoutNs = 5000000000LL;   // 5 s per barrier wait
static const double kBreakdownTolFp64 = 1e-13;
static const double kBreakdownTolFp32 = 1e-6;

bool make_devop(const lsa_op* op, DevOp* d) {
  if (!op || !d) return false;
  memset(d, 0, sizeof(*d));
  if (op->nx < 1 || op->ny < 1 || op->nz < 1) return false;
  if (!(op->dx > 0.0) || !isfinite(op->dx)) return false;
  for (int i = 0; i < 3; ++i)
    if (!isfinite(op->vel[i])) return false;
  if (!isfinite(op->diff) || !isfinite(op->diff2) || !isfinite(op->F) || !isfinite(op->k)) return false;
  d->kind = op->kind;
  d->nx = op->nx; d->ny = op->ny; d->nz = op->nz;
  d->npts = (long long)op->nx * op->ny * op->nz;
  const double inv = 1.0 / (op->dx * op->dx), ih = 1.0 / op->dx;
  switch (op->kind) {
    case LSA_OP_ADVDIFF2D:
      if (op->nz != 1) return false;
      d->ns = 1;
      d->cE = op->diff * inv - 0.5 * op->vel[0] * ih;
      d->cW = op->diff * inv + 0.5 * op->vel[0] * ih;
      d->cN = op->diff * inv - 0.5 * op->vel[1] * ih;
      d->cS = op->diff * inv + 0.5 * op->vel[1] * ih;
      d->cC = -4.0 * op->diff * inv;
      break;
    case LSA_OP_GRAYSCOTT2D:
    case LSA_OP_GRAYSCOTT2D_T:
    case LSA_OP_GRAYSCOTT2D_FRECHET:
      if (op->nz != 1 || !op->field0 || !op->field1) return false;
      if (op->kind == LSA_OP_GRAYSCOTT2D_FRECHET && (op->aux < 0 || op->aux > 3)) return false;
      d->ns = op->kind == LSA_OP_GRAYSCOTT2D_FRECHET ? 4 : 2;
      d->du = op->diff * inv;
      d->dv = op->diff2 * inv;
      d->F = op->F;
      d->k = op->k;
      d->idx2 = inv;
      d->dir = op->kind == LSA_OP_GRAYSCOTT2D_FRECHET ? op->aux : 0;
      d->f0 = op->field0;
      d->f1 = op->field1;
      break;
    case LSA_OP_ADR3D: {
      if (!op->field0) return false;
      d->ns = 1;
      const double e = op->diff * inv;
      const double ux = op->vel[0], uy = op->vel[1], uz = op->vel[2];
      d->cW = e + fmax(ux, 0.0) * ih;  d->cE = e + fmax(-ux, 0.0) * ih;
      d->cS = e + fmax(uy, 0.0) * ih;  d->cN = e + fmax(-uy, 0.0) * ih;
      d->cD = e + fmax(uz, 0.0) * ih;  d->cU = e + fmax(-uz, 0.0) * ih;
      d->cC = -6.0 * e - (fabs(ux) + fabs(uy) + fabs(uz)) * ih;
      d->f0 = op->field0;
      break;
    }
    default:
      return false;
  }
  d->N = d->ns * d->npts;
  if (d->N >= (1LL << 31)) return false;   // 32-bit element offsets in the dot phase
  return true;
}

static int sm_count();

Tiling make_tiling(const DevOp& d) {
  Tiling t;
  t.tiles_x = (d.nx + TX - 1) / TX;
  t.tiles_y = (d.ny + TY - 1) / TY;
  // z-segment (3D): a divisor of nz (uniform segments), at least 4 and at most
  // 64, that minimises the planes the busiest SM streams, tiles dealt
  // round-robin to one CTA per SM: ceil(tiles / SMs) * (ZS + 2), the two being
  // the segment's halo planes (longer segments: fewer halo planes; shorter
  // ones: a smaller last round).  Ties go to the longer segment.
  t.ZS = 1;
  if (d.kind == LSA_OP_ADR3D) {
    const int sms = sm_count();
    const long long txy = (long long)t.tiles_x * t.tiles_y;
    long long best = -1;
    for (int z = (d.nz < 64 ? d.nz : 64); z >= 1; --z) {
      if (d.nz % z != 0 || (z < 4 && z != d.nz)) continue;
      const long long tiles = txy * (d.nz / z);
      const long long rounds = sms > 0 ? (tiles + sms - 1) / sms : tiles;
      const long long cost = rounds * (z + 2);
      if (best < 0 || cost < best) { best = cost; t.ZS = z; }
    }
    if (best < 0) t.ZS = d.nz;
  }
  t.zsegs = (d.nz + t.ZS - 1) / t.ZS;
  t.ntiles = t.tiles_x * t.tiles_y * t.zsegs;
  return t;
}

static int sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return sms;
}

int arnoldi_blocks_per_sm(const DevOp& d, int precision) {
  static int cache[6][2][16];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 16) dev = 0;
  int& c = cache[d.kind][precision][dev];
  if (c > 0) return c;
  int nb = 0;
  if (d.kind == LSA_OP_ADVDIFF2D) nb = blocks_per_sm_advdiff2d(precision);
  else if (d.kind == LSA_OP_GRAYSCOTT2D) nb = blocks_per_sm_grayscott2d(precision);
  else if (d.kind == LSA_OP_GRAYSCOTT2D_T) nb = blocks_per_sm_grayscott2d_t(precision);
  else if (d.kind == LSA_OP_GRAYSCOTT2D_FRECHET) nb = blocks_per_sm_grayscott2d_frechet(precision);
  else nb = blocks_per_sm_adr3d(precision);
  c = nb;
  return nb;
}

// The TMA-staged kernel runs the hybrid variants of the float32-basis form
// whenever its stage buffers fit in shared memory and the grid meets the TMA
// alignment rules (LSA_TMA=0 in the environment disables it, LSA_TMA=1 also
// allows it for the float64 form).
static bool use_tma(const ArnoldiParams& P, int precision) {
  if (!is_hybrid(P.variant) || P.op.kind > LSA_OP_ADR3D || P.naug > 0) return false;
  const char* env = getenv("LSA_TMA");
  if (env && env[0] == '0') return false;
  if (precision == LSA_FP64 && !(env && env[0] == '1')) return false;
  if (P.op.kind == LSA_OP_ADVDIFF2D) return tma_applicable_advdiff2d(P.op, P.tl, P.m, precision);
  if (P.op.kind == LSA_OP_GRAYSCOTT2D) return tma_applicable_grayscott2d(P.op, P.tl, P.m, precision);
  return tma_applicable_adr3d(P.op, P.tl, P.m, precision);
}

// The streaming kernel (interior-only TMA stages, halo by plain loads) runs
// the hybrid variants of the float32-basis form for the single-species
// operators whenever its stages fit (LSA_STREAM=0 in the environment disables
// it; the other kernels then run).
static bool use_stream(const ArnoldiParams& P, int precision) {
  if (!is_hybrid(P.variant) || precision != LSA_FP32_BASIS || !P.E || P.naug > 0) return false;
  const char* env = getenv("LSA_STREAM");
  if (env && env[0] == '0') return false;
  if (P.op.kind == LSA_OP_ADVDIFF2D) return stream_applicable_advdiff2d(P.op, P.tl, P.m);
  if (P.op.kind == LSA_OP_ADR3D) return stream_applicable_adr3d(P.op, P.tl, P.m);
  return false;
}

// The single-cluster kernel (basis in the CTAs' shared memory, cluster
// barriers) runs the hybrid variants in float64 on small 2D advection-diffusion
// grids (at most 16 tiles of 16 x 16) when the device can place such a cluster
// (LSA_CLUSTER=0 in the environment disables it).  The device check is cached
// per device and m.
static bool use_cluster(const ArnoldiParams& P, int precision) {
  if (!is_hybrid(P.variant) || precision != LSA_FP64 || P.naug > 0 || P.op.kind != LSA_OP_ADVDIFF2D) return false;
  if (P.op.nx % TX != 0 || P.op.ny % TY != 0 || P.tl.tiles_x * P.tl.tiles_y > 16) return false;
  const char* env = getenv("LSA_CLUSTER");
  if (env && env[0] == '0') return false;
  static signed char cache[64][MMAX + 1][17];   // 0 unknown, 1 yes, -1 no
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64 || P.m < 1 || P.m > MMAX) return false;
  signed char& c = cache[dev][P.m][P.tl.tiles_x * P.tl.tiles_y];
  if (c == 0) c = cluster_applicable_advdiff2d(P.op, P.tl, P.m) ? 1 : -1;
  return c > 0;
}

// Step form of the grid kernel's hybrid variants: 0 one pass; 1 two-phase
// (project over flat shares; grid barrier; stencil and inner products over
// tiles: no halo projection, one more barrier per step); 2 flat two-phase (the
// ADR 3D, advection-diffusion and Gray-Scott operators: the second pass also
// over flat shares, the stencil's neighbours read through L2, no tile chain;
// its own kernel).  Chosen per
// device, operator shape, m, variant and precision:
// LSA_TWO_PHASE=0/1/2 in the environment forces it (2 runs form 1 where the
// flat kernel does not exist); otherwise the form that
// lsa_tune_step recorded for the shape; otherwise a default measured on
// GB300: a two-phase form for 3D grids (the z-halo planes make the repeated
// projection large): the flat one in float64 (ADR 256^3: 93 against 119 ms),
// the tile one for the float32 basis (where it is used at all: the streaming
// kernel runs those grids first); the flat form for 2D grids with at least
// six 16x16 tiles per SM (Gray-Scott 512^2: 9.33 against 9.60 ms in float64,
// 3.50 against 4.30 in float32), one-pass below that (the extra barrier
// costs more than the halo).
struct StepKey {
  int dev, kind, nx, ny, nz, m, variant, precision;
  bool operator<(const StepKey& o) const {
    const int a[8] = {dev, kind, nx, ny, nz, m, variant, precision};
    const int b[8] = {o.dev, o.kind, o.nx, o.ny, o.nz, o.m, o.variant, o.precision};
    for (int i = 0; i < 8; ++i)
      if (a[i] != b[i]) return a[i] < b[i];
    return false;
  }
};
static std::mutex g_step_mu;
static std::map<StepKey, int> g_step_choice;
static thread_local int g_step_force = -1;     // set by lsa_tune_step around its timing runs

static bool step_key(const ArnoldiParams& P, int precision, StepKey* k) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  *k = StepKey{dev, P.op.kind, P.op.nx, P.op.ny, P.op.nz, P.m, P.variant, precision};
  return true;
}

static bool two_phase_applies(const ArnoldiParams& P, int precision) {
  return is_hybrid(P.variant) && P.naug == 0 && !use_cluster(P, precision) &&
         !use_stream(P, precision) && !use_tma(P, precision);
}

static int two_phase_choice(const ArnoldiParams& P, int precision) {
  if (!two_phase_applies(P, precision)) return 0;
  if (g_step_force >= 0) return g_step_force;
  const char* env = getenv("LSA_TWO_PHASE");
  if (env && env[0] >= '0' && env[0] <= '2') return env[0] - '0';
  StepKey k;
  if (!step_key(P, precision, &k)) return 0;
  {
    std::lock_guard<std::mutex> lock(g_step_mu);
    auto it = g_step_choice.find(k);
    if (it != g_step_choice.end()) return it->second;
  }
  if (P.op.nz > 1) return precision == LSA_FP64 ? 2 : 1;
  return P.tl.ntiles >= 6 * sm_count() ? 2 : 0;
}

// The flat two-phase kernel exists for the ADR 3D, advection-diffusion and
// Gray-Scott operators, and its grid must be resident: as many CTAs per SM as
// the grid kernel's layout assumes.
static bool flat_fits(const ArnoldiParams& P, int precision) {
  const int kind = P.op.kind;
  if (kind != LSA_OP_ADR3D && kind != LSA_OP_ADVDIFF2D && kind != LSA_OP_GRAYSCOTT2D) return false;
  static int cache[6][2][16];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 16) dev = 0;
  int& c = cache[kind][precision][dev];
  if (c == 0) {
    const int nb = kind == LSA_OP_ADR3D ? flat_blocks_per_sm_adr3d(precision)
                   : kind == LSA_OP_ADVDIFF2D ? flat_blocks_per_sm_advdiff2d(precision)
                                              : flat_blocks_per_sm_grayscott2d(precision);
    c = nb >= arnoldi_blocks_per_sm(P.op, precision) ? 1 : -1;
  }
  return c > 0;
}

static int step_form(const ArnoldiParams& P, int precision) {
  const int form = two_phase_choice(P, precision);
  return (form == 2 && !flat_fits(P, precision)) ? 1 : form;
}

static int arnoldi_kernel_kind(const ArnoldiParams& P, int precision) {
  if (use_cluster(P, precision)) return 3;
  if (use_stream(P, precision)) return 2;
  if (use_tma(P, precision)) return 1;
  const int form = step_form(P, precision);
  return form == 0 ? 0 : 3 + form;
}

static cudaError_t launch_arnoldi_grid(const ArnoldiParams& P, int precision, int G, cudaStream_t s);

cudaError_t launch_arnoldi(const ArnoldiParams& P, int precision, int G, cudaStream_t s) {
  if (P.two_phase == 0) {
    const int form = step_form(P, precision);
    if (form) {
      ArnoldiParams Q = P;
      Q.two_phase = form;
      return launch_arnoldi_grid(Q, precision, G, s);
    }
  }
  return launch_arnoldi_grid(P, precision, G, s);
}

static cudaError_t launch_arnoldi_grid(const ArnoldiParams& P, int precision, int G, cudaStream_t s) {
  if (use_cluster(P, precision)) return launch_arnoldi_cluster_advdiff2d(P, nullptr, nullptr, s);
  if (use_stream(P, precision)) {
    if (P.op.kind == LSA_OP_ADVDIFF2D) return launch_arnoldi_stream_advdiff2d(P, s);
    return launch_arnoldi_stream_adr3d(P, s);
  }
  if (use_tma(P, precision)) {
    const int maxG = sm_count() * 2;
    if (P.op.kind == LSA_OP_ADVDIFF2D) return launch_arnoldi_tma_advdiff2d(P, precision, maxG, s);
    if (P.op.kind == LSA_OP_GRAYSCOTT2D) return launch_arnoldi_tma_grayscott2d(P, precision, maxG, s);
    return launch_arnoldi_tma_adr3d(P, precision, maxG, s);
  }
  if (P.op.kind == LSA_OP_ADVDIFF2D) return launch_arnoldi_advdiff2d(P, precision, G, s);
  if (P.op.kind == LSA_OP_GRAYSCOTT2D) return launch_arnoldi_grayscott2d(P, precision, G, s);
  if (P.op.kind == LSA_OP_GRAYSCOTT2D_T) return launch_arnoldi_grayscott2d_t(P, precision, G, s);
  if (P.op.kind == LSA_OP_GRAYSCOTT2D_FRECHET) return launch_arnoldi_grayscott2d_frechet(P, precision, G, s);
  return launch_arnoldi_adr3d(P, precision, G, s);
}

cudaError_t launch_matvec(const ArnoldiParams& P, int precision, const void* x, void* y, int G,
                          cudaStream_t s) {
  if (P.op.kind == LSA_OP_ADVDIFF2D) return launch_matvec_advdiff2d(P, precision, x, y, G, s);
  if (P.op.kind == LSA_OP_GRAYSCOTT2D) return launch_matvec_grayscott2d(P, precision, x, y, G, s);
  if (P.op.kind == LSA_OP_GRAYSCOTT2D_T) return launch_matvec_grayscott2d_t(P, precision, x, y, G, s);
  if (P.op.kind == LSA_OP_GRAYSCOTT2D_FRECHET)
    return launch_matvec_grayscott2d_frechet(P, precision, x, y, G, s);
  return launch_matvec_adr3d(P, precision, x, y, G, s);
}

// Workspace layout for (op, m, precision).  G = CTAs of the persistent kernel.
static bool make_layout(const DevOp& d, int m, int precision, Layout* L) {
  const int sms = sm_count();
  if (sms <= 0) return false;
  const int bps = arnoldi_blocks_per_sm(d, precision);
  if (bps <= 0) return false;
  const Tiling t = make_tiling(d);
  int G = sms * bps;
  if (G > t.ntiles) G = t.ntiles;
  if (G < 1) G = 1;
  const size_t bsz = precision == LSA_FP64 ? 8 : 4;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
  L->ctl = take(sizeof(Ctl));
  L->partials = take((size_t)sms * (bps > 2 ? bps : 2) * SLOTS * sizeof(double));
  L->gsum = take((size_t)RG_MAX * SLOTS * sizeof(double));
  L->T = take((size_t)MMAX * MMAX * sizeof(double));
  L->L = take((size_t)MMAX * MMAX * sizeof(double));
  L->H = take((size_t)(m + 1) * m * sizeof(double));
  // basis columns 0..m and the two matvec buffers as columns m+1, m+2 of one
  // contiguous block (one tensor for the TMA-staged kernel)
  L->V = take((size_t)d.N * (m + 3) * bsz);
  L->W0 = L->V + (size_t)d.N * (m + 1) * bsz;
  L->W1 = L->V + (size_t)d.N * (m + 2) * bsz;
  L->small = take((size_t)6 * SMALL_STRIDE * SMALL_STRIDE * sizeof(double));
  L->coefs = take((size_t)(PMAX + 2) * (MMAX + 2) * sizeof(double));
  size_t nfield = 0;
  if (precision == LSA_FP32_BASIS) {
    if (d.kind == LSA_OP_GRAYSCOTT2D) nfield = (size_t)d.nx * d.ny;
    else if (d.kind == LSA_OP_ADR3D) nfield = (size_t)d.npts;
  }
  L->g0 = take(nfield * sizeof(float));
  L->g1 = take(nfield * sizeof(float));
  // edge array of the streaming kernel (single-species float32 operators on whole tiles)
  const bool edges = precision == LSA_FP32_BASIS && d.ns == 1 && d.nx % TX == 0 && d.ny % TY == 0 &&
                     (d.kind == LSA_OP_ADVDIFF2D || (d.kind == LSA_OP_ADR3D && d.nz % t.ZS == 0));
  L->E = take(edges ? (size_t)(m + 3) * (size_t)(d.N / 8) * sizeof(float) : 0);
  if (!edges) L->E = 0;
  L->xaug = take((size_t)(m + 3) * PMAX * sizeof(double));
  L->total = off;
  L->G = G;
  return true;
}

static lsa_status from_cuda(cudaError_t e) { return e == cudaSuccess ? LSA_OK : LSA_ERR_CUDA; }

static lsa_status fill_stats(const void* work, lsa_stats* out, cudaStream_t s) {
  Ctl c;
  cudaError_t e = cudaMemcpyAsync(&c, work, sizeof(Ctl), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return LSA_ERR_CUDA;
  if (out) {
    out->status = c.status;
    out->m_eff = c.m_eff;
    out->breakdown = c.breakdown;
    out->norm_fallbacks = c.fallbacks;
    out->grid_syncs = c.syncs;
    out->grid_barriers = c.barriers;
    out->beta = c.beta;
    out->err_est = c.err_est;
    out->h_last = c.h_last;
    out->ms_arnoldi = out->ms_expm = out->ms_combine = 0.f;
    out->launches = 0;
    out->arnoldi_kernel = 0;
  }
  if (c.status < 0) return (lsa_status)c.status;
  if (c.breakdown) return LSA_BREAKDOWN;
  return (lsa_status)c.status;
}

static bool aligned256(const void* p) { return ((uintptr_t)p & 255u) == 0; }

// CUDA events around the kernels of one call, used only when the caller asks
// for statistics (the call synchronises then anyway).
struct CallTimer {
  bool on = false;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaStream_t s = nullptr;
  CallTimer(bool enable, cudaStream_t st) : on(enable), s(st) {
    if (!on) return;
    for (auto& e : ev)
      if (cudaEventCreate(&e) != cudaSuccess) { on = false; e = nullptr; }
  }
  void mark(int i) { if (on) cudaEventRecord(ev[i], s); }
  float ms(int a, int b) {
    float t = 0.f;
    if (on) cudaEventElapsedTime(&t, ev[a], ev[b]);
    return t;
  }
  ~CallTimer() {
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
  }
};

struct Prepared {
  DevOp d;
  Layout L;
  ArnoldiParams P;
  char* w;
};

static lsa_status prepare(const lsa_op* op, int m, int precision, void* work, size_t work_bytes,
                          Prepared* pr) {
  if (precision != LSA_FP64 && precision != LSA_FP32_BASIS) return LSA_ERR_ARG;
  if (!make_devop(op, &pr->d)) return LSA_ERR_ARG;
  if (pr->d.kind > LSA_OP_ADR3D && precision != LSA_FP64) return LSA_ERR_ARG;
  if (m < 1 || m > MMAX) return LSA_ERR_ARG;
  if (!make_layout(pr->d, m, precision, &pr->L)) return LSA_ERR_CUDA;
  if (!work || !aligned256(work) || work_bytes < pr->L.total) return LSA_ERR_WORKSPACE;
  pr->w = (char*)work;
  if (precision == LSA_FP32_BASIS) {
    pr->d.g0 = (const float*)(pr->w + pr->L.g0);
    pr->d.g1 = (const float*)(pr->w + pr->L.g1);
  }
  ArnoldiParams& P = pr->P;
  memset(&P, 0, sizeof(P));
  P.op = pr->d;
  P.tl = make_tiling(pr->d);
  P.ctl = (Ctl*)(pr->w + pr->L.ctl);
  P.partials = (double*)(pr->w + pr->L.partials);
  P.gsum = (double*)(pr->w + pr->L.gsum);
  P.T = (double*)(pr->w + pr->L.T);
  P.L = (double*)(pr->w + pr->L.L);
  P.V = pr->w + pr->L.V;
  P.W0 = pr->w + pr->L.W0;
  P.W1 = pr->w + pr->L.W1;
  P.H = (double*)(pr->w + pr->L.H);
  P.E = pr->L.E ? (float*)(pr->w + pr->L.E) : nullptr;
  P.xaug = (double*)(pr->w + pr->L.xaug);
  P.m = m;
  P.brk_tol = precision == LSA_FP64 ? kBreakdownTolFp64 : kBreakdownTolFp32;
  P.timeout_ns = kTimeoutNs;
  return LSA_OK;
}

}  // namespace lsa

using namespace lsa;

extern "C" {

int lsa_max_m(void) { return MMAX; }
int lsa_version(void) { return 100; }

const char* lsa_status_string(int s) {
  switch (s) {
    case LSA_OK: return "LSA_OK";
    case LSA_BREAKDOWN: return "LSA_BREAKDOWN";
    case LSA_NOT_CONVERGED: return "LSA_NOT_CONVERGED";
    case LSA_ERR_ARG: return "LSA_ERR_ARG";
    case LSA_ERR_CUDA: return "LSA_ERR_CUDA";
    case LSA_ERR_TIMEOUT: return "LSA_ERR_TIMEOUT";
    case LSA_ERR_NUMERIC: return "LSA_ERR_NUMERIC";
    case LSA_ERR_WORKSPACE: return "LSA_ERR_WORKSPACE";
    default: return "LSA_UNKNOWN";
  }
}

long long lsa_op_dof(const lsa_op* op) {
  DevOp d;
  if (!make_devop(op, &d)) return -1;
  return d.N;
}

size_t lsa_workspace_bytes(const lsa_op* op, int m, int p, int precision) {
  DevOp d;
  if (precision != LSA_FP64 && precision != LSA_FP32_BASIS) return 0;
  if (!make_devop(op, &d) || m < 1 || m > MMAX || p < 0 || p > PMAX) return 0;
  if (d.kind > LSA_OP_ADR3D && precision != LSA_FP64) return 0;
  Layout L;
  if (!make_layout(d, m, precision, &L)) return 0;
  return L.total;
}

lsa_status lsa_matvec(const lsa_op* op, const void* x, void* y, int precision, void* work,
                      size_t work_bytes, void* stream) {
  if (!x || !y) return LSA_ERR_ARG;
  Prepared pr;
  lsa_status st = prepare(op, 1, precision, work, work_bytes, &pr);
  if (st != LSA_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = launch_init(pr.P.ctl, pr.d, (float*)pr.d.g0, (float*)pr.d.g1, precision, nullptr, 0,
                              nullptr, nullptr, s);
  if (e == cudaSuccess) e = launch_matvec(pr.P, precision, x, y, pr.L.G, s);
  return from_cuda(e);
}

lsa_status lsa_arnoldi(const lsa_op* op, const double* v, int m, int variant, int precision,
                       void* V, double* H, void* work, size_t work_bytes, lsa_stats* stats,
                       void* stream) {
  if (!v || !V || !H) return LSA_ERR_ARG;
  if (variant < LSA_MGS || variant > LSA_IOCGS) return LSA_ERR_ARG;
  long long N = lsa_op_dof(op);
  if (N < 1 || m > N) return LSA_ERR_ARG;
  Prepared pr;
  lsa_status st = prepare(op, m, precision, work, work_bytes, &pr);
  if (st != LSA_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  ArnoldiParams P = pr.P;
  P.vin = v;
  P.H = H;
  P.variant = variant;
  P.write_vlast = 1;
  CallTimer tm(stats != nullptr, s);
  cudaError_t e = launch_init(P.ctl, pr.d, (float*)pr.d.g0, (float*)pr.d.g1, precision, H,
                              (m + 1) * m, v, P.V, s, use_stream(P, precision) ? P.E : nullptr);
  tm.mark(0);
  if (e == cudaSuccess) e = launch_arnoldi(P, precision, pr.L.G, s);
  tm.mark(1);
  if (e == cudaSuccess)
    e = launch_copy_basis(V, P.V, precision, N, m, P.ctl, is_hybrid(variant) ? 1 : 0, s);
  if (e != cudaSuccess) return LSA_ERR_CUDA;
  if (stats) {
    lsa_status r = fill_stats(P.ctl, stats, s);
    stats->ms_arnoldi = tm.ms(0, 1);
    stats->launches = 3;
    stats->arnoldi_kernel = arnoldi_kernel_kind(P, precision);
    return r;
  }
  return LSA_OK;
}

lsa_status lsa_phiv(const lsa_op* op, const double* v, double h, int p, int m, double tol,
                    int variant, int precision, double* y, void* work, size_t work_bytes,
                    lsa_stats* stats, void* stream) {
  if (!v || !y) return LSA_ERR_ARG;
  if (variant < LSA_MGS || variant > LSA_IOCGS) return LSA_ERR_ARG;
  if (p < 0 || p > PMAX || !isfinite(h) || isnan(tol)) return LSA_ERR_ARG;
  long long N = lsa_op_dof(op);
  if (N < 1 || m < 1) return LSA_ERR_ARG;
  if (m > N) m = (int)N;
  Prepared pr;
  lsa_status st = prepare(op, m, precision, work, work_bytes, &pr);
  if (st != LSA_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  ArnoldiParams P = pr.P;
  P.vin = v;
  P.variant = variant;
  P.write_vlast = 0;
  CallTimer tm(stats != nullptr, s);
  cudaError_t e = launch_init(P.ctl, pr.d, (float*)pr.d.g0, (float*)pr.d.g1, precision, P.H,
                              (m + 1) * m, v, P.V, s, use_stream(P, precision) ? P.E : nullptr);
  tm.mark(0);
  SmallParams S;
  memset(&S, 0, sizeof(S));
  S.H = P.H;
  S.ldh = m + 1;
  S.ctl_in = P.ctl;
  S.ctl = P.ctl;
  S.m = m;
  S.p = p;
  S.h = h;
  S.mats = (double*)(pr.w + pr.L.small);
  S.C = (double*)(pr.w + pr.L.coefs);
  S.ldc = MMAX + 2;
  S.scale_out = 1;
  S.timeout_ns = kTimeoutNs;
  S.tol = tol;
  // the single-cluster kernel runs S1-S6 in one launch
  const bool fused = use_cluster(P, precision);
  if (fused) {
    if (e == cudaSuccess) e = launch_arnoldi_cluster_advdiff2d(P, &S, y, s);
    tm.mark(1);
    tm.mark(2);
    tm.mark(3);
  } else {
    if (e == cudaSuccess) e = launch_arnoldi(P, precision, pr.L.G, s);
    tm.mark(1);
    if (e == cudaSuccess) e = launch_expm(S, s);
    tm.mark(2);
    if (e == cudaSuccess) e = launch_combine(P.V, precision, N, S.C, S.ldc, p, P.ctl, y, s);
    tm.mark(3);
  }
  if (e != cudaSuccess) return LSA_ERR_CUDA;
  if (stats) {
    lsa_status r = fill_stats(P.ctl, stats, s);
    stats->ms_arnoldi = tm.ms(0, 1);
    stats->ms_expm = tm.ms(1, 2);
    stats->ms_combine = tm.ms(2, 3);
    stats->launches = fused ? 2 : 4;
    stats->arnoldi_kernel = arnoldi_kernel_kind(P, precision);
    return r;
  }
  return LSA_OK;
}

lsa_status lsa_tune_step(const lsa_op* op, const double* v, int m, int variant, int precision,
                         void* work, size_t work_bytes, int reps, int* two_phase, float* ms_one,
                         float* ms_two, void* stream) {
  if (two_phase) *two_phase = 0;
  if (ms_one) *ms_one = 0.f;
  if (ms_two) *ms_two = 0.f;
  if (!v) return LSA_ERR_ARG;
  if (variant < LSA_MGS || variant > LSA_IOCGS) return LSA_ERR_ARG;
  const long long N = lsa_op_dof(op);
  if (N < 1 || m < 1) return LSA_ERR_ARG;
  if (m > N) m = (int)N;
  if (reps < 1) reps = 1;
  Prepared pr;
  lsa_status st = prepare(op, m, precision, work, work_bytes, &pr);
  if (st != LSA_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  ArnoldiParams P = pr.P;
  P.vin = v;
  P.variant = variant;
  P.write_vlast = 0;
  if (!two_phase_applies(P, precision)) return LSA_OK;
  StepKey key;
  if (!step_key(P, precision, &key)) return LSA_ERR_CUDA;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return LSA_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return LSA_ERR_CUDA;
  }
  const int nforms = flat_fits(P, precision) ? 3 : 2;
  float best[3] = {1e30f, 1e30f, 1e30f};
  lsa_status result = LSA_OK;
  for (int form = 0; form < nforms && result == LSA_OK; ++form) {
    g_step_force = form;
    for (int r = 0; r <= reps; ++r) {           // r = 0: warm-up
      cudaError_t e = launch_init(P.ctl, pr.d, (float*)pr.d.g0, (float*)pr.d.g1, precision, P.H,
                                  (m + 1) * m, v, P.V, s, nullptr);
      if (e == cudaSuccess) e = cudaEventRecord(e0, s);
      if (e == cudaSuccess) e = launch_arnoldi(P, precision, pr.L.G, s);
      if (e == cudaSuccess) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) {
        result = LSA_ERR_CUDA;
        break;
      }
      lsa_stats one;
      const lsa_status rs = fill_stats(P.ctl, &one, s);
      if (rs < 0) {
        result = rs;
        break;
      }
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      if (r > 0 && t < best[form]) best[form] = t;
    }
  }
  g_step_force = -1;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (result != LSA_OK) return result;
  int choice = 0;
  for (int form = 1; form < nforms; ++form)
    if (best[form] < best[choice]) choice = form;
  {
    std::lock_guard<std::mutex> lock(g_step_mu);
    g_step_choice[key] = choice;
  }
  if (two_phase) *two_phase = choice;
  if (ms_one) *ms_one = best[0];
  if (ms_two) *ms_two = best[1] < best[2] ? best[1] : best[2];
  return LSA_OK;
}

lsa_status lsa_phiv_host(const lsa_op* op, const double* v_host, double h, int p, int m, double tol,
                         int variant, int precision, double* y_host, double* v_dev, double* y_dev,
                         void* work, size_t work_bytes, void* stream) {
  if (!v_host || !y_host || !v_dev || !y_dev) return LSA_ERR_ARG;
  const long long N = lsa_op_dof(op);
  if (N < 1 || p < 0 || p > PMAX) return LSA_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(v_dev, v_host, (size_t)N * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return LSA_ERR_CUDA;
  lsa_status st = lsa_phiv(op, v_dev, h, p, m, tol, variant, precision, y_dev, work, work_bytes, nullptr, stream);
  if (st < 0) return st;
  if (cudaMemcpyAsync(y_host, y_dev, (size_t)(p + 1) * N * sizeof(double), cudaMemcpyDeviceToHost, s) !=
      cudaSuccess)
    return LSA_ERR_CUDA;
  return st;
}

lsa_status lsa_phiv_lincomb(const lsa_op* op, const double* b, int p, double tau, int nsub, int m,
                            double tol, int variant, int precision, double* u, void* work,
                            size_t work_bytes, lsa_stats* stats, void* stream) {
  if (!b || !u) return LSA_ERR_ARG;
  if (variant < LSA_MGS || variant > LSA_IOCGS || precision != LSA_FP64) return LSA_ERR_ARG;
  if (p < 0 || p > PMAX || !isfinite(tau) || nsub < 1 || nsub > (1 << 20) || isnan(tol))
    return LSA_ERR_ARG;
  if (!op || op->kind > LSA_OP_ADR3D) return LSA_ERR_ARG;
  long long N = lsa_op_dof(op);
  if (N < 1 || m < 1) return LSA_ERR_ARG;
  if (m > N + p) m = (int)(N + p);
  Prepared pr;
  lsa_status st = prepare(op, m, precision, work, work_bytes, &pr);
  if (st != LSA_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const double dt = tau / nsub;
  lsa_stats acc;
  memset(&acc, 0, sizeof(acc));
  acc.m_eff = m;
  lsa_status worst = LSA_OK;
  for (int k = 0; k < nsub; ++k) {
    // sub-step k: [u; xi] <- exp(dt Aaug) [u; xi], xi = exp(k dt K) e_p exactly
    ArnoldiParams P = pr.P;
    P.vin = (k == 0) ? b : u;
    P.variant = variant;
    P.write_vlast = 0;
    P.naug = p;
    P.baug = b;
    P.aug_t = k * dt;
    CallTimer tm(stats != nullptr, s);
    cudaError_t e = launch_init(P.ctl, pr.d, nullptr, nullptr, precision, P.H, (m + 1) * m, P.vin, P.V, s);
    tm.mark(0);
    if (e == cudaSuccess) e = launch_arnoldi(P, precision, pr.L.G, s);
    tm.mark(1);
    SmallParams S;
    memset(&S, 0, sizeof(S));
    S.H = P.H;
    S.ldh = m + 1;
    S.ctl_in = P.ctl;
    S.ctl = P.ctl;
    S.m = m;
    S.p = 0;
    S.h = dt;
    S.mats = (double*)(pr.w + pr.L.small);
    S.C = (double*)(pr.w + pr.L.coefs);
    S.ldc = MMAX + 2;
    S.scale_out = 1;
    S.timeout_ns = kTimeoutNs;
    S.tol = tol;
    if (e == cudaSuccess) e = launch_expm(S, s);
    tm.mark(2);
    if (e == cudaSuccess) e = launch_combine(P.V, precision, N, S.C, S.ldc, 0, P.ctl, u, s);
    tm.mark(3);
    if (e != cudaSuccess) return LSA_ERR_CUDA;
    if (stats) {
      lsa_stats one;
      lsa_status r = fill_stats(P.ctl, &one, s);
      if (one.m_eff < acc.m_eff) acc.m_eff = one.m_eff;
      acc.breakdown |= one.breakdown;
      acc.norm_fallbacks += one.norm_fallbacks;
      acc.grid_syncs += one.grid_syncs;
      acc.grid_barriers += one.grid_barriers;
      if (k == 0) acc.beta = one.beta;
      if (one.err_est > acc.err_est) acc.err_est = one.err_est;
      acc.h_last = one.h_last;
      acc.ms_arnoldi += tm.ms(0, 1);
      acc.ms_expm += tm.ms(1, 2);
      acc.ms_combine += tm.ms(2, 3);
      acc.launches += 4;
      acc.arnoldi_kernel = arnoldi_kernel_kind(P, precision);
      if (r < 0) { acc.status = r; *stats = acc; return r; }
      if (r > worst) worst = r;
    }
  }
  if (stats) {
    acc.status = worst;
    *stats = acc;
  }
  return worst;
}

// Step-size factor of the adaptive sub-steps: 0.9 (tol/err)^(1/(m+1)) clamped
// to [0.2, 4]; 4 when the projection was exact (this library's controller).
static double lincomb_step_factor(double err, double tol_abs, int m) {
  if (!(err > 0.0)) return 4.0;
  const double f = 0.9 * pow(tol_abs / err, 1.0 / (m + 1));
  return f < 0.2 ? 0.2 : (f > 4.0 ? 4.0 : f);
}

lsa_status lsa_phiv_lincomb_adaptive(const lsa_op* op, const double* b, int p, double tau, double tol,
                                     int m, int nsub0, int max_substeps, int variant, int precision,
                                     double* u, double* scratch, void* work, size_t work_bytes,
                                     lsa_stats* stats, int* substeps, int* rejected, void* stream) {
  if (!b || !u || !scratch || u == scratch) return LSA_ERR_ARG;
  if (variant < LSA_MGS || variant > LSA_IOCGS || precision != LSA_FP64) return LSA_ERR_ARG;
  if (p < 0 || p > PMAX || !isfinite(tau) || !(tol > 0.0) || !isfinite(tol) || nsub0 < 1 ||
      max_substeps < 1)
    return LSA_ERR_ARG;
  if (!op || op->kind > LSA_OP_ADR3D) return LSA_ERR_ARG;
  long long N = lsa_op_dof(op);
  if (N < 1 || m < 1) return LSA_ERR_ARG;
  if (m > N + p) m = (int)(N + p);
  Prepared pr;
  lsa_status st = prepare(op, m, precision, work, work_bytes, &pr);
  if (st != LSA_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  lsa_stats acc;
  memset(&acc, 0, sizeof(acc));
  acc.m_eff = m;
  const double* cur = b;                       // the accepted state (b_0 at t = 0)
  double t = 0.0, dt = tau / nsub0;
  const double floor_dt = fabs(tau) * ldexp(1.0, -30);
  int nacc = 0, nrej = 0;
  bool done = false, converged = true;
  lsa_status worst = LSA_OK;
  while (nacc + nrej < max_substeps) {
    const bool last = fabs(dt) >= fabs(tau - t);
    if (last) dt = tau - t;
    double* out = (u != cur) ? u : scratch;    // never the accepted state
    ArnoldiParams P = pr.P;
    P.vin = cur;
    P.variant = variant;
    P.write_vlast = 0;
    P.naug = p;
    P.baug = b;
    P.aug_t = t;
    CallTimer tm(stats != nullptr, s);
    cudaError_t e = launch_init(P.ctl, pr.d, nullptr, nullptr, precision, P.H, (m + 1) * m, P.vin, P.V, s);
    tm.mark(0);
    if (e == cudaSuccess) e = launch_arnoldi(P, precision, pr.L.G, s);
    tm.mark(1);
    SmallParams S;
    memset(&S, 0, sizeof(S));
    S.H = P.H;
    S.ldh = m + 1;
    S.ctl_in = P.ctl;
    S.ctl = P.ctl;
    S.m = m;
    S.p = 0;
    S.h = dt;
    S.mats = (double*)(pr.w + pr.L.small);
    S.C = (double*)(pr.w + pr.L.coefs);
    S.ldc = MMAX + 2;
    S.scale_out = 1;
    S.timeout_ns = kTimeoutNs;
    S.tol = 0.0;
    if (e == cudaSuccess) e = launch_expm(S, s);
    tm.mark(2);
    if (e == cudaSuccess) e = launch_combine(P.V, precision, N, S.C, S.ldc, 0, P.ctl, out, s);
    tm.mark(3);
    if (e != cudaSuccess) return LSA_ERR_CUDA;
    lsa_stats one;
    lsa_status r = fill_stats(P.ctl, &one, s);  // the controller needs the estimate on the host
    if (r < 0) {
      if (stats) { acc.status = r; *stats = acc; }
      return r;
    }
    acc.grid_syncs += one.grid_syncs;
    acc.grid_barriers += one.grid_barriers;
    acc.norm_fallbacks += one.norm_fallbacks;
    acc.ms_arnoldi += tm.ms(0, 1);
    acc.ms_expm += tm.ms(1, 2);
    acc.ms_combine += tm.ms(2, 3);
    acc.launches += 4;
    const double err = one.breakdown ? 0.0 : one.err_est;
    const double tol_abs = tol * one.beta;
    if (err <= tol_abs || fabs(dt) <= floor_dt) {
      if (err > tol_abs) converged = false;
      cur = out;
      ++nacc;
      if (one.m_eff < acc.m_eff) acc.m_eff = one.m_eff;
      acc.breakdown |= one.breakdown;
      if (nacc == 1) acc.beta = one.beta;
      if (one.err_est > acc.err_est) acc.err_est = one.err_est;
      acc.h_last = one.h_last;
      if (r == LSA_BREAKDOWN && worst == LSA_OK) worst = LSA_BREAKDOWN;
      if (last) { done = true; break; }
      t += dt;
      dt *= lincomb_step_factor(err, tol_abs, m);
    } else {
      ++nrej;
      const double f = lincomb_step_factor(err, tol_abs, m);
      dt *= f < 0.9 ? f : 0.9;
    }
  }
  if (cur != u) {
    if (cudaMemcpyAsync(u, cur, (size_t)N * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return LSA_ERR_CUDA;
  }
  if (!done || !converged) worst = LSA_NOT_CONVERGED;
  if (substeps) *substeps = nacc;
  if (rejected) *rejected = nrej;
  if (stats) {
    acc.status = worst;
    acc.arnoldi_kernel = 0;
    *stats = acc;
  }
  return worst;
}

// Sub-steps with adaptive size and Krylov dimension (this library's rule):
// after a projection of dimension m over dt with estimate err, the error model
// err(dt', m') = err kappa^(m - m') (dt'/dt)^(m'+1) -- kappa, the decay of the
// estimate per Krylov dimension, measured on the same projection between
// m - kAdaptProbe and m -- gives for every m' the size factor
// f(m') = 0.9 (tol beta / (err kappa^(m - m')))^(1/(m'+1)) in [0.2, 4], and the
// next sub-step takes the m' of smallest modeled cost per unit of time
// W(m') / f(m'), W(m) = m(m+1)/2 + 3m (vectors one m-step hybrid projection
// streams), when it beats keeping m by 10 %.  After a rejection only m' >= m
// is considered and f is capped at 0.9.  Without a usable kappa (exact
// projection, breakdown, m - kAdaptProbe < 1, kappa <= 1.05) only the size
// adapts, as in lsa_phiv_lincomb_adaptive.
constexpr int kAdaptProbe = 2;
constexpr double kKappaMin = 1.05;
constexpr double kAdaptHyst = 0.9;

static double adapt_cost(int m) { return 0.5 * m * (m + 1) + 3.0 * m; }

static void adapt_plan(double kappa, int m, double err, double tol_abs, int m_min, int m_max, bool accepted,
                       int* m_next, double* f_next) {
  double f_keep = lincomb_step_factor(err, tol_abs, m);
  if (!accepted && f_keep > 0.9) f_keep = 0.9;
  *m_next = m;
  *f_next = f_keep;
  if (!(kappa > 0.0)) return;
  const double keep = adapt_cost(m) / f_keep;
  double best = keep, best_f = f_keep;
  int best_m = m;
  for (int mp = accepted ? m_min : m; mp <= m_max; ++mp) {
    if (mp == m) continue;
    double f = 0.9 * pow(tol_abs / (err * pow(kappa, (double)(m - mp))), 1.0 / (mp + 1));
    f = f < 0.2 ? 0.2 : (f > 4.0 ? 4.0 : f);
    if (!accepted && f > 0.9) f = 0.9;
    const double c = adapt_cost(mp) / f;
    if (c < best) { best = c; best_m = mp; best_f = f; }
  }
  if (best < kAdaptHyst * keep) { *m_next = best_m; *f_next = best_f; }
}

struct AdaptLayout {
  size_t main, pctl, pc, total;
};

static bool adapt_layout(const lsa_op* op, int m_max, AdaptLayout* L) {
  const size_t w = lsa_workspace_bytes(op, m_max, 0, LSA_FP64);
  if (!w) return false;
  L->main = 0;
  L->pctl = align256(w);
  L->pc = L->pctl + align256(sizeof(Ctl));
  L->total = L->pc + align256((size_t)2 * (MMAX + 2) * sizeof(double));
  return true;
}

size_t lsa_lincomb_adaptive_m_workspace_bytes(const lsa_op* op, int m_max) {
  if (!op || op->kind > LSA_OP_ADR3D || m_max < 1 || m_max > MMAX) return 0;
  AdaptLayout L;
  return adapt_layout(op, m_max, &L) ? L.total : 0;
}

lsa_status lsa_phiv_lincomb_adaptive_m(const lsa_op* op, const double* b, int p, double tau, double tol,
                                       int m0, int m_min, int m_max, int nsub0, int max_substeps,
                                       int variant, double* u, double* scratch, void* work,
                                       size_t work_bytes, lsa_stats* stats, int* substeps, int* rejected,
                                       int* dims, int dims_cap, void* stream) {
  if (!b || !u || !scratch || u == scratch) return LSA_ERR_ARG;
  if (variant < LSA_MGS || variant > LSA_IOCGS) return LSA_ERR_ARG;
  if (p < 0 || p > PMAX || !isfinite(tau) || !(tol > 0.0) || !isfinite(tol) || nsub0 < 1 ||
      max_substeps < 1 || dims_cap < 0 || (dims_cap > 0 && !dims))
    return LSA_ERR_ARG;
  if (!op || op->kind > LSA_OP_ADR3D) return LSA_ERR_ARG;
  if (m_min < 1 || m_max < m_min || m_max > MMAX || m0 < 1) return LSA_ERR_ARG;
  const long long N = lsa_op_dof(op);
  if (N < 1) return LSA_ERR_ARG;
  if (m_max > N + p) m_max = (int)(N + p);
  if (m_min > m_max) m_min = m_max;
  int m = m0 < m_min ? m_min : (m0 > m_max ? m_max : m0);
  AdaptLayout AL;
  if (!adapt_layout(op, m_max, &AL)) return LSA_ERR_ARG;
  if (!work || !aligned256(work) || work_bytes < AL.total) return LSA_ERR_WORKSPACE;
  char* wbase = (char*)work;
  Ctl* pctl = (Ctl*)(wbase + AL.pctl);       // the probe exponential's control block
  double* pc = (double*)(wbase + AL.pc);     // ... and its coefficients (2 x (MMAX + 2))
  cudaStream_t s = (cudaStream_t)stream;
  lsa_stats acc;
  memset(&acc, 0, sizeof(acc));
  acc.m_eff = m_max;
  const double* cur = b;
  double t = 0.0, dt = tau / nsub0;
  const double floor_dt = fabs(tau) * ldexp(1.0, -30);
  int nacc = 0, nrej = 0;
  bool done = false, converged = true;
  lsa_status worst = LSA_OK;
  while (nacc + nrej < max_substeps) {
    const bool last = fabs(dt) >= fabs(tau - t);
    if (last) dt = tau - t;
    double* out = (u != cur) ? u : scratch;
    Prepared pr;
    lsa_status st = prepare(op, m, LSA_FP64, work, AL.pctl, &pr);   // layout of this sub-step's m
    if (st != LSA_OK) return st;
    ArnoldiParams P = pr.P;
    P.vin = cur;
    P.variant = variant;
    P.write_vlast = 0;
    P.naug = p;
    P.baug = b;
    P.aug_t = t;
    CallTimer tm(stats != nullptr, s);
    cudaError_t e = launch_init(P.ctl, pr.d, nullptr, nullptr, LSA_FP64, P.H, (m + 1) * m, P.vin, P.V, s);
    tm.mark(0);
    if (e == cudaSuccess) e = launch_arnoldi(P, LSA_FP64, pr.L.G, s);
    tm.mark(1);
    SmallParams S;
    memset(&S, 0, sizeof(S));
    S.H = P.H;
    S.ldh = m + 1;
    S.ctl_in = P.ctl;
    S.ctl = P.ctl;
    S.m = m;
    S.p = 0;
    S.h = dt;
    S.mats = (double*)(pr.w + pr.L.small);
    S.C = (double*)(pr.w + pr.L.coefs);
    S.ldc = MMAX + 2;
    S.scale_out = 1;
    S.timeout_ns = kTimeoutNs;
    S.tol = 0.0;
    if (e == cudaSuccess) e = launch_expm(S, s);
    tm.mark(2);
    if (e == cudaSuccess) e = launch_combine(P.V, LSA_FP64, N, S.C, S.ldc, 0, P.ctl, out, s);
    tm.mark(3);
    if (e != cudaSuccess) return LSA_ERR_CUDA;
    lsa_stats one;
    lsa_status r = fill_stats(P.ctl, &one, s);   // the controller reads the estimate on the host
    if (r < 0) {
      if (stats) { acc.status = r; *stats = acc; }
      return r;
    }
    acc.grid_syncs += one.grid_syncs;
    acc.grid_barriers += one.grid_barriers;
    acc.norm_fallbacks += one.norm_fallbacks;
    acc.ms_arnoldi += tm.ms(0, 1);
    acc.ms_expm += tm.ms(1, 2);
    acc.ms_combine += tm.ms(2, 3);
    acc.launches += 4;
    const double err = one.breakdown ? 0.0 : one.err_est;
    const double tol_abs = tol * one.beta;
    const bool accept = err <= tol_abs || fabs(dt) <= floor_dt;
    // kappa: the same projection's estimate at dimension mp = m - kAdaptProbe,
    // beta dt H_{mp+1,mp} |e_mp^T phi_1(dt H_mp) e_1| (one more small exponential)
    double kappa = 0.0;
    const int mp = m - kAdaptProbe;
    if (!one.breakdown && one.m_eff == m && err > 0.0 && mp >= 1) {
      if (cudaMemsetAsync(pctl, 0, sizeof(Ctl), s) != cudaSuccess) return LSA_ERR_CUDA;
      SmallParams Q;
      memset(&Q, 0, sizeof(Q));
      Q.H = P.H;
      Q.ldh = m + 1;
      Q.ctl_in = nullptr;
      Q.ctl = pctl;
      Q.m = mp;
      Q.p = 0;
      Q.h = dt;
      Q.mats = S.mats;
      Q.C = pc;
      Q.ldc = MMAX + 2;
      Q.scale_out = 0;
      Q.timeout_ns = kTimeoutNs;
      if (launch_expm(Q, s) != cudaSuccess) return LSA_ERR_CUDA;
      acc.launches += 2;
      double hsub = 0.0, phin = 0.0;
      int pst = 0;
      if (cudaMemcpyAsync(&hsub, P.H + mp + (size_t)(mp - 1) * (m + 1), sizeof(double), cudaMemcpyDeviceToHost,
                          s) != cudaSuccess ||
          cudaMemcpyAsync(&phin, pc + (MMAX + 2) + (mp - 1), sizeof(double), cudaMemcpyDeviceToHost, s) !=
              cudaSuccess ||
          cudaMemcpyAsync(&pst, &pctl->status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess)
        return LSA_ERR_CUDA;
      if (pst < 0) return (lsa_status)pst;
      const double e_p = one.beta * fabs(dt) * hsub * fabs(phin);
      if (e_p > err) {
        const double k = pow(e_p / err, 1.0 / kAdaptProbe);
        if (k > kKappaMin) kappa = k;
      }
    }
    if (accept) {
      if (err > tol_abs) converged = false;
      cur = out;
      if (dims && nacc < dims_cap) dims[nacc] = m;
      ++nacc;
      if (one.m_eff < acc.m_eff) acc.m_eff = one.m_eff;
      acc.breakdown |= one.breakdown;
      if (nacc == 1) acc.beta = one.beta;
      if (one.err_est > acc.err_est) acc.err_est = one.err_est;
      acc.h_last = one.h_last;
      if (r == LSA_BREAKDOWN && worst == LSA_OK) worst = LSA_BREAKDOWN;
      if (last) { done = true; break; }
      t += dt;
    } else {
      ++nrej;
    }
    int m_next = m;
    double f = 1.0;
    adapt_plan(kappa, m, err, tol_abs, m_min, m_max, accept, &m_next, &f);
    m = m_next;
    dt *= f;
  }
  if (cur != u) {
    if (cudaMemcpyAsync(u, cur, (size_t)N * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return LSA_ERR_CUDA;
  }
  if (!done || !converged) worst = LSA_NOT_CONVERGED;
  if (substeps) *substeps = nacc;
  if (rejected) *rejected = nrej;
  if (stats) {
    acc.status = worst;
    acc.arnoldi_kernel = 0;
    *stats = acc;
  }
  return worst;
}

lsa_status lsa_expm_phi(const double* H, int ldh, int m, double h, int p, double* C, void* work,
                        size_t work_bytes, void* stream) {
  if (!H || !C || m < 1 || m > MMAX || ldh < m || p < 0 || p > PMAX || !isfinite(h))
    return LSA_ERR_ARG;
  size_t need = align256(sizeof(Ctl)) + (size_t)6 * SMALL_STRIDE * SMALL_STRIDE * sizeof(double);
  if (!work || !aligned256(work) || work_bytes < need) return LSA_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  Ctl* ctl = (Ctl*)work;
  cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(Ctl), s);
  SmallParams S;
  memset(&S, 0, sizeof(S));
  S.H = H;
  S.ldh = ldh;
  S.ctl_in = nullptr;
  S.ctl = ctl;
  S.m = m;
  S.p = p;
  S.h = h;
  S.mats = (double*)((char*)work + align256(sizeof(Ctl)));
  S.C = C;
  S.ldc = m;
  S.scale_out = 0;
  S.timeout_ns = kTimeoutNs;
  if (e == cudaSuccess) e = launch_expm(S, s);
  return from_cuda(e);
}

lsa_status lsa_read_stats(const void* work, lsa_stats* out, void* stream) {
  if (!work) return LSA_ERR_ARG;
  return fill_stats(work, out, (cudaStream_t)stream);
}

lsa_status lsa_selftest_barrier_timeout(void* work, size_t work_bytes, double seconds,
                                        void* stream) {
  if (!work || !aligned256(work) || work_bytes < sizeof(Ctl)) return LSA_ERR_WORKSPACE;
  if (!(seconds > 0.0) || seconds > 10.0) return LSA_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Ctl* ctl = (Ctl*)work;
  cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(Ctl), s);
  if (e == cudaSuccess) e = launch_timeout_selftest(ctl, (long long)(seconds * 1e9), s);
  if (e != cudaSuccess) return LSA_ERR_CUDA;
  lsa_stats st;
  return fill_stats(ctl, &st, s);
}

}  // extern "C"
