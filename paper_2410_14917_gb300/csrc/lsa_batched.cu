// Batched phi products (host side): the plan (instance table, workspace
// layout, cost order), the CTA-group tiling and its tuner, CUDA-graph capture
// and replay, and the per-instance statistics.  The device code is in
// lsa_batched.cuh; the kernels are instantiated per operator in
// lsa_arnoldi_<op>.cu.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "lsa_batched.cuh"

namespace lsa {

cudaError_t launch_batched_advdiff2d(const BatchParams&, int, int, cudaStream_t);
cudaError_t launch_batched_grayscott2d(const BatchParams&, int, int, cudaStream_t);
cudaError_t launch_batched_adr3d(const BatchParams&, int, int, cudaStream_t);
int batched_blocks_per_sm_advdiff2d(int);
int batched_blocks_per_sm_grayscott2d(int);
int batched_blocks_per_sm_adr3d(int);

static const long long kBatchTimeoutNs = 5000000000LL;

// Zero the batch control block, the group mailboxes and every instance's
// control block and H; make the float copies of the operator fields in the
// float32-basis form.  CTA b handles instances b, b + grid, ...
__global__ void k_batch_init(BatchParams BP, int nmail, int precision) {
  if (blockIdx.x == 0) {
    for (int k = threadIdx.x; k < (int)(sizeof(BatchCtl) / sizeof(int)); k += blockDim.x)
      reinterpret_cast<int*>(BP.bctl)[k] = 0;
    for (int k = threadIdx.x; k < nmail * (int)(sizeof(BatchMail) / sizeof(int)); k += blockDim.x)
      reinterpret_cast<int*>(BP.mail)[k] = 0;
  }
  for (int i = blockIdx.x; i < BP.count; i += gridDim.x) {
    const BatchInst& I = BP.inst[i];
    const int nctl = (int)(sizeof(Ctl) / sizeof(int));
    for (int k = threadIdx.x; k < nctl; k += blockDim.x) reinterpret_cast<int*>(I.ctl)[k] = 0;
    const int hc = (I.m + 1) * I.m;
    for (int k = threadIdx.x; k < hc; k += blockDim.x) I.H[k] = 0.0;
    if (precision == LSA_FP32_BASIS) {
      const DevOp& d = I.op;
      if (d.kind == LSA_OP_GRAYSCOTT2D) {
        const long long n = (long long)d.nx * d.ny;
        for (long long k = threadIdx.x; k < n; k += blockDim.x) {
          const double u0 = d.f0[k], v0 = d.f1[k];
          const_cast<float*>(d.g0)[k] = (float)(v0 * v0);
          const_cast<float*>(d.g1)[k] = (float)(2.0 * u0 * v0);
        }
      } else if (d.kind == LSA_OP_ADR3D) {
        for (long long k = threadIdx.x; k < d.npts; k += blockDim.x)
          const_cast<float*>(d.g0)[k] = (float)d.f0[k];
      }
    }
  }
}

static int sm_count_b() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return sms;
}

static int batched_blocks_per_sm(int kind, int precision) {
  if (kind == LSA_OP_ADVDIFF2D) return batched_blocks_per_sm_advdiff2d(precision);
  if (kind == LSA_OP_GRAYSCOTT2D) return batched_blocks_per_sm_grayscott2d(precision);
  return batched_blocks_per_sm_adr3d(precision);
}

// Layout of a batch workspace.  Shared regions first, then per instance: the
// control blocks in one contiguous array (one copy reads all statistics),
// then H, C, the basis block and the float fields of each instance.
struct BatchLayout {
  int G = 0, count = 0;
  size_t bctl = 0, mail = 0, inst = 0, order = 0, partials = 0, T = 0, L = 0, mats = 0;
  size_t ctl = 0, ctl_stride = 0, total = 0;
  std::vector<size_t> H, C, V, g0, g1;
  std::vector<DevOp> d;
  std::vector<int> m;
};

static lsa_status batch_layout(const lsa_op* ops, const int* ms, int count, int p, int precision,
                               BatchLayout* BL) {
  if (!ops || !ms || count < 1) return LSA_ERR_ARG;
  if (precision != LSA_FP64 && precision != LSA_FP32_BASIS) return LSA_ERR_ARG;
  if (p < 0 || p > PMAX) return LSA_ERR_ARG;
  BL->count = count;
  BL->d.resize(count);
  BL->m.resize(count);
  for (int i = 0; i < count; ++i) {
    if (!make_devop(&ops[i], &BL->d[i])) return LSA_ERR_ARG;
    if (BL->d[i].kind > LSA_OP_ADR3D) return LSA_ERR_ARG;     // the three workload operators
    if (BL->d[i].kind != BL->d[0].kind) return LSA_ERR_ARG;   // one operator family per batch
    if (ms[i] < 1 || ms[i] > MMAX) return LSA_ERR_ARG;
    BL->m[i] = (long long)ms[i] > BL->d[i].N ? (int)BL->d[i].N : ms[i];
  }
  const int sms = sm_count_b();
  if (sms <= 0) return LSA_ERR_CUDA;
  int bps = batched_blocks_per_sm(BL->d[0].kind, precision);
  if (bps <= 0) return LSA_ERR_CUDA;
  if (bps > 4) bps = 4;
  const int G = sms * bps;
  BL->G = G;
  const size_t bsz = precision == LSA_FP64 ? 8 : 4;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
  BL->bctl = take(sizeof(BatchCtl));
  BL->mail = take((size_t)G * sizeof(BatchMail));
  BL->inst = take((size_t)count * sizeof(BatchInst));
  BL->order = take((size_t)count * sizeof(int));
  BL->partials = take((size_t)G * SLOTS * sizeof(double));
  BL->T = take((size_t)G * MMAX * MMAX * sizeof(double));
  BL->L = take((size_t)G * MMAX * MMAX * sizeof(double));
  BL->mats = take((size_t)G * kMatsPerWorker * sizeof(double));
  BL->ctl_stride = align256(sizeof(Ctl));
  BL->ctl = take((size_t)count * BL->ctl_stride);
  BL->H.resize(count); BL->C.resize(count); BL->V.resize(count);
  BL->g0.resize(count); BL->g1.resize(count);
  for (int i = 0; i < count; ++i) {
    const DevOp& d = BL->d[i];
    const int m = BL->m[i];
    BL->H[i] = take((size_t)(m + 1) * m * sizeof(double));
    BL->C[i] = take((size_t)(PMAX + 2) * (MMAX + 2) * sizeof(double));
    BL->V[i] = take((size_t)d.N * (m + 3) * bsz);
    size_t nfield = 0;
    if (precision == LSA_FP32_BASIS) {
      if (d.kind == LSA_OP_GRAYSCOTT2D) nfield = (size_t)d.nx * d.ny;
      else if (d.kind == LSA_OP_ADR3D) nfield = (size_t)d.npts;
    }
    BL->g0[i] = take(nfield * sizeof(float));
    BL->g1[i] = take(nfield * sizeof(float));
  }
  BL->total = off;
  return LSA_OK;
}

}  // namespace lsa

using namespace lsa;

struct lsa_batch {
  int count = 0, kind = 0, precision = 0, variant = 0, p = 0;
  double h = 0.0, tol = 0.0;
  int G = 0;
  int gsize = 1, nlarge = 0;
  int two_phase = 0;                 // step form of the hybrid variants
  char* w = nullptr;
  BatchLayout BL;
  std::vector<BatchInst> inst;
  std::vector<int> order;            // instance indices by decreasing cost
  std::vector<double> cost;
  std::vector<long long> voff, yoff;
  long long nv = 0, ny = 0;
  cudaStream_t cap = nullptr;        // private stream used only for graph capture
  cudaGraphExec_t gexec = nullptr;
  const double* gv = nullptr;
  double* gy = nullptr;
  int g_gsize = 0, g_nlarge = -1, g_two = -1;

  BatchParams params(const double* v, double* y) const {
    BatchParams BP;
    memset(&BP, 0, sizeof(BP));
    BP.inst = (const BatchInst*)(w + BL.inst);
    BP.order = (const int*)(w + BL.order);
    BP.count = count;
    BP.nlarge = nlarge;
    BP.gsize = gsize;
    BP.two_phase = two_phase;
    BP.variant = variant;
    BP.p = p;
    BP.h = h;
    BP.tol = tol;
    BP.brk_tol = precision == LSA_FP64 ? 1e-13 : 1e-6;
    BP.timeout_ns = kBatchTimeoutNs;
    BP.bctl = (BatchCtl*)(w + BL.bctl);
    BP.mail = (BatchMail*)(w + BL.mail);
    BP.ws.partials = (double*)(w + BL.partials);
    BP.ws.T = (double*)(w + BL.T);
    BP.ws.L = (double*)(w + BL.L);
    BP.ws.mats = (double*)(w + BL.mats);
    BP.v = v;
    BP.y = y;
    return BP;
  }

  cudaError_t enqueue(const double* v, double* y, cudaStream_t s) const {
    BatchParams BP = params(v, y);
    const int nmail = G;
    int nb = count < G ? count : G;
    if (nb < 1) nb = 1;
    k_batch_init<<<nb, 256, 0, s>>>(BP, nmail, precision);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (kind == LSA_OP_ADVDIFF2D) return launch_batched_advdiff2d(BP, precision, G, s);
    if (kind == LSA_OP_GRAYSCOTT2D) return launch_batched_grayscott2d(BP, precision, G, s);
    return launch_batched_adr3d(BP, precision, G, s);
  }

  void drop_graph() {
    if (gexec) cudaGraphExecDestroy(gexec);
    gexec = nullptr;
    gv = nullptr;
    gy = nullptr;
    g_nlarge = -1;
    g_two = -1;
  }

  ~lsa_batch() {
    drop_graph();
    if (cap) cudaStreamDestroy(cap);
  }
};

extern "C" {

size_t lsa_batch_workspace_bytes(const lsa_op* ops, const int* m, int count, int p, int precision) {
  BatchLayout BL;
  if (batch_layout(ops, m, count, p, precision, &BL) != LSA_OK) return 0;
  return BL.total;
}

lsa_status lsa_batch_create(const lsa_op* ops, const int* m, int count, double h, int p,
                            double tol, int variant, int precision, void* work, size_t work_bytes,
                            lsa_batch** out, void* stream) {
  if (!out) return LSA_ERR_ARG;
  *out = nullptr;
  if (variant < LSA_MGS || variant > LSA_IOCGS) return LSA_ERR_ARG;
  if (!isfinite(h) || isnan(tol)) return LSA_ERR_ARG;
  lsa_batch* b = new (std::nothrow) lsa_batch();
  if (!b) return LSA_ERR_ARG;
  lsa_status st = batch_layout(ops, m, count, p, precision, &b->BL);
  if (st != LSA_OK) { delete b; return st; }
  if (!work || ((uintptr_t)work & 255u) || work_bytes < b->BL.total) { delete b; return LSA_ERR_WORKSPACE; }
  b->w = (char*)work;
  b->count = count;
  b->kind = b->BL.d[0].kind;
  b->precision = precision;
  b->variant = variant;
  b->p = p;
  b->h = h;
  b->tol = tol;
  b->G = b->BL.G;
  b->inst.resize(count);
  b->voff.resize(count);
  b->yoff.resize(count);
  b->cost.resize(count);
  long long nv = 0, ny = 0;
  for (int i = 0; i < count; ++i) {
    BatchInst& I = b->inst[i];
    memset(&I, 0, sizeof(I));
    I.op = b->BL.d[i];
    if (precision == LSA_FP32_BASIS) {
      I.op.g0 = (const float*)(b->w + b->BL.g0[i]);
      I.op.g1 = (const float*)(b->w + b->BL.g1[i]);
    }
    I.tl = make_tiling(I.op);
    I.m = b->BL.m[i];
    I.voff = nv;
    I.yoff = ny;
    I.ctl = (Ctl*)(b->w + b->BL.ctl + (size_t)i * b->BL.ctl_stride);
    I.H = (double*)(b->w + b->BL.H[i]);
    I.C = (double*)(b->w + b->BL.C[i]);
    I.V = b->w + b->BL.V[i];
    b->voff[i] = nv;
    b->yoff[i] = ny;
    nv += I.op.N;
    ny += (long long)(p + 1) * I.op.N;
    // streamed columns of m Arnoldi steps: sum_j (j + 3) ~ m(m+7)/2, times N
    b->cost[i] = (double)I.op.N * (0.5 * I.m * (I.m + 7.0));
  }
  b->nv = nv;
  b->ny = ny;
  b->order.resize(count);
  std::iota(b->order.begin(), b->order.end(), 0);
  std::stable_sort(b->order.begin(), b->order.end(),
                   [&](int a, int c) { return b->cost[a] > b->cost[c]; });
  // default tiling: groups of 4 CTAs take every instance (in cost order) that
  // has at least one tile per CTA of the group; single CTAs take the rest.
  // (On the 512-instance advection-diffusion batch this is the tuner's pick
  // for both precisions; a single CTA per instance leaves the largest ones as
  // a long tail.)
  b->gsize = b->G >= 4 ? 4 : 1;
  int nl = 0;
  if (b->gsize > 1)
    while (nl < count && b->inst[b->order[nl]].tl.ntiles >= b->gsize) ++nl;
  b->nlarge = nl;
  if (b->nlarge == 0) b->gsize = 1;
  // default step form of the hybrid variants: two-phase (its barrier between
  // the passes counts only an instance's group; faster in both precisions on
  // the 512-instance advection-diffusion batch)
  b->two_phase = is_hybrid(variant) ? 1 : 0;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(b->w + b->BL.inst, b->inst.data(), (size_t)count * sizeof(BatchInst),
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->w + b->BL.order, b->order.data(), (size_t)count * sizeof(int),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { delete b; return LSA_ERR_CUDA; }
  *out = b;
  return LSA_OK;
}

void lsa_batch_destroy(lsa_batch* b) { delete b; }

lsa_status lsa_batch_info(const lsa_batch* b, int* ctas, int* group_size, int* nlarge,
                          long long* v_elems, long long* y_elems, long long* voff, long long* yoff) {
  if (!b) return LSA_ERR_ARG;
  if (ctas) *ctas = b->G;
  if (group_size) *group_size = b->gsize;
  if (nlarge) *nlarge = b->nlarge;
  if (v_elems) *v_elems = b->nv;
  if (y_elems) *y_elems = b->ny;
  if (voff) memcpy(voff, b->voff.data(), sizeof(long long) * b->count);
  if (yoff) memcpy(yoff, b->yoff.data(), sizeof(long long) * b->count);
  return LSA_OK;
}

lsa_status lsa_batch_set_tiling(lsa_batch* b, int group_size, int nlarge) {
  if (!b) return LSA_ERR_ARG;
  if (nlarge < 0 || nlarge > b->count) return LSA_ERR_ARG;
  if (group_size < 1 || group_size > b->G) return LSA_ERR_ARG;
  b->gsize = group_size;
  b->nlarge = nlarge;
  return LSA_OK;
}

lsa_status lsa_batch_set_step_form(lsa_batch* b, int two_phase) {
  if (!b || (two_phase != 0 && two_phase != 1)) return LSA_ERR_ARG;
  b->two_phase = two_phase;
  return LSA_OK;
}

int lsa_batch_step_form(const lsa_batch* b) { return b ? b->two_phase : -1; }

lsa_status lsa_batch_run(lsa_batch* b, const double* v, double* y, int use_graph, void* stream) {
  if (!b || !v || !y) return LSA_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (!use_graph) return b->enqueue(v, y, s) == cudaSuccess ? LSA_OK : LSA_ERR_CUDA;
  if (!(b->gexec && b->gv == v && b->gy == y && b->g_gsize == b->gsize && b->g_nlarge == b->nlarge &&
        b->g_two == b->two_phase)) {
    b->drop_graph();
    if (!b->cap && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
      b->cap = nullptr;
      return LSA_ERR_CUDA;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return LSA_ERR_CUDA;
    cudaError_t e1 = b->enqueue(v, y, b->cap);
    e = cudaStreamEndCapture(b->cap, &g);
    if (e1 != cudaSuccess || e != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return LSA_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&b->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { b->gexec = nullptr; return LSA_ERR_CUDA; }
    b->gv = v;
    b->gy = y;
    b->g_gsize = b->gsize;
    b->g_two = b->two_phase;
    b->g_nlarge = b->nlarge;
  }
  return cudaGraphLaunch(b->gexec, s) == cudaSuccess ? LSA_OK : LSA_ERR_CUDA;
}

lsa_status lsa_batch_read_stats(const lsa_batch* b, lsa_stats* out, int* finished, void* stream) {
  if (!b) return LSA_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<unsigned char> raw((size_t)b->count * b->BL.ctl_stride);
  BatchCtl bc;
  cudaError_t e = cudaMemcpyAsync(raw.data(), b->w + b->BL.ctl, raw.size(), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&bc, b->w + b->BL.bctl, sizeof(bc), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return LSA_ERR_CUDA;
  lsa_status worst = (lsa_status)(bc.status < 0 ? bc.status : 0);
  for (int i = 0; i < b->count; ++i) {
    Ctl c;
    memcpy(&c, raw.data() + (size_t)i * b->BL.ctl_stride, sizeof(Ctl));
    int st = c.status;
    if (st >= 0 && !c.finished) st = LSA_ERR_TIMEOUT;
    else if (st == LSA_OK && c.breakdown) st = LSA_BREAKDOWN;
    if (out) {
      lsa_stats& o = out[i];
      memset(&o, 0, sizeof(o));
      o.status = st;
      o.m_eff = c.m_eff;
      o.breakdown = c.breakdown;
      o.norm_fallbacks = c.fallbacks;
      o.grid_syncs = c.syncs;
      o.grid_barriers = c.barriers;
      o.beta = c.beta;
      o.err_est = c.err_est;
      o.h_last = c.h_last;
    }
    // the first error wins; otherwise the largest warning (NOT_CONVERGED > BREAKDOWN)
    if (worst >= 0 && (st < 0 || st > worst)) worst = (lsa_status)st;
  }
  if (finished) *finished = (int)bc.finished;
  return worst;
}

lsa_status lsa_batch_tune(lsa_batch* b, const double* v, double* y, int reps, int* group_size,
                          int* nlarge, float* ms_best, void* stream) {
  if (!b || !v || !y) return LSA_ERR_ARG;
  if (reps < 1) reps = 1;
  cudaStream_t s = (cudaStream_t)stream;
  struct Cand { int g, nl; };
  std::vector<Cand> cands;
  cands.push_back({1, 0});                       // one CTA per instance
  cands.push_back({b->G, b->count});             // the whole grid per instance
  const int fr[] = {64, 32, 16, 8, 4, 2, 1};
  for (int g = 2; g <= 32 && g <= b->G / 2; g *= 2)
    for (int f : fr) {
      int nl = b->count / f;
      if (nl < 1) continue;
      bool dup = false;
      for (const Cand& c : cands) dup |= (c.g == g && c.nl == nl);
      if (!dup) cands.push_back({g, nl});
    }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return LSA_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return LSA_ERR_CUDA; }
  lsa_status result = LSA_OK;
  // best of `reps` timed runs after one warm-up (negative: the run failed)
  auto time_it = [&](int g, int nl, int two) -> float {
    b->gsize = g;
    b->nlarge = nl;
    b->two_phase = two;
    if (b->enqueue(v, y, s) != cudaSuccess) { result = LSA_ERR_CUDA; return -1.f; }
    float tmin = 1e30f;
    for (int r = 0; r < reps; ++r) {
      cudaEventRecord(e0, s);
      if (b->enqueue(v, y, s) != cudaSuccess) { result = LSA_ERR_CUDA; return -1.f; }
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) { result = LSA_ERR_CUDA; return -1.f; }
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      tmin = t < tmin ? t : tmin;
    }
    int fin = 0;
    lsa_status st = lsa_batch_read_stats(b, nullptr, &fin, stream);
    if (st < 0) { result = st; return -1.f; }
    return tmin;
  };
  const int two0 = b->two_phase;
  float best = 1e30f;
  Cand bc = {b->gsize, b->nlarge};
  int btwo = two0;
  for (const Cand& c : cands) {
    const float t = time_it(c.g, c.nl, two0);
    if (t < 0.f) break;
    if (t < best) { best = t; bc = c; }
  }
  // then the other step form of the hybrid variants on the best tiling
  if (result == LSA_OK && is_hybrid(b->variant)) {
    const float t = time_it(bc.g, bc.nl, 1 - two0);
    if (t >= 0.f && t < best) { best = t; btwo = 1 - two0; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->gsize = bc.g;
  b->nlarge = bc.nl;
  b->two_phase = btwo;
  if (group_size) *group_size = bc.g;
  if (nlarge) *nlarge = bc.nl;
  if (ms_best) *ms_best = best;
  return result;
}

lsa_status lsa_phiv_batched(const lsa_op* ops, const int* m, int count, const double* v, double h,
                            int p, double tol, int variant, int precision, double* y, void* work,
                            size_t work_bytes, lsa_stats* stats, void* stream) {
  lsa_batch* b = nullptr;
  lsa_status st = lsa_batch_create(ops, m, count, h, p, tol, variant, precision, work, work_bytes,
                                   &b, stream);
  if (st != LSA_OK) return st;
  st = lsa_batch_run(b, v, y, 0, stream);
  if (st == LSA_OK) st = lsa_batch_read_stats(b, stats, nullptr, stream);
  lsa_batch_destroy(b);
  return st;
}

}  // extern "C"
