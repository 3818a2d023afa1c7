/*
 * lsarnoldi -- Krylov phi-function products with low-synchronisation Arnoldi
 * on one GB300 (sm_103a).  C ABI: plain pointers and sizes only.
 *
 * The library computes, for a matrix-free stencil operator A,
 *     y_k = phi_k(h A) v,   k = 0..p,
 * by an m-step Arnoldi projection (Sect. 2.2, Eq. 13: e^A b ~ ||b|| V_m e^{H_m} e_1)
 * with the phi-functions of Sect. 2 (Eqs. 5-6) read off one exponential of the
 * small augmented Hessenberg matrix (the m-sized analogue of Sect. 2.1, Eqs. 7-9).
 * The Gram-Schmidt step is one of
 *   LSA_MGS     Alg. 1 (modified Gram-Schmidt, j+1 reductions at step j),
 *   LSA_CGS2    classical Gram-Schmidt applied twice (textbook; 3 reductions
 *               per step; Sect. 2.3 discusses classical GS),
 *   LSA_HCWY    Alg. 4 with the compact-WY correction of Alg. 5 (Sect. 3.2.1),
 *   LSA_HNCWY   Alg. 4 with the truncated Neumann correction of Alg. 6 (Sect. 3.2.2),
 *   LSA_HGSMGS  Alg. 4 with the two-sweep Gauss-Seidel correction of Alg. 7 (Sect. 3.2.3);
 * the three hybrid variants need one global reduction per Arnoldi step.
 *
 * Conventions for every entry point:
 *  - Device pointers ("dev") point to memory on the current CUDA device; the
 *    caller owns and allocates every buffer, including the workspace.  The
 *    library never allocates device memory.
 *  - Vectors are contiguous.  Grid index i = ix + nx*(iy + ny*iz), x fastest;
 *    Gray-Scott stacks the species as [u-block; v-block] (N = 2*nx*ny).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Work is enqueued asynchronously.  When `stats` is non-NULL the call
 *    synchronises the stream, fills *stats and returns the device-side status
 *    (which may be LSA_BREAKDOWN, LSA_NOT_CONVERGED or LSA_ERR_TIMEOUT);
 *    with stats == NULL only argument and launch errors are reported, and
 *    lsa_read_stats() retrieves the rest later.
 *  - No exception or longjmp crosses the ABI; errors are status codes.
 *  - Statuses >= 0 leave valid outputs; statuses < 0 leave outputs undefined.
 */
#ifndef LSARNOLDI_H
#define LSARNOLDI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LSA_OK = 0,
  LSA_BREAKDOWN = 1,        /* lucky breakdown at step m_eff < m; result exact in the subspace */
  LSA_NOT_CONVERGED = 2,    /* a-posteriori estimate err_est > tol * beta */
  LSA_ERR_ARG = -1,         /* invalid argument (null pointer, size, enum, m out of range...) */
  LSA_ERR_CUDA = -2,        /* a CUDA runtime call failed */
  LSA_ERR_TIMEOUT = -3,     /* an in-kernel grid barrier gave up waiting (bounded spin) */
  LSA_ERR_NUMERIC = -4,     /* non-finite value in H or in a norm */
  LSA_ERR_WORKSPACE = -5    /* workspace too small or misaligned (needs 256-byte alignment) */
} lsa_status;

typedef enum { LSA_MGS = 0, LSA_CGS2 = 1, LSA_HCWY = 2, LSA_HNCWY = 3, LSA_HGSMGS = 4,
               LSA_IOCGS = 5 } lsa_variant;

/* LSA_FP64: basis, matvec and all reductions in IEEE double.
 * LSA_FP32_BASIS: basis vectors and the stencil matvec in float; inner products
 * with float products, short float runs and compensated (Kahan) accumulation,
 * reduced across the GPU in double; H, the correction matrices, the norm
 * estimate and the small exponential stay in double. */
typedef enum { LSA_FP64 = 0, LSA_FP32_BASIS = 1 } lsa_precision;

typedef enum {
  LSA_OP_ADVDIFF2D = 1,
  LSA_OP_GRAYSCOTT2D = 2,
  LSA_OP_ADR3D = 3,
  LSA_OP_GRAYSCOTT2D_T = 4,        /* LSA_FP64 only */
  LSA_OP_GRAYSCOTT2D_FRECHET = 5   /* LSA_FP64 only */
} lsa_op_kind;

/* Operator descriptor (plain data; the library only borrows the field pointers).
 *  LSA_OP_ADVDIFF2D  periodic nx*ny grid:  A v = diff*Lap5 v - vel[0]*Dx v - vel[1]*Dy v,
 *                    central differences; nz must be 1.
 *  LSA_OP_GRAYSCOTT2D Jacobian of Gray-Scott at (u0, v0) = (field0, field1), each nx*ny:
 *                    [[diff*Lap - v0^2 - F, -2 u0 v0], [v0^2, diff2*Lap + 2 u0 v0 - (F+k)]];
 *                    nz must be 1, N = 2*nx*ny.
 *  LSA_OP_ADR3D      periodic nx*ny*nz grid: A v = diff*Lap7 v - sum_a vel[a]*Upwind_a v + r.*v,
 *                    r = field0 (N values), first-order upwind differences.
 *  LSA_OP_GRAYSCOTT2D_T  the transpose A^T of the Gray-Scott Jacobian (same fields):
 *                    [[diff*Lap - v0^2 - F, v0^2], [-2 u0 v0, diff2*Lap + 2 u0 v0 - (F+k)]].
 *  LSA_OP_GRAYSCOTT2D_FRECHET  the block operator K = [[A, dA/dtheta], [0, A]] of the
 *                    Gray-Scott Jacobian A (same fields) on [a; b], N = 4*nx*ny (four
 *                    species blocks a_u, a_v, b_u, b_v), theta = (diff, diff2, F, k)[aux]:
 *                    dA/ddiff = [[Lap, 0], [0, 0]], dA/ddiff2 = [[0, 0], [0, Lap]],
 *                    dA/dF = -I, dA/dk = [[0, 0], [0, -I]].  The top half of
 *                    phi_1(hK)[0; v] is the derivative of phi_1(hA)v along h*dA/dtheta
 *                    (Sect. 2.1, Eq. 7 with the block-triangular augmentation of the
 *                    Frechet derivative of exp).
 * All operators use the uniform spacing dx in every direction. */
typedef struct {
  int kind;
  int nx, ny, nz;
  double dx;
  double diff;
  double diff2;
  double vel[3];
  double F, k;
  const double* field0;   /* dev, see above; NULL when unused */
  const double* field1;   /* dev, see above; NULL when unused */
  int aux;                /* LSA_OP_GRAYSCOTT2D_FRECHET: derivative direction 0..3; else 0 */
} lsa_op;

typedef struct {
  int status;             /* device-side lsa_status of the last call on this workspace */
  int m_eff;              /* completed Arnoldi steps */
  int breakdown;          /* 1 after a lucky breakdown */
  int norm_fallbacks;     /* explicit-norm fallbacks of the hybrid norm estimate (Alg. 4) */
  int grid_syncs;         /* global reductions performed (in-kernel grid barriers with reduction) */
  int grid_barriers;      /* all grid barriers, including those without a reduction */
  double beta;            /* ||v|| */
  double err_est;         /* beta*h*H_{m+1,m}*|e_m^T phi_{p+1}(h H_m) e_1| (phiv only) */
  double h_last;          /* H_{m+1,m} */
  float ms_arnoldi;       /* device time of the Arnoldi kernel (CUDA events; filled when stats != NULL) */
  float ms_expm;          /* device time of the small exponential (phiv only) */
  float ms_combine;       /* device time of the output combination (phiv only) */
  int launches;           /* kernels this call launched */
  int arnoldi_kernel;     /* Arnoldi kernel that ran: 0 plain loads, 1 TMA-staged tile+halo,
                             2 streaming (interior-only TMA stages), 3 single thread-block
                             cluster, 4 plain loads with the two-phase step, 5 the flat
                             two-phase step (see lsa_tune_step); filled by
                             lsa_arnoldi/lsa_phiv */
} lsa_stats;

/* Largest supported Krylov dimension m. */
int lsa_max_m(void);

/* Library version (major*10000 + minor*100 + patch). */
int lsa_version(void);

/* Human-readable name of a status code (static string). */
const char* lsa_status_string(int status);

/* Number of unknowns N of an operator (-1 if the descriptor is invalid). */
long long lsa_op_dof(const lsa_op* op);

/* Bytes of device workspace needed by lsa_phiv / lsa_arnoldi for (op, m, p,
 * precision) on the current device; 0 if the arguments are invalid.  The
 * workspace must be 256-byte aligned.  Its contents need not be initialised. */
size_t lsa_workspace_bytes(const lsa_op* op, int m, int p, int precision);

/* S1 alone: y = A x.  x, y: dev, N elements of the basis type (double for
 * LSA_FP64, float for LSA_FP32_BASIS).  Uses the same stencil code as the
 * Arnoldi kernels.  work: dev workspace of lsa_workspace_bytes(op, 1, 0, precision). */
lsa_status lsa_matvec(const lsa_op* op, const void* x, void* y, int precision,
                      void* work, size_t work_bytes, void* stream);

/* Arnoldi decomposition A V_m = V_{m+1} Hbar_m (Sect. 2.2, Eq. 12).
 *  v  dev, N doubles: start vector b (not modified).
 *  m  1 <= m <= min(lsa_max_m(), N).
 *  V  dev, N x (m+1) column-major (leading dimension N) of the basis type; on
 *     return columns 0..m_eff hold the orthonormal basis (column m_eff is
 *     v_{m_eff+1}; after a breakdown it is unspecified).
 *  H  dev, (m+1) x m column-major doubles (leading dimension m+1); entries
 *     outside the leading (m_eff+1) x m_eff block are set to zero.
 * Sync count: LSA_MGS j+1 at step j (plus one for ||v||), LSA_CGS2 3 per step
 * (plus one), LSA_IOCGS 2 per step (plus one), hybrid variants 1 per step plus
 * 1 final (plus one per fallback).  With LSA_IOCGS the columns are unit vectors
 * orthogonal to their two predecessors only. */
lsa_status lsa_arnoldi(const lsa_op* op, const double* v, int m, int variant, int precision,
                       void* V, double* H, void* work, size_t work_bytes,
                       lsa_stats* stats, void* stream);

/* Step form of the grid Arnoldi kernel's hybrid variants (Alg. 4 with
 * Algs. 5/6/7).  Form 0, one pass: each tile is projected together with its
 * one-point halo (the halo values are projected again by the neighbouring
 * tile), then the stencil and the inner products, then the reduction: one
 * grid barrier per step.  Form 1, two-phase: every value is projected once
 * (equal flat shares per CTA), a grid barrier without a reduction, then a
 * pass over tiles reads the projected vector back with its halo for the
 * stencil and the inner products: no repeated projection, one more barrier
 * per step; bitwise the basis and H of form 0.  Form 2, flat two-phase (the
 * ADR 3D, advection-diffusion and Gray-Scott operators): the second pass also
 * runs over the equal flat shares,
 * reading the stencil's neighbours through L2, with no tiles; the same
 * stencil values, inner products summed over other groups of points (equal
 * to forms 0 and 1 to rounding).
 * lsa_tune_step times the forms of lsa_arnoldi's Arnoldi kernel that apply
 * on (op, m, variant, precision) and records the fastest; later lsa_arnoldi,
 * lsa_phiv and lsa_phiv_host calls on the current device with the same
 * operator kind and grid, m, variant and precision use it (process-wide
 * table, thread-safe).  LSA_TWO_PHASE=0, 1 or 2 in the environment overrides
 * the table (2 runs form 1 where form 2 does not apply).  Without either:
 * form 2 for float64 3D grids and for 2D grids of at least six 16 x 16 tiles
 * per SM, form 1 for float32-basis 3D grids, form 0 otherwise (the
 * crossovers measured on GB300).
 *  v      dev, N doubles: start vector of the timing runs (not modified).
 *  work   dev workspace of lsa_workspace_bytes(op, m, 0, precision).
 *  reps   timed runs per form (>= 1; one untimed run precedes them).
 *  two_phase  out (may be NULL): the recorded form (0, 1 or 2).
 *  ms_one, ms_two  out (may be NULL): best Arnoldi kernel time of form 0 and
 *         of the fastest two-phase form, in ms.
 * When the forms do not apply (the variant is not hybrid, or the call would
 * run the TMA, streaming or cluster kernel) nothing is timed or recorded and
 * the outputs are 0.  Synchronises the stream. */
lsa_status lsa_tune_step(const lsa_op* op, const double* v, int m, int variant, int precision,
                         void* work, size_t work_bytes, int reps, int* two_phase, float* ms_one,
                         float* ms_two, void* stream);

/* phi products y_k = phi_k(h A) v, k = 0..p (Sect. 2.2, Eq. 13 with the phi
 * augmentation of Sect. 2.1).
 *  v    dev, N doubles.       y  dev, (p+1) x N doubles, y + k*N = phi_k(hA)v.
 *  p    0 <= p <= 8.          m  1 <= m <= lsa_max_m() (capped at N).
 *  h    finite; h = 0 returns y_k = v/k!.
 *  tol  a-posteriori check only (no substepping): LSA_NOT_CONVERGED when
 *       err_est > tol*beta; tol <= 0 disables the check. */
lsa_status lsa_phiv(const lsa_op* op, const double* v, double h, int p, int m, double tol,
                    int variant, int precision, double* y, void* work, size_t work_bytes,
                    lsa_stats* stats, void* stream);

/* Linear combination u = sum_{j=0}^p tau^j phi_j(tau A) b_j of phi-function
 * products (Sect. 2.1, Eqs. 7-9), the quantity an exponential integrator
 * needs per stage.  It is the first N entries of exp(tau Aaug) [b_0; e_p]
 * with the (N+p)-sized augmented operator Aaug = [[A, B], [0, K]],
 * B = [b_p, ..., b_1], K the p x p upper shift.  The Krylov process runs on
 * (N+p)-vectors: the extra p entries of every basis vector are kept beside
 * the basis and the stencil adds B x_bot, so only products with A are formed
 * on the grid (Sect. 2.1).  tau is split into nsub equal sub-steps (Sect. 2.2
 * sub-stepping: [u; xi] <- exp(dt Aaug) [u; xi], where the extra entries
 * follow exp(t K) e_p exactly and restart each sub-step); each sub-step is
 * one Arnoldi projection of dimension m (the paper's KIOPS layer picks sizes
 * and dimensions adaptively by formulas it does not give; here they are the
 * caller's).
 *  b          dev, (p+1) x N doubles: b + j*N = b_j.  Not modified.
 *  p          0 <= p <= 8 (p = 0: u = exp(tau A) b_0).
 *  tau        finite; tau = 0 returns u = b_0.
 *  nsub       sub-steps, 1 <= nsub <= 2^20.
 *  m          1 <= m <= lsa_max_m() per sub-step (capped at N + p).
 *  tol        per sub-step a-posteriori check as lsa_phiv (tol <= 0: off).
 *  op         LSA_OP_ADVDIFF2D, LSA_OP_GRAYSCOTT2D or LSA_OP_ADR3D.
 *  precision  LSA_FP64 only (the float32-basis form returns LSA_ERR_ARG).
 *  u          dev, N doubles; may be b_0 itself but must not overlap b_1..b_p.
 *  work       dev workspace of lsa_workspace_bytes(op, m, 0, LSA_FP64).
 *  stats      summed over the sub-steps (grid syncs, fallbacks, times),
 *             smallest m_eff, largest err_est, beta of the first sub-step;
 *             with stats the call synchronises the stream after each sub-step.
 * Returns the worst informational status of the sub-steps, or the first
 * error. */
lsa_status lsa_phiv_lincomb(const lsa_op* op, const double* b, int p, double tau, int nsub, int m,
                            double tol, int variant, int precision, double* u, void* work,
                            size_t work_bytes, lsa_stats* stats, void* stream);

/* lsa_phiv_lincomb with sub-steps chosen by the a-posteriori estimate of each
 * projection (this library's controller; the paper uses KIOPS's, which it
 * cites but does not give).  A sub-step of size dt from state (t, u_t) is one
 * m-step projection of the augmented operator; with err = beta dt H_{m+1,m}
 * |e_m^T phi_1(dt H_m) e_1| and beta the norm of its augmented start vector it
 * is accepted when err <= tol * beta, and the next size is dt * f,
 * f = 0.9 (tol beta / err)^(1/(m+1)) clamped to [0.2, 4] (4 after an exact
 * projection); a rejected sub-step is retried with dt * min(f, 0.9).  The first
 * size is tau / nsub0; a sub-step shorter than |tau| 2^-30 is accepted
 * regardless.
 *  tol        > 0, relative to beta.      max_substeps  accepted + rejected cap.
 *  u          dev, N doubles: the result; may be b_0 itself.
 *  scratch    dev, N doubles, distinct from u and from b (the trial sub-step
 *             result while u holds the accepted state, or the reverse).
 *  substeps, rejected  (host, may be NULL): accepted and rejected sub-steps.
 *  Other arguments as lsa_phiv_lincomb.  The stream is synchronised after
 *  every sub-step (the controller reads the estimate on the host).
 * Returns LSA_NOT_CONVERGED when a sub-step at the size floor missed the
 * tolerance or max_substeps ended the process before tau (u then holds the
 * last accepted state), LSA_BREAKDOWN after an exact projection, else LSA_OK,
 * or the first error. */
lsa_status lsa_phiv_lincomb_adaptive(const lsa_op* op, const double* b, int p, double tau, double tol,
                                     int m, int nsub0, int max_substeps, int variant, int precision,
                                     double* u, double* scratch, void* work, size_t work_bytes,
                                     lsa_stats* stats, int* substeps, int* rejected, void* stream);

/* lsa_phiv_lincomb_adaptive with the Krylov dimension of every sub-step
 * adaptive as well as its size: Sect. 2.2 chooses both "as in KIOPS", whose
 * formulas the paper does not give, so the rule is this library's own.  After
 * a projection of dimension m over dt with estimate err (as in
 * lsa_phiv_lincomb_adaptive), kappa -- the decay of the estimate per Krylov
 * dimension -- is measured on the same projection (its estimate at dimension
 * m - 2 costs one more small exponential); the error model
 * err(dt', m') = err kappa^(m - m') (dt'/dt)^(m'+1) gives for every m' in
 * [m_min, m_max] the size factor f(m') = 0.9 (tol beta / (err kappa^(m-m')))^(1/(m'+1))
 * clamped to [0.2, 4], and the next sub-step takes the m' with the smallest
 * modeled cost per unit of time (m'(m'+1)/2 + 3m') / f(m') -- the vectors one
 * m'-step projection streams -- when that beats keeping m by 10 %.  After a
 * rejection only m' >= m is considered and f is capped at 0.9.  Without a
 * usable kappa (exact projection, breakdown, m < 3, kappa <= 1.05) only the
 * size adapts.  Acceptance, the first size tau / nsub0 and the size floor are
 * those of lsa_phiv_lincomb_adaptive.
 *  m0         first dimension, clamped to [m_min, m_max];  1 <= m_min <= m_max
 *             <= lsa_max_m() (m_max capped at N + p).
 *  work       dev, lsa_lincomb_adaptive_m_workspace_bytes(op, m_max) bytes,
 *             256-byte aligned.
 *  dims       host, may be NULL when dims_cap = 0: the dimension of each
 *             accepted sub-step, the first dims_cap of them.
 *  Float64 form only; other arguments and the status as
 *  lsa_phiv_lincomb_adaptive (the stream is synchronised after every
 *  sub-step: the controller runs on the host). */
size_t lsa_lincomb_adaptive_m_workspace_bytes(const lsa_op* op, int m_max);
lsa_status lsa_phiv_lincomb_adaptive_m(const lsa_op* op, const double* b, int p, double tau, double tol,
                                       int m0, int m_min, int m_max, int nsub0, int max_substeps,
                                       int variant, double* u, double* scratch, void* work,
                                       size_t work_bytes, lsa_stats* stats, int* substeps, int* rejected,
                                       int* dims, int dims_cap, void* stream);

/* lsa_phiv from and to host memory, for callers whose vectors live on the host:
 * copies v (v_host -> v_dev), runs lsa_phiv into y_dev, copies y back
 * (y_dev -> y_host), all enqueued on `stream` in that order; the call returns
 * once they are enqueued (synchronise the stream before reading y_host).
 *  v_host     host, N doubles (pinned memory lets the copy overlap).
 *  y_host     host, (p+1) x N doubles, row k = phi_k(hA)v.
 *  v_dev      dev, N doubles;  y_dev  dev, (p+1) x N doubles (caller-owned
 *             staging buffers, distinct).
 *  Other arguments as lsa_phiv (no stats).  Returns lsa_phiv's status, or
 *  LSA_ERR_CUDA when a copy cannot be enqueued. */
lsa_status lsa_phiv_host(const lsa_op* op, const double* v_host, double h, int p, int m, double tol,
                         int variant, int precision, double* y_host, double* v_dev, double* y_dev,
                         void* work, size_t work_bytes, void* stream);

/* Measurement utility (not part of the paper's method): a kernel of
 * independent float64 fused multiply-add chains on every SM, `iters` FMAs per
 * chain, for the float64 roofline's denominator.  out: dev, 1 double (a
 * checksum that keeps the chains live).  Returns the FLOPs it executes (2 per
 * FMA) in *flops; time it with events on `stream`. */
lsa_status lsa_probe_fp64_fma(int iters, double* out, double* flops, void* stream);

/* Exponential-integrator building blocks (Sect. 4) besides the phi products.
 * lsa_rhs: f = F(u) for the Gray-Scott system whose Jacobian at a state is
 *   the LSA_OP_GRAYSCOTT2D operator: F(u, v) = [Du Lap u - u v^2 + F (1 - u);
 *   Dv Lap v + u v^2 - (F + k) v], periodic 5-point Laplacian with spacing dx.
 *   op: that operator's descriptor (its fields are not read).  u, f: dev,
 *   2*nx*ny doubles, species-major; must not overlap.  LSA_ERR_ARG for other
 *   operator kinds.
 * lsa_axpby: w = a x + b y over n doubles (dev); w may be x or y. */
lsa_status lsa_rhs(const lsa_op* op, const double* u, double* f, void* stream);
lsa_status lsa_axpby(long long n, double a, const double* x, double b, const double* y, double* w,
                     void* stream);

/* S5 alone: coefficients C (dev, (p+2) x m doubles, row k = phi_k(h H_m) e_1,
 * k = 0..p+1) from one exponential of the augmented (m+p+1)-sized matrix,
 * computed on the GPU.  H: dev, column-major with leading dimension ldh >= m. */
lsa_status lsa_expm_phi(const double* H, int ldh, int m, double h, int p, double* C,
                        void* work, size_t work_bytes, void* stream);

/* Size of the fixed device workspace used by lsa_phiv_noalloc (32 MiB). */
#define LSA_STATIC_WORKSPACE_BYTES (32u << 20)

/* lsa_phiv for callers that cannot allocate device memory -- plugins inside a
 * host application that owns the device memory through its own pool, and
 * latency-critical code that must not call cudaMalloc/cudaFree after start-up
 * (they can synchronise the device).  The paper has no counterpart: this is a
 * deployment convenience of this library.
 *  Arguments and results as lsa_phiv, without work/work_bytes: the workspace
 *  is a static device array of LSA_STATIC_WORKSPACE_BYTES inside the library,
 *  held by every GPU that loads the library until the process exits.
 *  Returns LSA_ERR_WORKSPACE when lsa_workspace_bytes(op, min(m, N), p,
 *  precision) exceeds that size (nothing is launched then).
 *  The first call on a device looks up the array's device address
 *  (cudaGetSymbolAddress, with that device current); make that first call
 *  before any stream capture.  All calls share the one array and it keeps the
 *  last call's contents (each call re-initialises what must start at zero), so
 *  calls whose work overlaps on the GPU -- on different streams, or from
 *  different host threads -- race and must be serialised by the caller.
 *  The call allocates nothing (no cudaMalloc/cudaFree, no event creation);
 *  since it records no events, the stats it fills (when non-NULL) report
 *  ms_arnoldi, ms_expm, ms_combine, launches and arnoldi_kernel as 0 -- the
 *  status, m_eff, breakdown, fallback, sync and scalar fields are as lsa_phiv's.
 *  After cudaDeviceReset on a device, do not call it on that device again in
 *  the same process (the device address it cached belongs to the old context). */
lsa_status lsa_phiv_noalloc(const lsa_op* op, const double* v, double h, int p, int m, double tol,
                            int variant, int precision, double* y, lsa_stats* stats,
                            void* stream);

/* ---------------------------------------------------------------------------
 * Gradients of a loss L(y) of the phi_1 product y = phi_1(h A(theta)) v on the
 * Gray-Scott Jacobian (LSA_OP_GRAYSCOTT2D), theta = (diff, diff2, F, k), given
 * r = dL/dy -- the vector-Jacobian product behind an autograd function:
 *   dL/dv     = phi_1(h A^T) r                       (phi_1(hA)^T = phi_1(hA^T), Eq. 6)
 *   dL/dh     = r . (phi_0(hA)v - phi_1(hA)v) / h    (d/dh [h phi_1(hA)] = e^{hA})
 *   dL/dtheta = r . [phi_1(hK)[0; v]]_top, K = [[A, dA/dtheta], [0, A]]
 *               (LSA_OP_GRAYSCOTT2D_FRECHET: the block-triangular augmentation of
 *               the Frechet derivative of exp applied to Sect. 2.1's Eq. 7 matrix)
 *               for theta = diff, diff2, k;
 *   dL/dF     = -h r . (phi_1(hA)v - phi_2(hA)v)    (dA/dF = -I commutes with A;
 *               phi_1' = phi_1 - phi_2 follows from Eq. 6).
 * Four phi products with m Krylov steps each, all float64: one on A^T (N) and
 * three on K (2N); no Krylov basis is kept between calls (each is rebuilt).
 *  op        LSA_OP_GRAYSCOTT2D descriptor of A(theta) (aux ignored).
 *  v, r      dev, N doubles.    y  dev, 3 x N doubles: phi_0(hA)v, phi_1(hA)v,
 *            phi_2(hA)v (lsa_phiv with p = 2 and the same h, m and variant; p
 *            only enlarges the small exponential, not the Arnoldi process).
 *  h         finite and nonzero.   m, variant as lsa_phiv.
 *  grad_v    dev, N doubles (output).
 *  grad_s    dev, 5 doubles (output): dL/dh, dL/ddiff, dL/ddiff2, dL/dF, dL/dk.
 *  work      dev workspace of lsa_phiv_vjp_workspace_bytes(op, m), 256-byte aligned.
 * stats as lsa_phiv (when non-NULL: the calls synchronise, the worst status of
 * the four products is returned and their counters are summed). */
size_t lsa_phiv_vjp_workspace_bytes(const lsa_op* op, int m);
lsa_status lsa_phiv_vjp(const lsa_op* op, const double* v, double h, int m, int variant,
                        const double* r, const double* y, double* grad_v, double* grad_s,
                        void* work, size_t work_bytes, lsa_stats* stats, void* stream);

/* ---------------------------------------------------------------------------
 * Batched form: many independent phi products of one operator family (uneven
 * grid sizes N_i and Krylov dimensions m_i) in one persistent launch.  Each
 * instance is the computation of lsa_phiv; an exponential integrator needs
 * one such Arnoldi projection per sub-step (Sect. 2.2, Eqs. 14-15), and many
 * small ones do not fill the GPU one at a time.
 *
 * Packing: v holds v_0, v_1, ... back to back (instance i at element offset
 * sum_{l<i} N_l); y holds the (p+1) x N_i outputs back to back (instance i at
 * sum_{l<i} (p+1) N_l, row k at +k*N_i).  lsa_batch_info returns the offsets.
 * All instances share h, p, tol, variant and precision; m_i is capped at N_i.
 * Operator fields (field0/field1) must stay valid for the plan's lifetime.
 *
 * Tiling: the group_size CTAs of a group run one instance together (every
 * barrier counted over the group); the nlarge costliest instances go to
 * groups, the rest to single CTAs, each queue taken in order of decreasing
 * cost.  group_size = lsa_batch_info's ctas with nlarge = count is one grid
 * per instance; nlarge = 0 is one CTA per instance.  lsa_batch_tune times a
 * set of tilings on the caller's data and keeps the fastest, then (hybrid
 * variants) the other step form on that tiling, and keeps the faster. */
typedef struct lsa_batch lsa_batch;

/* Device workspace bytes for a batch (0 if the arguments are invalid).
 * ops, m: host arrays of `count` entries. */
size_t lsa_batch_workspace_bytes(const lsa_op* ops, const int* m, int count, int p, int precision);

/* Build a plan over a caller-provided workspace (256-byte aligned, at least
 * lsa_batch_workspace_bytes).  Copies the instance table to the workspace
 * (synchronising `stream`).  The plan owns host memory only; the workspace
 * stays the caller's and must outlive the plan. */
lsa_status lsa_batch_create(const lsa_op* ops, const int* m, int count, double h, int p,
                            double tol, int variant, int precision, void* work, size_t work_bytes,
                            lsa_batch** plan, void* stream);

/* Plan facts: CTAs of the persistent launch, current tiling, packed sizes and
 * (optional, `count` entries each) per-instance element offsets into v and y. */
lsa_status lsa_batch_info(const lsa_batch* plan, int* ctas, int* group_size, int* nlarge,
                          long long* v_elems, long long* y_elems, long long* voff, long long* yoff);

/* Set the tiling: 1 <= group_size <= ctas, 0 <= nlarge <= count. */
lsa_status lsa_batch_set_tiling(lsa_batch* plan, int group_size, int nlarge);

/* Step form of the hybrid variants in this plan (see lsa_tune_step): 0 the
 * one-pass step, 1 the two-phase step (the default for the hybrid variants;
 * its extra barrier is counted over an instance's group).  Both compute
 * bitwise the same result.
 * lsa_batch_step_form returns the plan's form (-1 for a null plan). */
lsa_status lsa_batch_set_step_form(lsa_batch* plan, int two_phase);
int lsa_batch_step_form(const lsa_batch* plan);

/* Enqueue one batched evaluation on `stream` (two kernels: initialisation and
 * the persistent kernel; nothing is read back).  use_graph != 0 captures the
 * two launches once into a CUDA graph (on a private stream of the plan) and
 * replays that graph on `stream`; the graph is rebuilt when v, y or the tiling
 * change.  Per-instance results: lsa_batch_read_stats. */
lsa_status lsa_batch_run(lsa_batch* plan, const double* v, double* y, int use_graph, void* stream);

/* Synchronise `stream` and read the per-instance statistics of the last run
 * into stats[0..count) (may be NULL) and the number of completed instances.
 * Returns the first error of any instance (an instance that did not complete
 * reports LSA_ERR_TIMEOUT), else the largest warning, else LSA_OK. */
lsa_status lsa_batch_read_stats(const lsa_batch* plan, lsa_stats* stats, int* finished, void* stream);

/* Time candidate tilings (one CTA per instance, one grid per instance, and
 * groups of 2..32 CTAs for the costliest count/64 .. count instances), each
 * `reps` times after one warm-up run on the caller's v and y, keep the fastest
 * and return it (with, for the hybrid variants, the faster step form on it,
 * see lsa_batch_step_form).  Synchronises `stream`; overwrites y. */
lsa_status lsa_batch_tune(lsa_batch* plan, const double* v, double* y, int reps, int* group_size,
                          int* nlarge, float* ms_best, void* stream);

/* Release the plan's host memory and its graph (not the workspace). */
void lsa_batch_destroy(lsa_batch* plan);

/* One-shot batched call: create a plan with the default tiling, run it without
 * a graph, read the statistics (stats: `count` entries or NULL), destroy it. */
lsa_status lsa_phiv_batched(const lsa_op* ops, const int* m, int count, const double* v, double h,
                            int p, double tol, int variant, int precision, double* y, void* work,
                            size_t work_bytes, lsa_stats* stats, void* stream);

/* Synchronise `stream` and read the statistics of the last call that used `work`. */
lsa_status lsa_read_stats(const void* work, lsa_stats* out, void* stream);

/* Failure-detection self-test: launches a two-block kernel whose grid barrier
 * waits on a flag that nothing sets, with a wait limit of `seconds` (> 0,
 * <= 10).  Expected result: LSA_ERR_TIMEOUT, with the CUDA context still usable. */
lsa_status lsa_selftest_barrier_timeout(void* work, size_t work_bytes, double seconds, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LSARNOLDI_H */
