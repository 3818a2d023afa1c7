// Batched phi products: many independent instances (uneven grid sizes and
// Krylov dimensions) in one persistent cooperative launch.
//
// Two work queues, both ordered by decreasing cost (N_i times the streamed
// columns of m_i Arnoldi steps):
//   * the "group" queue holds the nlarge costliest instances; the grid is cut
//     into groups of gsize CTAs and each group takes the next instance, runs
//     it with every barrier counted over the group, and comes back;
//   * the "single" queue holds the rest; one CTA takes one instance (its
//     barriers have a count of one and never wait).
// A CTA serves the group queue while that has work, then the single queue,
// so the cheap instances fill the tail left by the expensive ones.
// gsize = grid with nlarge = count is "the whole grid per instance" and
// nlarge = 0 is "one CTA per instance"; the host-side tuner picks in between,
// and the step form of the hybrid variants (one-pass or two-phase, whose
// barrier between its passes is counted over the group).
#pragma once

#include "lsa_engine.cuh"
#include "lsa_expm.cuh"

namespace lsa {

struct BatchInst {      // one instance, with its slice of the workspace
  DevOp op;
  Tiling tl;
  int m;
  int pad;
  long long voff;       // element offset of v_i in the packed input
  long long yoff;       // element offset of y_i in the packed output ((p+1) N_i values)
  Ctl* ctl;
  double* H;            // (m+1) x m
  double* C;            // (PMAX+2) x (MMAX+2) coefficients
  void* V;              // N x (m+3): basis, then the two matvec buffers
};

struct BatchMail {      // group-queue claim of one group, published by its first CTA
  unsigned gen;
  int idx;
  int dead;             // a member left after a failed barrier: the group stops
  int pad;
};

struct BatchCtl {
  unsigned head[2];     // next position in the group and single queues
  int status;           // LSA_ERR_TIMEOUT when a queue hand-off gave up
  int abort_flag;
  unsigned finished;    // instances completed
  int pad[3];
};

// Per-worker scratch: a worker is a group (indexed by its first CTA) or a
// single CTA (its own index).  Workers that run at the same time never share
// an index.
struct BatchScratch {
  double* partials;     // G x SLOTS
  double* T;            // G x MMAX^2
  double* L;            // G x MMAX^2
  double* mats;         // G x 6 SMALL_STRIDE^2
};

struct BatchParams {
  const BatchInst* inst;
  const int* order;        // group queue (nlarge entries) then single queue
  int count, nlarge, gsize;
  int two_phase;           // hybrid variants: the two-phase step (see ArnoldiParams)
  int variant, p;
  double h, tol, brk_tol;
  long long timeout_ns;
  BatchCtl* bctl;
  BatchMail* mail;         // one per group
  BatchScratch ws;
  const double* v;         // packed inputs
  double* y;               // packed outputs
};

constexpr size_t kMatsPerWorker = (size_t)6 * SMALL_STRIDE * SMALL_STRIDE;

// One instance, run by a worker of gsize CTAs (this CTA has rank grank; the
// worker's scratch index is wbase).  Returns false when a barrier of the
// instance gave up (the caller leaves the kernel).
template <class Op, class Tc>
__device__ __noinline__ bool batch_instance(const BatchParams& BP, const BatchInst& I, int grank,
                                               int gsize, int wbase,
                                               typename Engine<Op, Tc, Tc>::Smem& S, double* small,
                                               ExpmShared& esh, ArnoldiParams& P, SmallParams& SP) {
  using E = Engine<Op, Tc, Tc>;
  // the parameters live in shared memory (written by one thread): the engine
  // reads them all through, as the standalone kernel reads its parameter bank
  if (threadIdx.x == 0) {
    P.op = I.op;
    P.tl = I.tl;
    P.vin = BP.v + I.voff;
    P.V = I.V;
    const size_t bs = sizeof(Tc);
    P.W0 = reinterpret_cast<unsigned char*>(I.V) + (size_t)I.op.N * (I.m + 1) * bs;
    P.W1 = reinterpret_cast<unsigned char*>(I.V) + (size_t)I.op.N * (I.m + 2) * bs;
    P.H = I.H;
    P.ctl = I.ctl;
    P.partials = BP.ws.partials + (size_t)wbase * SLOTS;
    P.gsum = nullptr;
    P.naug = 0;
    P.T = BP.ws.T + (size_t)wbase * MMAX * MMAX;
    P.L = BP.ws.L + (size_t)wbase * MMAX * MMAX;
    P.m = I.m;
    P.variant = BP.variant;
    P.write_vlast = 0;
    P.two_phase = BP.two_phase;
    P.brk_tol = BP.brk_tol;
    P.timeout_ns = BP.timeout_ns;
    SP.H = I.H;
    SP.ldh = I.m + 1;
    SP.ctl_in = I.ctl;
    SP.ctl = I.ctl;
    SP.m = I.m;
    SP.p = BP.p;
    SP.h = BP.h;
    SP.mats = BP.ws.mats + (size_t)wbase * kMatsPerWorker;
    SP.C = I.C;
    SP.ldc = MMAX + 2;
    SP.scale_out = 1;
    SP.timeout_ns = BP.timeout_ns;
    SP.tol = BP.tol;
  }
  __syncthreads();
  {
    E e(P, S, small);
    e.grank = grank;
    e.gsize = gsize;
    if (P.variant == LSA_MGS) e.run_mgs(false);
    else if (P.variant == LSA_CGS2) e.run_cgs2(false);
    else if (P.variant == LSA_IOCGS) e.run_iocgs(false);
    else e.run_hybrid();
  }
  __syncthreads();
  if (ld_volatile_i32(&I.ctl->abort_flag)) return false;
  if (!expm_group(SP, grank, gsize, esh)) return false;
  __syncthreads();
  if (BP.p <= 3)
    combine_group<Tc, 3>(reinterpret_cast<const Tc*>(I.V), I.op.N, I.C, MMAX + 2, BP.p, I.ctl,
                         BP.y + I.yoff, grank, gsize);
  else
    combine_group<Tc, PMAX>(reinterpret_cast<const Tc*>(I.V), I.op.N, I.C, MMAX + 2, BP.p, I.ctl,
                            BP.y + I.yoff, grank, gsize);
  __syncthreads();
  if (grank == 0 && threadIdx.x == 0) {
    I.ctl->finished = 1;
    atomicAdd(&BP.bctl->finished, 1u);
  }
  return true;
}

template <class Op, class Tc>
__global__ void __launch_bounds__(NT, 2) k_batched(BatchParams BP) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ ExpmShared esh;
  __shared__ ArnoldiParams sP;
  __shared__ SmallParams sSP;
  __shared__ int s_idx;
  using E = Engine<Op, Tc, Tc>;
  typename E::Smem& S = *reinterpret_cast<typename E::Smem*>(smem_raw);
  double* small = reinterpret_cast<double*>(smem_raw + E::small_offset());
  const int b = blockIdx.x;
  const int gs = BP.gsize;
  const int ngroups = (BP.nlarge > 0 && gs >= 1) ? (int)gridDim.x / gs : 0;

  // group phase
  if (b < ngroups * gs) {
    const int group = b / gs, grank = b - group * gs, base = group * gs;
    BatchMail* mb = BP.mail + group;
    for (unsigned k = 0;; ++k) {
      if (threadIdx.x == 0) {
        int idx;
        if (grank == 0) {
          idx = (int)atomicAdd(&BP.bctl->head[0], 1u);
          *(volatile int*)&mb->idx = idx;
          st_release_u32(&mb->gen, k + 1u);
        } else {
          idx = -1;
          const unsigned long long t0 = global_ns();
          unsigned it = 0;
          for (;;) {
            if (ld_acquire_u32(&mb->gen) >= k + 1u) { idx = *(volatile int*)&mb->idx; break; }
            if ((++it & 255u) == 0u) {
              if (ld_volatile_i32(&mb->dead) || ld_volatile_i32(&BP.bctl->abort_flag)) break;
              if ((long long)(global_ns() - t0) > BP.timeout_ns) {
                atomicExch(&BP.bctl->abort_flag, 1);
                atomicCAS(&BP.bctl->status, 0, (int)LSA_ERR_TIMEOUT);
                break;
              }
              if (it > 4096u) __nanosleep(64);
            }
          }
        }
        s_idx = idx;
      }
      __syncthreads();
      const int idx = s_idx;
      __syncthreads();
      if (idx < 0) return;
      if (idx >= BP.nlarge) break;
      const BatchInst& I = BP.inst[BP.order[idx]];
      if (!batch_instance<Op, Tc>(BP, I, grank, gs, base, S, small, esh, sP, sSP)) {
        if (threadIdx.x == 0) atomicExch(&mb->dead, 1);
        return;
      }
    }
  }
  // single phase
  const int nsingle = BP.count - BP.nlarge;
  for (;;) {
    if (threadIdx.x == 0) s_idx = (int)atomicAdd(&BP.bctl->head[1], 1u);
    __syncthreads();
    const int idx = s_idx;
    __syncthreads();
    if (idx >= nsingle) break;
    const BatchInst& I = BP.inst[BP.order[BP.nlarge + idx]];
    if (!batch_instance<Op, Tc>(BP, I, 0, 1, b, S, small, esh, sP, sSP)) return;
  }
}

template <class Op, class Tc>
cudaError_t launch_batched_t(const BatchParams& BP, int G, cudaStream_t s) {
  auto k = k_batched<Op, Tc>;
  const size_t sm = Engine<Op, Tc, Tc>::smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  // cooperative launch (all CTAs co-resident: the group barriers and the
  // group-queue hand-off wait on one another), issued so that stream capture
  // records it as a cooperative kernel node
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, BP);
}

template <class Op>
cudaError_t launch_batched_op(const BatchParams& BP, int precision, int G, cudaStream_t s) {
  if (precision == LSA_FP64) return launch_batched_t<Op, double>(BP, G, s);
  return launch_batched_t<Op, float>(BP, G, s);
}

template <class Op>
int batched_blocks_per_sm_op(int precision) {
  int nb = 0;
  if (precision == LSA_FP64) {
    auto k = k_batched<Op, double>;
    const size_t sm = Engine<Op, double, double>::smem_bytes();
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, NT, sm);
  } else {
    auto k = k_batched<Op, float>;
    const size_t sm = Engine<Op, float, float>::smem_bytes();
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, NT, sm);
  }
  return nb;
}

}  // namespace lsa
