// Matrix-free stencil operators (S1), applied to a tile held in shared memory.
//
// Each operator reads one grid point and its face neighbours from the
// shared-memory planes of the projected vector (a TX x TY footprint plus a
// one-point halo, row pitch RP, PW by default) and returns A x at that point for every
// species.  The paper only needs the action v -> J v (Sect. 2.1); the three
// operators are the synthetic stand-ins of the benchmark workloads.
#pragma once

#include "lsa_internal.cuh"

namespace lsa {

template <class Tc>
struct Coef {
  Tc cW, cE, cS, cN, cD, cU, cC, du, dv, F, k, idx2;
  int dir;
  __device__ void load(const DevOp& d) {
    cW = (Tc)d.cW; cE = (Tc)d.cE; cS = (Tc)d.cS; cN = (Tc)d.cN;
    cD = (Tc)d.cD; cU = (Tc)d.cU; cC = (Tc)d.cC;
    du = (Tc)d.du; dv = (Tc)d.dv; F = (Tc)d.F; k = (Tc)d.k; idx2 = (Tc)d.idx2;
    dir = d.dir;
  }
};

// 2D periodic advection-diffusion: A v = c Lap5 v - u.grad v (central).
struct OpAdvDiff2D {
  static constexpr int NS = 1, DIM = 2, KIND = LSA_OP_ADVDIFF2D, NF = 0;
  template <class Tc, int RP = PW, int SP = PS>
  __device__ __forceinline__ static void apply_f(const Coef<Tc>& c, const Tc* zm, const Tc* z0,
                                                 const Tc* zp, int o, Tc, Tc, Tc* out) {
    (void)zm; (void)zp;
    Tc x = z0[o];
    Tc r = c.cC * x;
    r = fma(c.cW, z0[o - 1], r);
    r = fma(c.cE, z0[o + 1], r);
    r = fma(c.cS, z0[o - RP], r);
    r = fma(c.cN, z0[o + RP], r);
    out[0] = r;
  }
  template <class Tc, int RP = PW, int SP = PS>
  __device__ __forceinline__ static void apply(const DevOp&, const Coef<Tc>& c, const Tc* zm,
                                               const Tc* z0, const Tc* zp, int o, long long,
                                               Tc* out) {
    apply_f<Tc, RP, SP>(c, zm, z0, zp, o, (Tc)0, (Tc)0, out);
  }
};

// Jacobian of 2D Gray-Scott at (u0, v0), species-major [u; v].  Field values:
// (u0, v0) in the float64 form, the float copies (a, b) = (v0^2, 2 u0 v0) in the
// float32 form.
struct OpGrayScott2D {
  static constexpr int NS = 2, DIM = 2, KIND = LSA_OP_GRAYSCOTT2D, NF = 2;
  // RP: row pitch of the staged values; SP: offset of the second species
  template <class Tc, int RP = PW, int SP = PS>
  __device__ __forceinline__ static void apply_f(const Coef<Tc>& c, const Tc* zm, const Tc* z0,
                                                 const Tc* zp, int o, Tc f0, Tc f1, Tc* out) {
    (void)zm; (void)zp;
    Tc a, b;
    if constexpr (sizeof(Tc) == 8) { a = f1 * f1; b = (Tc)2 * f0 * f1; }
    else { a = f0; b = f1; }
    const Tc* U = z0;
    const Tc* Vv = z0 + SP;
    Tc u = U[o], v = Vv[o];
    Tc lu = (U[o - 1] + U[o + 1]) + (U[o - RP] + U[o + RP]) - (Tc)4 * u;
    Tc lv = (Vv[o - 1] + Vv[o + 1]) + (Vv[o - RP] + Vv[o + RP]) - (Tc)4 * v;
    out[0] = c.du * lu - (a + c.F) * u - b * v;
    out[1] = c.dv * lv + (b - c.F - c.k) * v + a * u;
  }
  template <class Tc, int RP = PW, int SP = PS>
  __device__ __forceinline__ static void apply(const DevOp& d, const Coef<Tc>& c, const Tc* zm,
                                               const Tc* z0, const Tc* zp, int o, long long gpt,
                                               Tc* out) {
    Tc f0, f1;
    if constexpr (sizeof(Tc) == 8) { f0 = __ldg(d.f0 + gpt); f1 = __ldg(d.f1 + gpt); }
    else { f0 = __ldg(d.g0 + gpt); f1 = __ldg(d.g1 + gpt); }
    apply_f<Tc, RP, SP>(c, zm, z0, zp, o, f0, f1, out);
  }
};

// Transpose of the Gray-Scott Jacobian (float64 form only): the coupling
// blocks swap, [[A11, A21], [A12, A22]] with A12 = -diag(2 u0 v0), A21 =
// diag(v0^2); the Laplacian is symmetric.  Used for the gradient with respect
// to v of a loss on phi_1(hA) v (phi_1(hA)^T = phi_1(hA^T)).
struct OpGrayScott2DT {
  static constexpr int NS = 2, DIM = 2, KIND = LSA_OP_GRAYSCOTT2D_T, NF = 2;
  template <class Tc, int RP = PW>
  __device__ __forceinline__ static void apply_f(const Coef<Tc>& c, const Tc* zm, const Tc* z0,
                                                 const Tc* zp, int o, Tc f0, Tc f1, Tc* out) {
    (void)zm; (void)zp;
    const Tc a = f1 * f1, b = (Tc)2 * f0 * f1;
    const Tc* U = z0;
    const Tc* Vv = z0 + PS;
    Tc u = U[o], v = Vv[o];
    Tc lu = (U[o - 1] + U[o + 1]) + (U[o - RP] + U[o + RP]) - (Tc)4 * u;
    Tc lv = (Vv[o - 1] + Vv[o + 1]) + (Vv[o - RP] + Vv[o + RP]) - (Tc)4 * v;
    out[0] = c.du * lu - (a + c.F) * u + a * v;
    out[1] = c.dv * lv + (b - c.F - c.k) * v - b * u;
  }
  template <class Tc>
  __device__ __forceinline__ static void apply(const DevOp& d, const Coef<Tc>& c, const Tc* zm,
                                               const Tc* z0, const Tc* zp, int o, long long gpt,
                                               Tc* out) {
    apply_f<Tc>(c, zm, z0, zp, o, (Tc)__ldg(d.f0 + gpt), (Tc)__ldg(d.f1 + gpt), out);
  }
};

// Block operator K = [[A, dA/dtheta], [0, A]] of the Gray-Scott Jacobian A on
// [a; b] = [a_u, a_v, b_u, b_v] (four species blocks; float64 form only),
// theta = (Du, Dv, F, k)[dir]: dA/dDu = [[Lap, 0], [0, 0]], dA/dDv =
// [[0, 0], [0, Lap]], dA/dF = -I, dA/dk = [[0, 0], [0, -I]] (Lap the
// periodic five-point Laplacian / dx^2).  The top half of phi_1(hK)[0; v] is
// the derivative of phi_1(hA)v along h dA/dtheta (block-triangular augmentation
// of the Frechet derivative of exp, applied to Sect. 2.1's Eq. 7 matrix).
struct OpGrayScottFrechet2D {
  static constexpr int NS = 4, DIM = 2, KIND = LSA_OP_GRAYSCOTT2D_FRECHET, NF = 2;
  template <class Tc, int RP = PW>
  __device__ __forceinline__ static void apply_f(const Coef<Tc>& c, const Tc* zm, const Tc* z0,
                                                 const Tc* zp, int o, Tc f0, Tc f1, Tc* out) {
    (void)zm; (void)zp;
    const Tc a = f1 * f1, b = (Tc)2 * f0 * f1;
    Tc x[4], l[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const Tc* P = z0 + s * PS;
      x[s] = P[o];
      l[s] = (P[o - 1] + P[o + 1]) + (P[o - RP] + P[o + RP]) - (Tc)4 * x[s];
    }
    // A on the a-block and on the b-block
    out[0] = c.du * l[0] - (a + c.F) * x[0] - b * x[1];
    out[1] = c.dv * l[1] + (b - c.F - c.k) * x[1] + a * x[0];
    out[2] = c.du * l[2] - (a + c.F) * x[2] - b * x[3];
    out[3] = c.dv * l[3] + (b - c.F - c.k) * x[3] + a * x[2];
    // + dA/dtheta on the b-block, into the a-block
    if (c.dir == 0) out[0] += c.idx2 * l[2];
    else if (c.dir == 1) out[1] += c.idx2 * l[3];
    else if (c.dir == 2) { out[0] -= x[2]; out[1] -= x[3]; }
    else out[1] -= x[3];
  }
  template <class Tc>
  __device__ __forceinline__ static void apply(const DevOp& d, const Coef<Tc>& c, const Tc* zm,
                                               const Tc* z0, const Tc* zp, int o, long long gpt,
                                               Tc* out) {
    apply_f<Tc>(c, zm, z0, zp, o, (Tc)__ldg(d.f0 + gpt), (Tc)__ldg(d.f1 + gpt), out);
  }
};

// 3D periodic advection-diffusion-reaction with first-order upwinding.
struct OpADR3D {
  static constexpr int NS = 1, DIM = 3, KIND = LSA_OP_ADR3D, NF = 1;
  template <class Tc, int RP = PW, int SP = PS>
  __device__ __forceinline__ static void apply_f(const Coef<Tc>& c, const Tc* zm, const Tc* z0,
                                                 const Tc* zp, int o, Tc rr, Tc, Tc* out) {
    Tc x = z0[o];
    Tc r = (c.cC + rr) * x;
    r = fma(c.cW, z0[o - 1], r);
    r = fma(c.cE, z0[o + 1], r);
    r = fma(c.cS, z0[o - RP], r);
    r = fma(c.cN, z0[o + RP], r);
    r = fma(c.cD, zm[o], r);
    r = fma(c.cU, zp[o], r);
    out[0] = r;
  }
  template <class Tc, int RP = PW, int SP = PS>
  __device__ __forceinline__ static void apply(const DevOp& d, const Coef<Tc>& c, const Tc* zm,
                                               const Tc* z0, const Tc* zp, int o, long long gpt,
                                               Tc* out) {
    Tc rr;
    if constexpr (sizeof(Tc) == 8) rr = __ldg(d.f0 + gpt);
    else rr = __ldg(d.g0 + gpt);
    apply_f<Tc, RP, SP>(c, zm, z0, zp, o, rr, (Tc)0, out);
  }
};

}  // namespace lsa
