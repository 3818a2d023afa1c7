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
  Tc cW, cE, cS, cN, cD, cU, cC, du, dv, F, k;
  __device__ void load(const DevOp& d) {
    cW = (Tc)d.cW; cE = (Tc)d.cE; cS = (Tc)d.cS; cN = (Tc)d.cN;
    cD = (Tc)d.cD; cU = (Tc)d.cU; cC = (Tc)d.cC;
    du = (Tc)d.du; dv = (Tc)d.dv; F = (Tc)d.F; k = (Tc)d.k;
  }
};

// 2D periodic advection-diffusion: A v = c Lap5 v - u.grad v (central).
struct OpAdvDiff2D {
  static constexpr int NS = 1, DIM = 2, KIND = LSA_OP_ADVDIFF2D, NF = 0;
  template <class Tc, int RP = PW>
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
  template <class Tc>
  __device__ __forceinline__ static void apply(const DevOp&, const Coef<Tc>& c, const Tc* zm,
                                               const Tc* z0, const Tc* zp, int o, long long,
                                               Tc* out) {
    apply_f<Tc>(c, zm, z0, zp, o, (Tc)0, (Tc)0, out);
  }
};

// Jacobian of 2D Gray-Scott at (u0, v0), species-major [u; v].  Field values:
// (u0, v0) in the float64 form, the float copies (a, b) = (v0^2, 2 u0 v0) in the
// float32 form.
struct OpGrayScott2D {
  static constexpr int NS = 2, DIM = 2, KIND = LSA_OP_GRAYSCOTT2D, NF = 2;
  template <class Tc, int RP = PW>
  __device__ __forceinline__ static void apply_f(const Coef<Tc>& c, const Tc* zm, const Tc* z0,
                                                 const Tc* zp, int o, Tc f0, Tc f1, Tc* out) {
    (void)zm; (void)zp;
    Tc a, b;
    if constexpr (sizeof(Tc) == 8) { a = f1 * f1; b = (Tc)2 * f0 * f1; }
    else { a = f0; b = f1; }
    const Tc* U = z0;
    const Tc* Vv = z0 + PS;
    Tc u = U[o], v = Vv[o];
    Tc lu = (U[o - 1] + U[o + 1]) + (U[o - RP] + U[o + RP]) - (Tc)4 * u;
    Tc lv = (Vv[o - 1] + Vv[o + 1]) + (Vv[o - RP] + Vv[o + RP]) - (Tc)4 * v;
    out[0] = c.du * lu - (a + c.F) * u - b * v;
    out[1] = c.dv * lv + (b - c.F - c.k) * v + a * u;
  }
  template <class Tc>
  __device__ __forceinline__ static void apply(const DevOp& d, const Coef<Tc>& c, const Tc* zm,
                                               const Tc* z0, const Tc* zp, int o, long long gpt,
                                               Tc* out) {
    Tc f0, f1;
    if constexpr (sizeof(Tc) == 8) { f0 = __ldg(d.f0 + gpt); f1 = __ldg(d.f1 + gpt); }
    else { f0 = __ldg(d.g0 + gpt); f1 = __ldg(d.g1 + gpt); }
    apply_f<Tc>(c, zm, z0, zp, o, f0, f1, out);
  }
};

// 3D periodic advection-diffusion-reaction with first-order upwinding.
struct OpADR3D {
  static constexpr int NS = 1, DIM = 3, KIND = LSA_OP_ADR3D, NF = 1;
  template <class Tc, int RP = PW>
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
  template <class Tc>
  __device__ __forceinline__ static void apply(const DevOp& d, const Coef<Tc>& c, const Tc* zm,
                                               const Tc* z0, const Tc* zp, int o, long long gpt,
                                               Tc* out) {
    Tc rr;
    if constexpr (sizeof(Tc) == 8) rr = __ldg(d.f0 + gpt);
    else rr = __ldg(d.g0 + gpt);
    apply_f<Tc>(c, zm, z0, zp, o, rr, (Tc)0, out);
  }
};

}  // namespace lsa
