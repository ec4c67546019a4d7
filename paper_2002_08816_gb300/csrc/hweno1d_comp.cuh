// The 1D operator on increments, for the FP32 resident launch with float-pair
// cell averages (precision HWENO_FP32C; Zhao & Qiu, arXiv:2002.08816,
// Sec. 2.1, Eq. (odeH), Eq. (RK)).
//
// The right-hand side of the first moments is (F_i - (fhat_l + fhat_r)/2)/dx:
// O(|f|/dx) terms that cancel to O(|f'| |u_x|), and it reacts to a change of
// the averages with a factor 1/dx.  Rounding the averages to FP32 at every
// stage therefore moves the first moments of the 2000-step shocked workload
// by ~4e-3 relative L1 even with exact arithmetic (the study in
// tests/study_first_moment_rounding.py).  Here the averages are carried as
// float pairs hi + lo between stages, and every part of the operator that
// reaches the first moments is formed from increments over the cell's own hi:
//   * the stencil data of cell i are d_k = (hi_{i+k} - hi_i) + lo_{i+k} (the
//     difference of two FP32 values within a factor two of each other is
//     exact), and the interface and interior values are the linear p0 (or
//     HWENO) maps of these increments: each map's coefficients sum to one and
//     its smoothness indicators are differences, so p(hi_i + d) = hi_i + p(d);
//   * fluxes enter as increments f(hi_i + d) - f(hi_i) in closed forms whose
//     rounding errors are relative to the increment (flux_inc);
//   * an interface flux shared by cells i and i + 1 is carried relative to
//     the left cell's base and moved to the right cell's by the increment
//     f(hi_{i+1}) - f(hi_i), so f(hi_i) itself never forms: it cancels from
//     F_i - (fhat_l + fhat_r)/2 exactly and from fhat_r - fhat_l exactly;
//   * the Runge-Kutta combination of the averages runs in float-pair
//     arithmetic (error-free sums and products), with the alpha-dependent
//     increment added last.
// The KXRCF flags, the limiter of troubled cells, the eigen-systems and the
// wave speeds use hi (their results do not need more than FP32), and the first
// moments stay FP32.
#pragma once
#include "hweno1d_stage.cuh"

namespace hw {
namespace c1d {

using s1d::H;
using s1d::Smem1D;

// f(B + D) - f(B) for a base state B and an increment D, with rounding errors
// relative to the increment (no difference of O(|f|) terms).  Euler: with
// mu = m / rho, q = m mu, p = (gamma - 1)(E - q / 2),
//   dmu = (dm - mu drho) / (rho + drho),  dq = m dmu + dm (mu + dmu),
//   dp = (gamma - 1)(dE - dq / 2),
//   df = (dm, dq + dp, dmu (E + p + dE + dp) + mu (dE + dp)).
template <int C>
__device__ __forceinline__ void flux_inc(float gas, const float* B, const float* D, float* dF) {
  if constexpr (C == 1) {
    dF[0] = D[0] * (B[0] + 0.5f * D[0]);
  } else {
    const float rho = B[0], m = B[1], E = B[2];
    const float dr = D[0], dm = D[1], dE = D[2];
    const float mu = m * fast_rcp(rho);
    const float dmu = (dm - mu * dr) * fast_rcp(rho + dr);
    const float q = m * mu;
    const float dq = m * dmu + dm * (mu + dmu);
    const float g1 = gas - 1.0f;
    const float p = g1 * (E - 0.5f * q);
    const float dp = g1 * (dE - 0.5f * dq);
    dF[0] = dm;
    dF[1] = dq + dp;
    dF[2] = dmu * ((E + p) + (dE + dp)) + mu * (dE + dp);
  }
}

// KXRCF on float-pair averages (um + lm, u0 + l0, up + lp; FP32 first
// moments), in three tiers: the plain kernel's FP32 fast test on hi, whose
// margins (6e-7 S on the jump, 4.8e-7 on the threshold) exceed what the low
// parts can change (below 2^-24 of |u0| + |u_nb|); where it cannot decide (on
// fine grids, where the threshold h^(3/2) |u0| falls below the jump's rounding
// bound, that is most cells), the jump and the threshold as unevaluated float
// pairs with the low parts added in (jump_pair_lo: within ~2^-45 S of the
// exact jump of hi + lo; r = |u0 + l0| (hthr + hthr_lo) within ~2^-46 r),
// decided when their difference clears 1e-12 (S + r), far above those
// bounds; and only inside that margin the FP64 product form on hi + lo.  The
// decision is the oracle's on the same state except within a few FP64 ulp of
// the threshold (deciding on hi alone would flip the rare cell that hi's
// rounding moves across it).
__device__ __forceinline__ bool kxrcf_troubled_pair(float um, float lm, float u0, float l0,
                                                    float up, float lp, float vm, float v0,
                                                    float vp, bool left, double h, double thr,
                                                    float hthr, float hthr_lo) {
  float a, b, s;
  if (left) {
    a = u0 - 6.0f * v0;
    b = um + 6.0f * vm;
    s = fabsf(u0) + 6.0f * fabsf(v0) + fabsf(um) + 6.0f * fabsf(vm);
  } else {
    a = u0 + 6.0f * v0;
    b = up - 6.0f * vp;
    s = fabsf(u0) + 6.0f * fabsf(v0) + fabsf(up) + 6.0f * fabsf(vp);
  }
  const float j = fabsf(a - b);
  const float e = 6.0e-7f * s;
  const float r = hthr * fmaxf(fabsf(u0), 1e-12f);
  if (j - e > r * (1.0f + 4.8e-7f)) return true;
  if (j + e < r * (1.0f - 4.8e-7f)) return false;
  float jh, jl;
  jump_pair_lo(u0, l0, v0, left ? um : up, left ? lm : lp, left ? vm : vp, left, jh, jl);
  if (jh < 0.0f) {
    jh = -jh;
    jl = -jl;
  }
  // |u0 + l0| as a pair: a normalised pair's hi carries the sign
  float nh = fabsf(u0), nl = u0 < 0.0f ? -l0 : l0;
  if (nh < 1e-12f) {
    nh = 1e-12f;
    nl = 0.0f;
  }
  const float rh = __fmul_rn(nh, hthr);
  const float rl = __fadd_rn(fmaf(nh, hthr, -rh),
                             __fadd_rn(__fmul_rn(nh, hthr_lo), __fmul_rn(nl, hthr)));
  const float d = __fadd_rn(__fsub_rn(jh, rh), __fsub_rn(jl, rl));
  if (fabsf(d) > 1e-12f * (s + r)) return d > 0.0f;
  return kxrcf_troubled((double)um + (double)lm, (double)u0 + (double)l0,
                        (double)up + (double)lp, (double)vm, (double)v0, (double)vp, left, h,
                        thr, 0.0f, 0.0f);
}

// Step 2.1 of an Euler cell on increments: the HWENO values at x_{i-1/2} and
// x_{i+1/2} in the characteristic fields of the state (b0, b1, b2), of the
// stencil data given as increments (am*, a0*, ap* the averages', vm*, v0*,
// vp* the first moments); the results are increments too (the projections
// and the HWENO combination commute with adding a constant state).
__device__ __noinline__ s1d::ConsFaces<float> char_faces_inc(
    float gas, float g0, float g1, float g2, float eps, float b0, float b1, float b2, float am0,
    float am1, float am2, float a00, float a01, float a02, float ap0, float ap1, float ap2,
    float vm0, float vm1, float vm2, float v00, float v01, float v02, float vp0, float vp1,
    float vp2) {
  const float U[3] = {b0, b1, b2};
  const float gam[3] = {g0, g1, g2};
  float Rm[3][3], Lm[3][3];
  Euler1D<float>::eigen(gas, U, Rm, Lm);
  float cl[3], cr[3];
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    const float* l = Lm[f];
    hweno_faces(l[0] * am0 + l[1] * am1 + l[2] * am2, l[0] * a00 + l[1] * a01 + l[2] * a02,
                l[0] * ap0 + l[1] * ap1 + l[2] * ap2, l[0] * vm0 + l[1] * vm1 + l[2] * vm2,
                l[0] * v00 + l[1] * v01 + l[2] * v02, l[0] * vp0 + l[1] * vp1 + l[2] * vp2, gam,
                eps, cl[f], cr[f]);
  }
  s1d::ConsFaces<float> o;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    o.L[c] = Rm[c][0] * cl[0] + Rm[c][1] * cl[1] + Rm[c][2] * cl[2];
    o.Rt[c] = Rm[c][0] * cr[0] + Rm[c][1] * cr[1] + Rm[c][2] * cr[2];
    o.fL[c] = o.fR[c] = 0.0f;
  }
  return o;
}

// The increments d_{-1}, d_0, d_{+1} of the averages of the cells beside and
// at sm.u slot e over hi_e, component c (ulo: the low parts of the averages,
// same slots).
template <int C, int NTH>
__device__ __forceinline__ void data_inc(const Smem1D<float, C, NTH>& sm, const float (*ulo)[NTH],
                                         int c, int e, float& dm, float& d0, float& dp) {
  const float b = sm.u[c][0][e];
  dm = __fadd_rn(__fsub_rn(sm.u[c][0][e - 1], b), ulo[c][e - 1]);
  d0 = ulo[c][e];
  dp = __fadd_rn(__fsub_rn(sm.u[c][0][e + 1], b), ulo[c][e + 1]);
}

// Step 2 at the interfaces of the cell in slot e = k + 2 of sm.u, on
// increments: sm.fm / sm.fp the traces u^+_{i-1/2}, u^-_{i+1/2} minus hi_e,
// sm.ffm / sm.ffp their flux increments over f(hi_e), fb[c][k] = f(hi_{e+1}) -
// f(hi_e) (the base change across x_{i+1/2}).
template <int C, int NTH>
__device__ __forceinline__ void faces_of_cell_inc(Smem1D<float, C, NTH>& sm,
                                                  const float (*ulo)[NTH], float (*fb)[NTH],
                                                  int k, float gas, const float* gam, float eps,
                                                  int variant) {
  const int e = k + 2;  // sm.u index e; sm.vl / sm.fl index of cell e is e - 1
  const bool hw = sm.fl[k] | sm.fl[k + 1] | sm.fl[k + 2];
  float B[C], dM[C], d0[C], dP[C], L[C], Rt[C], fL[C], fR[C], Dh[C], fD[C];
#pragma unroll
  for (int c = 0; c < C; ++c) {
    B[c] = sm.u[c][0][e];
    data_inc(sm, ulo, c, e, dM[c], d0[c], dP[c]);
    Dh[c] = __fsub_rn(sm.u[c][0][e + 1], B[c]);
  }
  if (!hw) {
#pragma unroll
    for (int c = 0; c < C; ++c)
      linear_faces(dM[c], d0[c], dP[c], sm.vl[c][e - 2], sm.vl[c][e - 1], sm.vl[c][e], L[c],
                   Rt[c]);
  } else if constexpr (C == 1) {
    hweno_faces(dM[0], d0[0], dP[0], sm.vl[0][e - 2], sm.vl[0][e - 1], sm.vl[0][e], gam, eps,
                L[0], Rt[0]);
  } else {
    const bool mean = variant & HWENO_VARIANT_MEAN_EIGEN;
    for (int side = 0; side < (mean ? 2 : 1); ++side) {
      float E[3];
#pragma unroll
      for (int c = 0; c < 3; ++c)
        E[c] = !mean ? B[c]
               : side ? 0.5f * (B[c] + sm.u[c][0][e + 1])
                      : 0.5f * (sm.u[c][0][e - 1] + B[c]);
      const s1d::ConsFaces<float> o = char_faces_inc(
          gas, gam[0], gam[1], gam[2], eps, E[0], E[1], E[2], dM[0], dM[1], dM[2], d0[0], d0[1],
          d0[2], dP[0], dP[1], dP[2], sm.vl[0][e - 2], sm.vl[1][e - 2], sm.vl[2][e - 2],
          sm.vl[0][e - 1], sm.vl[1][e - 1], sm.vl[2][e - 1], sm.vl[0][e], sm.vl[1][e],
          sm.vl[2][e]);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        if (!mean || side == 0) L[c] = o.L[c];
        if (!mean || side == 1) Rt[c] = o.Rt[c];
      }
    }
  }
  flux_inc<C>(gas, B, L, fL);
  flux_inc<C>(gas, B, Rt, fR);
  flux_inc<C>(gas, B, Dh, fD);
#pragma unroll
  for (int c = 0; c < C; ++c) {
    sm.fm[c][k] = L[c];
    sm.fp[c][k] = Rt[c];
    sm.ffm[c][k] = fL[c];
    sm.ffp[c][k] = fR[c];
    fb[c][k] = fD[c];
  }
}

// Eq. (odeH) of the own cell of thread tid (sm.u slot e = tid + 3) on
// increments, split by its dependence on alpha as in s1d::rhs_parts_of_cell:
// the central parts of the Lax-Friedrichs fluxes relative to f(hi_e), the
// trace jumps from the increments and the differences of the neighbours' hi,
// F_i from the flux increments (its weights sum to one).
template <int C, int NTH>
__device__ __forceinline__ void rhs_parts_inc(const Smem1D<float, C, NTH>& sm,
                                              const float (*ulo)[NTH], const float (*fb)[NTH],
                                              int tid, float gas, float inv_dx, float* L0u,
                                              float* Du, float* L0v, float* Dv) {
  const int e = tid + H, k = tid + 1;  // sm.u slot; sm.fm/fp slot of the cell
  float B[C], gm[C], gp[C], f2[C], f3[C];
#pragma unroll
  for (int c = 0; c < C; ++c) {
    float dm, d0, dp;
    B[c] = sm.u[c][0][e];
    data_inc(sm, ulo, c, e, dm, d0, dp);
    linear_interior(dm, d0, dp, sm.vl[c][e - 2], sm.vl[c][e - 1], sm.vl[c][e], gm[c], gp[c]);
  }
  flux_inc<C>(gas, B, gm, f2);
  flux_inc<C>(gas, B, gp, f3);
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const float dhl = __fsub_rn(sm.u[c][0][e], sm.u[c][0][e - 1]);
    const float dhr = __fsub_rn(sm.u[c][0][e + 1], sm.u[c][0][e]);
    const float cl = 0.5f * ((sm.ffp[c][k - 1] - fb[c][k - 1]) + sm.ffm[c][k]);
    const float cr = 0.5f * (sm.ffp[c][k] + (sm.ffm[c][k + 1] + fb[c][k]));
    const float jl = sm.fm[c][k] - (sm.fp[c][k - 1] - dhl);
    const float jr = (sm.fm[c][k + 1] + dhr) - sm.fp[c][k];
    const float F = (1.0f / 12.0f) * (sm.ffm[c][k] + sm.ffp[c][k]) + (5.0f / 12.0f) * (f2[c] + f3[c]);
    L0u[c] = -(cr - cl) * inv_dx;
    Du[c] = -0.5f * (jr - jl) * inv_dx;
    L0v[c] = (F - 0.5f * (cl + cr)) * inv_dx;
    Dv[c] = -0.25f * (jl + jr) * inv_dx;
  }
}

}  // namespace c1d
}  // namespace hw
