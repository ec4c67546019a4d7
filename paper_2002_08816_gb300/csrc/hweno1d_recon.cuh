// 1D reconstruction arithmetic of the hybrid HWENO scheme (Zhao & Qiu,
// arXiv:2002.08816, Sec. 2.1), for one scalar field on the three cells
// I_{i-1}, I_i, I_{i+1} (m, 0, p below).  The coefficients are the paper's
// printed rationals:
//   Step 1     q0, q1, q2 and beta_0..2 of the first-moment modification; the
//              last square of beta_0 uses v-coefficients +6, -6 (the printed
//              +1, -1 does not follow from Eq. (GHYZ));
//   Step 2.1   p0, p1, p2 at x_{i+1/2} and beta_0..2; the values at x_{i-1/2}
//              of p1 and p2 are their mirror images about x_i (p1 at
//              x_{i-1/2}: u_m/6 + 5u_0/6 - 4v_0; p2: 5u_0/6 + u_p/6 - 8v_0);
//   Step 2.2   p0 at x_{i-+1/2};   Step 2.3 p0 at x_{i-+sqrt5/10}.
#pragma once

#include "hweno_device.cuh"

namespace hw {

// Nonlinear combination shared by Step 1 and Step 2.1:
//   tau = ((|b0-b1| + |b0-b2|)/2)^2                          Eq. (tao5)
//   wbar_n = gamma_n (1 + tau/(beta_n + eps)),  w_n = wbar_n / sum wbar
//   out = w0 (v0/gamma0 - gamma1/gamma0 v1 - gamma2/gamma0 v2) + w1 v1 + w2 v2
template <typename R>
struct Weights3 {
  R w0g, w1, w2, g1, g2;  // w0/gamma0, w1, w2, gamma1, gamma2
  __device__ __forceinline__ Weights3(const R* gam, R eps, R b0, R b1, R b2) {
    R s = R(0.5) * (fabs(b0 - b1) + fabs(b0 - b2));
    R tau = s * s;
    if constexpr (sizeof(R) == 4) {
      // FP32: approximate reciprocals (the weights need a few ulp, not IEEE
      // rounding), which shortens the dependent chain of a troubled cell
      const R a0 = gam[0] * (R(1) + tau * fast_rcp(b0 + eps));
      const R a1 = gam[1] * (R(1) + tau * fast_rcp(b1 + eps));
      const R a2 = gam[2] * (R(1) + tau * fast_rcp(b2 + eps));
      const R inv = fast_rcp(a0 + a1 + a2);
      w0g = a0 * inv * fast_rcp(gam[0]);
      w1 = a1 * inv;
      w2 = a2 * inv;
      g1 = gam[1];
      g2 = gam[2];
      return;
    }
    R a0 = gam[0] * (R(1) + tau / (b0 + eps));
    R a1 = gam[1] * (R(1) + tau / (b1 + eps));
    R a2 = gam[2] * (R(1) + tau / (b2 + eps));
    R inv = R(1) / (a0 + a1 + a2);
    w0g = a0 * inv / gam[0];
    w1 = a1 * inv;
    w2 = a2 * inv;
    g1 = gam[1];
    g2 = gam[2];
  }
  __device__ __forceinline__ R apply(R v0, R v1, R v2) const {
    return w0g * (v0 - g1 * v1 - g2 * v2) + w1 * v1 + w2 * v2;
  }
};

// Step 1: modified first moment of I_i from u_m, u_0, u_p, v_m, v_p.
template <typename R>
__device__ __forceinline__ R limit_first_moment(R um, R u0, R up, R vm, R vp, const R* gam,
                                                R eps) {
  const R q0 = R(5.0 / 76.0) * (up - um) - R(11.0 / 38.0) * (vm + vp);
  const R q1 = R(1.0 / 12.0) * (u0 - um);
  const R q2 = R(1.0 / 12.0) * (up - u0);
  const R t1 = R(29.0 / 38.0) * (um - up) + R(60.0 / 19.0) * (vm + vp);
  const R t2 = R(9.0 / 4.0) * (um + up) - R(9.0 / 2.0) * u0 + R(15.0 / 2.0) * (vm - vp);
  const R t3 = (um - up) + R(12) * (vm + vp);
  const R t4 = R(5.0 / 2.0) * (um + up) - R(5) * u0 + R(9) * (vm - vp);
  const R t5 = (um - R(2) * u0 + up) + R(6) * (vm - vp);
  const R b0 = t1 * t1 + t2 * t2 + R(3905.0 / 1444.0) * t3 * t3 + R(1.0 / 12.0) * t4 * t4 +
               R(109341.0 / 448.0) * t5 * t5;
  const R d1 = u0 - um, d2 = up - u0;
  Weights3<R> w(gam, eps, b0, d1 * d1, d2 * d2);
  return w.apply(q0, q1, q2);
}

// Step 2.2: linear p0 at x_{i-1/2} (left) and x_{i+1/2} (right).
template <typename R>
__device__ __forceinline__ void linear_faces(R um, R u0, R up, R vm, R v0, R vp, R& left,
                                             R& right) {
  left = R(8.0 / 27.0) * um + R(7.0 / 12.0) * u0 + R(13.0 / 108.0) * up + R(28.0 / 27.0) * vm -
         R(241.0 / 54.0) * v0 - R(25.0 / 54.0) * vp;
  right = R(13.0 / 108.0) * um + R(7.0 / 12.0) * u0 + R(8.0 / 27.0) * up + R(25.0 / 54.0) * vm +
          R(241.0 / 54.0) * v0 - R(28.0 / 27.0) * vp;
}

// Packed FP32 (two values per instruction, fma.rn.f32x2): a broadcast pair
// and a - b in one rounding.
__device__ __forceinline__ float2 bcast2(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __ffma2_rn(bcast2(-1.0f), b, a);
}

// linear_faces of two components at once (each argument a pair), the same
// terms in packed FP32.
__device__ __forceinline__ void linear_faces_x2(float2 um, float2 u0, float2 up, float2 vm,
                                                float2 v0, float2 vp, float2& left, float2& right) {
  auto k = [](double c) { return bcast2((float)c); };
  left = __ffma2_rn(k(-25.0 / 54.0), vp,
         __ffma2_rn(k(-241.0 / 54.0), v0,
         __ffma2_rn(k(28.0 / 27.0), vm,
         __ffma2_rn(k(13.0 / 108.0), up, __ffma2_rn(k(7.0 / 12.0), u0, __fmul2_rn(k(8.0 / 27.0), um))))));
  right = __ffma2_rn(k(-28.0 / 27.0), vp,
          __ffma2_rn(k(241.0 / 54.0), v0,
          __ffma2_rn(k(25.0 / 54.0), vm,
          __ffma2_rn(k(8.0 / 27.0), up, __ffma2_rn(k(7.0 / 12.0), u0, __fmul2_rn(k(13.0 / 108.0), um))))));
}

// Step 2.3: linear p0 at x_{i-sqrt5/10} (gm) and x_{i+sqrt5/10} (gp).
template <typename R>
__device__ __forceinline__ void linear_interior(R um, R u0, R up, R vm, R v0, R vp, R& gm,
                                                R& gp) {
  constexpr double r5 = 2.2360679774997896964;
  constexpr double a = 101.0 / 5400.0 * r5, b = 1.0 / 24.0;
  constexpr double c = 3.0 / 20.0, d = 841.0 / 13500.0 * r5, e = 10289.0 / 6750.0 * r5;
  gm = R(-(a + b)) * um + R(13.0 / 12.0) * u0 + R(a - b) * up - R(c + d) * vm - R(e) * v0 +
       R(c - d) * vp;
  gp = R(a - b) * um + R(13.0 / 12.0) * u0 - R(a + b) * up + R(d - c) * vm + R(e) * v0 +
       R(c + d) * vp;
}

// linear_interior of two components at once, in packed FP32.
__device__ __forceinline__ void linear_interior_x2(float2 um, float2 u0, float2 up, float2 vm,
                                                   float2 v0, float2 vp, float2& gm, float2& gp) {
  constexpr double r5 = 2.2360679774997896964;
  constexpr double a = 101.0 / 5400.0 * r5, b = 1.0 / 24.0;
  constexpr double c = 3.0 / 20.0, d = 841.0 / 13500.0 * r5, e = 10289.0 / 6750.0 * r5;
  auto k = [](double x) { return bcast2((float)x); };
  gm = __ffma2_rn(k(c - d), vp,
       __ffma2_rn(k(-e), v0,
       __ffma2_rn(k(-(c + d)), vm,
       __ffma2_rn(k(a - b), up, __ffma2_rn(k(13.0 / 12.0), u0, __fmul2_rn(k(-(a + b)), um))))));
  gp = __ffma2_rn(k(c + d), vp,
       __ffma2_rn(k(e), v0,
       __ffma2_rn(k(d - c), vm,
       __ffma2_rn(k(-(a + b)), up, __ffma2_rn(k(13.0 / 12.0), u0, __fmul2_rn(k(a - b), um))))));
}

// Step 2.1: HWENO values at x_{i-1/2} (left) and x_{i+1/2} (right); one set of
// nonlinear weights serves both points (same candidates, same beta on I_i).
template <typename R>
__device__ __forceinline__ void hweno_faces(R um, R u0, R up, R vm, R v0, R vp, const R* gam,
                                            R eps, R& left, R& right) {
  R p0l, p0r;
  linear_faces(um, u0, up, vm, v0, vp, p0l, p0r);
  const R p1r = R(1.0 / 6.0) * um + R(5.0 / 6.0) * u0 + R(8) * v0;
  const R p1l = R(1.0 / 6.0) * um + R(5.0 / 6.0) * u0 - R(4) * v0;
  const R p2r = R(5.0 / 6.0) * u0 + R(1.0 / 6.0) * up + R(4) * v0;
  const R p2l = R(5.0 / 6.0) * u0 + R(1.0 / 6.0) * up - R(8) * v0;
  const R dU = um - up, sV = vm + vp, cU = um - R(2) * u0 + up, dV = vm - vp;
  const R s1 = R(19.0 / 108.0) * dU + R(31.0 / 54.0) * sV - R(241.0 / 27.0) * v0;
  const R s2 = R(9.0 / 4.0) * cU + R(15.0 / 2.0) * dV;
  const R s3 = R(70.0 / 9.0) * dU + R(200.0 / 9.0) * sV + R(1280.0 / 9.0) * v0;
  const R s4 = R(5.0 / 2.0) * cU + R(9) * dV;
  const R s5 = R(175.0 / 18.0) * dU + R(277.0 / 9.0) * sV + R(1546.0 / 9.0) * v0;
  const R s6 = R(95.0 / 18.0) * dU + R(155.0 / 9.0) * sV + R(830.0 / 9.0) * v0;
  const R s7 = R(5.0 / 8.0) * cU + R(15.0 / 4.0) * dV;
  const R s8 = R(35.0 / 36.0) * dU + R(77.0 / 18.0) * sV + R(133.0 / 9.0) * v0;
  const R b0 = s1 * s1 + s2 * s2 + s3 * s3 + R(1.0 / 12.0) * (s4 * s4 + s5 * s5) +
               R(1.0 / 180.0) * s6 * s6 + R(109341.0 / 175.0) * s7 * s7 +
               R(27553933.0 / 1764.0) * s8 * s8;
  const R v2 = R(144) * v0 * v0;
  const R e1 = um - u0 + R(12) * v0, e2 = u0 - up + R(12) * v0;
  const R b1 = v2 + R(13.0 / 3.0) * e1 * e1;
  const R b2 = v2 + R(13.0 / 3.0) * e2 * e2;
  Weights3<R> w(gam, eps, b0, b1, b2);
  left = w.apply(p0l, p1l, p2l);
  right = w.apply(p0r, p1r, p2r);
}

// KXRCF decision (reading of Sec. 2.1 Step 1 and Remark 1: Krivodonova et
// al. with the degree-1 cell polynomial ubar + 12 vbar (x - x_i)/dx, h = dx/2,
// the inflow face chosen by the sign of the velocity, normalised by
// max(|ubar_i|, 1e-12)): troubled iff |jump| / (h max(|u0|, 1e-12)) > thr.
// The FP64 form is evaluated without contraction, as the product form
// |jump| > thr h max(|u0|, 1e-12).
__device__ __forceinline__ bool kxrcf_troubled(double um, double u0, double up, double vm,
                                               double v0, double vp, bool left, double h,
                                               double thr, float /*hthr*/, float /*hthr_lo*/) {
  double jump;
  if (left)
    jump = __dsub_rn(__dsub_rn(u0, __dmul_rn(6.0, v0)), __dadd_rn(um, __dmul_rn(6.0, vm)));
  else
    jump = __dsub_rn(__dadd_rn(u0, __dmul_rn(6.0, v0)), __dsub_rn(up, __dmul_rn(6.0, vp)));
  // |jump| / (h nrm) > thr without the divide (FP64 divides occupy the FP64
  // pipe for many cycles): the decision differs from the quotient form only
  // within a few ulp of the threshold
  const double nrm = fmax(fabs(u0), 1e-12);
  return fabs(jump) > __dmul_rn(thr, __dmul_rn(h, nrm));
}

// s + e = a + b exactly (Knuth's two-sum); the intrinsics keep the compiler
// from contracting or reordering the steps.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// a (ah + al) + b (bh + bl) for float pairs, as a normalised pair (s + e, |e|
// <= ulp(s) / 2): error-free products (fma) and sums, the small terms rounded
// once; relative error ~2^-45.
__device__ __forceinline__ void pair_axpby(float ah, float al, float xh, float xl, float bh,
                                           float bl, float yh, float yl, float& s, float& e) {
  const float p = __fmul_rn(ah, xh), pe = fmaf(ah, xh, -p);
  const float q = __fmul_rn(bh, yh), qe = fmaf(bh, yh, -q);
  float t, te;
  two_sum(p, q, t, te);
  const float small = __fadd_rn(
      __fadd_rn(__fadd_rn(te, pe), qe),
      __fadd_rn(__fadd_rn(__fmul_rn(ah, xl), __fmul_rn(al, xh)),
                __fadd_rn(__fmul_rn(bh, yl), __fmul_rn(bl, yh))));
  two_sum(t, small, s, e);
}

// (h + l) + x as a normalised pair (x small next to h)
__device__ __forceinline__ void pair_add(float h, float l, float x, float& s, float& e) {
  two_sum(h, __fadd_rn(l, x), s, e);
}

// The KXRCF jump (u0 -+ 6 v0) - (u_nb +- 6 v_nb) of FP32 data as an unevaluated
// float pair jh + jl, with jh carrying its sign and |jl| <= ulp(jh) / 2, within
// ~2^-46 S of the exact value (S = |u0| + 6|v0| + |u_nb| + 6|v_nb|): the four
// terms u0, s 6 v0, -u_nb, s 6 v_nb (s = -1 on the low face, +1 on the high
// one) are exact as pairs (fma gives the rounding error of 6v), three two-sums
// add them, the five small terms are rounded into jl, and a last two-sum
// renormalises (after cancellation the small terms may outweigh the sum).
__device__ __forceinline__ void jump_pair(float u0, float v0, float unb, float vnb, bool low,
                                          float& jh, float& jl) {
  const float sv = low ? -1.0f : 1.0f;
  const float p0 = __fmul_rn(6.0f, v0), e0 = fmaf(6.0f, v0, -p0);
  const float p1 = __fmul_rn(6.0f, vnb), e1 = fmaf(6.0f, vnb, -p1);
  float s1, t1, s2, t2, s3, t3;
  two_sum(u0, sv * p0, s1, t1);
  two_sum(s1, -unb, s2, t2);
  two_sum(s2, sv * p1, s3, t3);
  two_sum(s3, __fadd_rn(__fadd_rn(__fadd_rn(t1, t2), t3), sv * __fadd_rn(e0, e1)), jh, jl);
}

// jump_pair of float-pair averages u0 + l0 and u_nb + l_nb (FP32 first
// moments): the hi parts' jump plus l0 - l_nb, renormalised; within ~2^-45 S
// of the exact jump of hi + lo (each low part is below 2^-24 of its hi, so
// their difference and its addition round at ~2^-48 S and ~2^-46 S).
__device__ __forceinline__ void jump_pair_lo(float u0, float l0, float v0, float unb, float lnb,
                                             float vnb, bool low, float& jh, float& jl) {
  jump_pair(u0, v0, unb, vnb, low, jh, jl);
  two_sum(jh, __fadd_rn(jl, __fsub_rn(l0, lnb)), jh, jl);
}

// FP32 inputs: decide in FP32 when the rounding-error bound allows, else
// evaluate the jump and the threshold as unevaluated float pairs (error-free
// sums and products), so that the decision equals the FP64 one away from the
// threshold without any FP64 arithmetic (a dependent FP64 division costs about
// a thousand cycles on GB300, and the band is wide on fine grids: the jump is
// a difference of O(|u|) numbers, the threshold O(h |u|)).
//   Fast test: with S = |u0| + 6|v0| + |u_nb| + 6|v_nb|, the FP32 jump (four
//   roundings) is within 3 * 2^-24 * S of the exact one (bounded here by
//   6e-7 S), and r = thr*h*max(|u0|,1e-12) (three roundings) within a
//   relative 4.8e-7; hthr = (float)(thr*h), hthr_lo = (float)(thr*h - hthr).
//   Pair test: the four terms u0, -+6v0, -u_nb, -+6v_nb are exact as pairs
//   (fma gives the rounding error of 6v); three two-sums leave the jump as
//   jh + jl with jl rounded from five small terms, so within ~2^-46 S of the
//   exact value, renormalised so that jh has the jump's sign; r = nrm * (hthr
//   + hthr_lo) as rh + rl within ~2^-46 r.  The sign of (|jh| - rh) +
//   (+-jl - rl) then equals the sign of |jump| - r
//   unless they are within ~1e-13 S, i.e. well inside a 1e-6 relative band
//   around the threshold for any grid with S / r below 1e7.
__device__ __forceinline__ bool kxrcf_troubled(float um, float u0, float up, float vm, float v0,
                                               float vp, bool left, double /*h*/, double /*thr*/,
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
  const float nrm = fmaxf(fabsf(u0), 1e-12f);
  const float r = hthr * nrm;
  if (j - e > r * (1.0f + 4.8e-7f)) return true;
  if (j + e < r * (1.0f - 4.8e-7f)) return false;
  float jh, jl;
  jump_pair(u0, v0, left ? um : up, left ? vm : vp, left, jh, jl);
  if (jh < 0.0f) {
    jh = -jh;
    jl = -jl;
  }
  const float rh = __fmul_rn(nrm, hthr);
  const float rl = __fadd_rn(fmaf(nrm, hthr, -rh), __fmul_rn(nrm, hthr_lo));
  return __fadd_rn(__fsub_rn(jh, rh), __fsub_rn(jl, rl)) > 0.0f;
}

// Side of the inflow face: left when the velocity m/rho is >= 0 (its sign
// without the division when rho > 0).
template <typename R>
__device__ __forceinline__ bool inflow_left(R rho, R m) {
  return rho > R(0) ? (m >= R(0)) : (m / rho >= R(0));
}

}  // namespace hw
