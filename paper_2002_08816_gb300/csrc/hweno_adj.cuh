// Reverse-mode pieces of the hybrid HWENO scheme (Zhao & Qiu,
// arXiv:2002.08816) with its troubled cells held fixed: the vector-Jacobian
// products of the nonlinear weights (Eq. (99) with tau of Eq. (tao5) or
// Eq. (tao4)), of Step 1's modified first moment, of the Euler flux and of the
// Euler eigen-system (by a forward-mode number with four tangents).
// At a kink of |beta_0 - beta_n| the derivative taken is the one with
// sign(0) = 0.
#pragma once
#include <math.h>

#include "hweno2d_common.cuh"

namespace hw {

// ------------------------------------------------------------- weights

// Weights (99): a_n = gamma_n (1 + tau/(b_n + eps)), tau = (sfac sum_{n>=1}
// |b_0 - b_n|)^2, w_n = a_n / sum a; combination coefficients c_0 = w_0/gamma_0,
// c_n = w_n - c_0 gamma_n, so that the combined value is sum_n c_n v_n.
template <typename R, int N>
struct NLWeights {
  R a[N], c[N], inv, s, tau;
  __device__ __forceinline__ NLWeights(const R* gam, R eps, R sfac, const R* b) {
    R t = R(0);
#pragma unroll
    for (int n = 1; n < N; ++n) t += fabs(b[0] - b[n]);
    s = sfac * t;
    tau = s * s;
    // FP32: approximate reciprocals, as the forward kernels' weights
    R sum = R(0);
#pragma unroll
    for (int n = 0; n < N; ++n) {
      a[n] = gam[n] * (R(1) + (sizeof(R) == 4 ? tau * fast_rcp(b[n] + eps) : tau / (b[n] + eps)));
      sum += a[n];
    }
    inv = fast_rcp(sum);
    c[0] = sizeof(R) == 4 ? a[0] * inv * fast_rcp(gam[0]) : a[0] * inv / gam[0];
#pragma unroll
    for (int n = 1; n < N; ++n) c[n] = a[n] * inv - c[0] * gam[n];
  }
  // lc: adjoints of c_0..c_{N-1}; adds the adjoints of b_0..b_{N-1} to lb.
  __device__ __forceinline__ void vjp(const R* gam, R eps, R sfac, const R* b, const R* lc,
                                      R* lb) const {
    R lc0 = lc[0], linv = R(0), la[N];
#pragma unroll
    for (int n = 1; n < N; ++n) {
      la[n] = lc[n] * inv;
      linv += lc[n] * a[n];
      lc0 -= lc[n] * gam[n];
    }
    const R ig0 = fast_rcp(gam[0]);
    la[0] = sizeof(R) == 4 ? lc0 * inv * ig0 : lc0 * inv / gam[0];
    linv += sizeof(R) == 4 ? lc0 * a[0] * ig0 : lc0 * a[0] / gam[0];
    const R lsum = -linv * inv * inv;
    R ltau = R(0);
#pragma unroll
    for (int n = 0; n < N; ++n) {
      la[n] += lsum;
      const R ib = fast_rcp(b[n] + eps);
      ltau += la[n] * gam[n] * ib;
      lb[n] -= la[n] * gam[n] * tau * ib * ib;
    }
    const R lt = R(2) * s * sfac * ltau;
#pragma unroll
    for (int n = 1; n < N; ++n) {
      const R sg = b[0] > b[n] ? R(1) : (b[0] < b[n] ? R(-1) : R(0));
      lb[0] += lt * sg;
      lb[n] -= lt * sg;
    }
  }
};

// Step 1's modified first moment (limit_first_moment) and its gradient:
// g[0..4] += lam * d out / d (u_m, u_0, u_p, v_m, v_p).  Returns the value.
template <typename R>
__device__ __forceinline__ R limit_first_moment_vjp(R um, R u0, R up, R vm, R vp, const R* gam,
                                                    R eps, R lam, R* g) {
  const R q[3] = {R(5.0 / 76.0) * (up - um) - R(11.0 / 38.0) * (vm + vp),
                  R(1.0 / 12.0) * (u0 - um), R(1.0 / 12.0) * (up - u0)};
  const R t1 = R(29.0 / 38.0) * (um - up) + R(60.0 / 19.0) * (vm + vp);
  const R t2 = R(9.0 / 4.0) * (um + up) - R(9.0 / 2.0) * u0 + R(15.0 / 2.0) * (vm - vp);
  const R t3 = (um - up) + R(12) * (vm + vp);
  const R t4 = R(5.0 / 2.0) * (um + up) - R(5) * u0 + R(9) * (vm - vp);
  const R t5 = (um - R(2) * u0 + up) + R(6) * (vm - vp);
  const R d1 = u0 - um, d2 = up - u0;
  const R b[3] = {t1 * t1 + t2 * t2 + R(3905.0 / 1444.0) * t3 * t3 + R(1.0 / 12.0) * t4 * t4 +
                      R(109341.0 / 448.0) * t5 * t5,
                  d1 * d1, d2 * d2};
  NLWeights<R, 3> w(gam, eps, R(0.5), b);
  const R lc[3] = {lam * q[0], lam * q[1], lam * q[2]};
  R lb[3] = {R(0), R(0), R(0)};
  w.vjp(gam, eps, R(0.5), b, lc, lb);
  const R lq0 = lam * w.c[0], lq1 = lam * w.c[1], lq2 = lam * w.c[2];
  g[0] += -R(5.0 / 76.0) * lq0 - R(1.0 / 12.0) * lq1;
  g[1] += R(1.0 / 12.0) * (lq1 - lq2);
  g[2] += R(5.0 / 76.0) * lq0 + R(1.0 / 12.0) * lq2;
  g[3] += -R(11.0 / 38.0) * lq0;
  g[4] += -R(11.0 / 38.0) * lq0;
  const R e1 = R(2) * lb[0] * t1, e2 = R(2) * lb[0] * t2;
  const R e3 = R(2.0 * 3905.0 / 1444.0) * lb[0] * t3, e4 = R(2.0 / 12.0) * lb[0] * t4;
  const R e5 = R(2.0 * 109341.0 / 448.0) * lb[0] * t5;
  g[0] += R(29.0 / 38.0) * e1 + R(9.0 / 4.0) * e2 + e3 + R(5.0 / 2.0) * e4 + e5;
  g[1] += -R(9.0 / 2.0) * e2 - R(5) * e4 - R(2) * e5;
  g[2] += -R(29.0 / 38.0) * e1 + R(9.0 / 4.0) * e2 - e3 + R(5.0 / 2.0) * e4 + e5;
  g[3] += R(60.0 / 19.0) * e1 + R(15.0 / 2.0) * e2 + R(12) * e3 + R(9) * e4 + R(6) * e5;
  g[4] += R(60.0 / 19.0) * e1 - R(15.0 / 2.0) * e2 + R(12) * e3 - R(9) * e4 - R(6) * e5;
  const R f1 = R(2) * lb[1] * d1, f2 = R(2) * lb[2] * d2;
  g[0] -= f1;
  g[1] += f1 - f2;
  g[2] += f2;
  return w.c[0] * q[0] + w.c[1] * q[1] + w.c[2] * q[2];
}

// ---------------------------------------------------------------- 2D HWENO

template <int NG, typename R>
__device__ __forceinline__ void p0_faces_T(const R* l, R* g) {
  if constexpr (NG == 3) hw2::p0_faces_ng3_T(l, g); else hw2::p0_faces_ng2_T(l, g);
}
template <int NG, typename R>
__device__ __forceinline__ void p0_interior_T(const R* l, R* g) {
  if constexpr (NG == 3) hw2::p0_interior_ng3_T(l, g); else hw2::p0_interior_ng2_T(l, g);
}
// The same two transposes on two components at once (packed FP32).
template <int NG>
__device__ __forceinline__ void p0_faces_T_x2(const float2* l, float2* g) {
  if constexpr (NG == 3) hw2::p0_faces_ng3_T_x2(l, g); else hw2::p0_faces_ng2_T_x2(l, g);
}
template <int NG>
__device__ __forceinline__ void p0_interior_T_x2(const float2* l, float2* g) {
  if constexpr (NG == 3) hw2::p0_interior_ng3_T_x2(l, g); else hw2::p0_interior_ng2_T_x2(l, g);
}
template <int NG, typename R>
__device__ __forceinline__ void q_faces_T(int n, const R* l, R* g) {
  if constexpr (NG == 3) {
    if (n == 1) hw2::q1_faces_ng3_T(l, g);
    else if (n == 2) hw2::q2_faces_ng3_T(l, g);
    else if (n == 3) hw2::q3_faces_ng3_T(l, g);
    else hw2::q4_faces_ng3_T(l, g);
  } else {
    if (n == 1) hw2::q1_faces_ng2_T(l, g);
    else if (n == 2) hw2::q2_faces_ng2_T(l, g);
    else if (n == 3) hw2::q3_faces_ng2_T(l, g);
    else hw2::q4_faces_ng2_T(l, g);
  }
}

// Gradient of hweno2d_faces: g[0..18] += (d out[p]/d d)^T lam[p] over the
// interface points (lam zero outside the points the forward evaluated).
template <int NG, typename R>
__device__ __forceinline__ void hweno2d_faces_vjp(const R* d, const R* gam, R eps, const R* lam,
                                                  R* g) {
  constexpr int NF = 4 * NG;
  const R b[5] = {hw2::beta_p0(d), hw2::beta_q1(d), hw2::beta_q2(d), hw2::beta_q3(d),
                  hw2::beta_q4(d)};
  NLWeights<R, 5> w(gam, eps, R(0.25), b);
  R tmp[NF], sl[NF], lc[5];
  p0_faces<NG>(d, tmp);
  lc[0] = R(0);
#pragma unroll
  for (int p = 0; p < NF; ++p) {
    lc[0] += lam[p] * tmp[p];
    sl[p] = w.c[0] * lam[p];
  }
  p0_faces_T<NG>(sl, g);
#pragma unroll
  for (int n = 1; n < 5; ++n) {
    q_faces<NG>(n, d, tmp);
    lc[n] = R(0);
#pragma unroll
    for (int p = 0; p < NF; ++p) {
      lc[n] += lam[p] * tmp[p];
      sl[p] = w.c[n] * lam[p];
    }
    q_faces_T<NG>(n, sl, g);
  }
  R lb[5] = {R(0), R(0), R(0), R(0), R(0)};
  w.vjp(gam, eps, R(0.25), b, lc, lb);
  hw2::beta_p0_grad(d, lb[0], g);
  hw2::beta_q1_grad(d, lb[1], g);
  hw2::beta_q2_grad(d, lb[2], g);
  hw2::beta_q3_grad(d, lb[3], g);
  hw2::beta_q4_grad(d, lb[4], g);
}

// ------------------------------------------------------------- Euler

// o = A(U)^T l, A = dF/dU (dir 0) or dG/dU (dir 1) of the 2D Euler flux
// (Burgers f = g = u^2/2: o = u l).
template <typename R, int C>
__device__ __forceinline__ void flux_jt2(R gas, const R* U, int dir, const R* l, R* o) {
  if constexpr (C == 1) {
    o[0] = U[0] * l[0];
  } else {
    const R ir = fast_rcp(U[0]);  // FP32: approximate, as the forward flux
    const R u = U[1] * ir, v = U[2] * ir;
    const R g1 = gas - R(1);
    const R kq = g1 * R(0.5) * (u * u + v * v);
    const R p = g1 * U[3] - U[0] * kq;
    const R H = (U[3] + p) * ir;
    if (dir == 0) {
      o[0] = l[1] * (kq - u * u) - l[2] * u * v + l[3] * u * (kq - H);
      o[1] = l[0] + l[1] * (R(3) - gas) * u + l[2] * v + l[3] * (H - g1 * u * u);
      o[2] = -l[1] * g1 * v + l[2] * u - l[3] * g1 * u * v;
      o[3] = l[1] * g1 + l[3] * gas * u;
    } else {
      o[0] = -l[1] * u * v + l[2] * (kq - v * v) + l[3] * v * (kq - H);
      o[1] = l[1] * v - l[2] * g1 * u - l[3] * g1 * u * v;
      o[2] = l[0] + l[1] * u + l[2] * (R(3) - gas) * v + l[3] * (H - g1 * v * v);
      o[3] = l[2] * g1 + l[3] * gas * v;
    }
  }
}

// flux_jt2 (Euler) of two points at once: each component a pair, the same
// arithmetic in packed FP32 (one approximate reciprocal per point).
__device__ __forceinline__ void flux_jt2_x2(float gas, const float2* U, int dir, const float2* l,
                                            float2* o) {
  const float2 ir = make_float2(fast_rcp(U[0].x), fast_rcp(U[0].y));
  const float2 u = __fmul2_rn(U[1], ir), v = __fmul2_rn(U[2], ir);
  const float g1 = gas - 1.0f;
  const float2 kq = __fmul2_rn(bcast2(g1 * 0.5f), __ffma2_rn(v, v, __fmul2_rn(u, u)));
  const float2 p = __ffma2_rn(bcast2(-1.0f), __fmul2_rn(U[0], kq), __fmul2_rn(bcast2(g1), U[3]));
  const float2 H = __fmul2_rn(__fadd2_rn(U[3], p), ir);
  const float2 uv = __fmul2_rn(u, v);
  if (dir == 0) {
    const float2 uu = __fmul2_rn(u, u);
    // l1 (kq - u u) - l2 u v + l3 u (kq - H)
    o[0] = __ffma2_rn(l[3], __fmul2_rn(u, sub2(kq, H)),
                      __ffma2_rn(l[1], sub2(kq, uu), __fmul2_rn(bcast2(-1.0f), __fmul2_rn(l[2], uv))));
    // l0 + l1 (3 - gamma) u + l2 v + l3 (H - g1 u u)
    o[1] = __ffma2_rn(l[3], __ffma2_rn(bcast2(-g1), uu, H),
                      __ffma2_rn(l[2], v, __ffma2_rn(__fmul2_rn(l[1], bcast2(3.0f - gas)), u, l[0])));
    // -l1 g1 v + l2 u - l3 g1 u v
    o[2] = __ffma2_rn(__fmul2_rn(l[3], bcast2(-g1)), uv,
                      __ffma2_rn(l[2], u, __fmul2_rn(__fmul2_rn(l[1], bcast2(-g1)), v)));
    // l1 g1 + l3 gamma u
    o[3] = __ffma2_rn(__fmul2_rn(l[3], bcast2(gas)), u, __fmul2_rn(l[1], bcast2(g1)));
  } else {
    const float2 vv = __fmul2_rn(v, v);
    // -l1 u v + l2 (kq - v v) + l3 v (kq - H)
    o[0] = __ffma2_rn(l[3], __fmul2_rn(v, sub2(kq, H)),
                      __ffma2_rn(l[2], sub2(kq, vv), __fmul2_rn(bcast2(-1.0f), __fmul2_rn(l[1], uv))));
    // l1 v - l2 g1 u - l3 g1 u v
    o[1] = __ffma2_rn(__fmul2_rn(l[3], bcast2(-g1)), uv,
                      __ffma2_rn(l[1], v, __fmul2_rn(__fmul2_rn(l[2], bcast2(-g1)), u)));
    // l0 + l1 u + l2 (3 - gamma) v + l3 (H - g1 v v)
    o[2] = __ffma2_rn(l[3], __ffma2_rn(bcast2(-g1), vv, H),
                      __ffma2_rn(__fmul2_rn(l[2], bcast2(3.0f - gas)), v, __ffma2_rn(l[1], u, l[0])));
    // l2 g1 + l3 gamma v
    o[3] = __ffma2_rn(__fmul2_rn(l[3], bcast2(gas)), v, __fmul2_rn(l[2], bcast2(g1)));
  }
}

// A number with four tangents (forward mode), for the derivatives of the
// eigen-system with respect to the cell average.
template <typename R>
struct Tan4 {
  R v, d[4];
  __device__ __forceinline__ Tan4() {}
  __device__ __forceinline__ Tan4(double x) : v(R(x)) { d[0] = d[1] = d[2] = d[3] = R(0); }
};
template <typename R>
__device__ __forceinline__ Tan4<R> operator+(const Tan4<R>& a, const Tan4<R>& b) {
  Tan4<R> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int k = 0; k < 4; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
template <typename R>
__device__ __forceinline__ Tan4<R> operator-(const Tan4<R>& a, const Tan4<R>& b) {
  Tan4<R> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int k = 0; k < 4; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}
template <typename R>
__device__ __forceinline__ Tan4<R> operator-(const Tan4<R>& a) {
  Tan4<R> r;
  r.v = -a.v;
#pragma unroll
  for (int k = 0; k < 4; ++k) r.d[k] = -a.d[k];
  return r;
}
template <typename R>
__device__ __forceinline__ Tan4<R> operator*(const Tan4<R>& a, const Tan4<R>& b) {
  Tan4<R> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int k = 0; k < 4; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
  return r;
}
template <typename R>
__device__ __forceinline__ Tan4<R> operator/(const Tan4<R>& a, const Tan4<R>& b) {
  Tan4<R> r;
  const R ib = R(1) / b.v;
  r.v = a.v * ib;
#pragma unroll
  for (int k = 0; k < 4; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
  return r;
}
template <typename R>
__device__ __forceinline__ Tan4<R> sqrt(const Tan4<R>& a) {
  Tan4<R> r;
  if constexpr (sizeof(R) == 4) r.v = sqrtf(a.v); else r.v = ::sqrt(a.v);
  const R h = R(0.5) / r.v;
#pragma unroll
  for (int k = 0; k < 4; ++k) r.d[k] = a.d[k] * h;
  return r;
}

// gU[t] += sum lR[c][f] dR[c][f]/dU_t + lL[f][c] dL[f][c]/dU_t for the
// eigen-system Euler2D::eigen of direction dir at U.
template <typename R>
__device__ __noinline__ void euler2d_eigen_vjp(R gas, const R* U, int dir, R (*lR)[4],
                                               R (*lL)[4], R* gU) {
  Tan4<R> Ut[4], Rm[4][4], Lm[4][4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    Ut[c] = Tan4<R>(0.0);
    Ut[c].v = U[c];
    Ut[c].d[c] = R(1);
  }
  Euler2D<Tan4<R>>::eigen(Tan4<R>((double)gas), Ut, dir, Rm, Lm);
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    R s = R(0);
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int f = 0; f < 4; ++f) s += lR[c][f] * Rm[c][f].d[t] + lL[f][c] * Lm[f][c].d[t];
    gU[t] += s;
  }
}

}  // namespace hw
