// 2D pieces shared by the stage kernel and the adjoint kernels of the hybrid
// HWENO scheme (Zhao & Qiu, arXiv:2002.08816, Sec. 2.2): the Euler flux and
// its eigen-system, the wave speeds, and Step 5.1's nonlinear combination on
// the generated straight-line maps of hweno2d_coef.cuh.
#pragma once
#include <math.h>

#include "hweno1d_recon.cuh"
#include "hweno2d_coef.cuh"

namespace hw {

// ------------------------------------------------------------ physics (2D)

template <typename R>
struct Euler2D {
  static __device__ __forceinline__ void flux(R g, const R* U, int dir, R* F) {
    const R rho = U[0], m = U[1], n = U[2], E = U[3];
    const R ir = fast_rcp(rho);  // FP32: approximate; FP64: 1 / rho
    const R mu = sizeof(R) == 4 ? m * ir : m / rho;
    const R nu = sizeof(R) == 4 ? n * ir : n / rho;
    const R p = (g - R(1)) * (E - R(0.5) * (m * mu + n * nu));
    const R vn = dir == 0 ? mu : nu;
    F[0] = dir == 0 ? m : n;
    F[1] = m * vn + (dir == 0 ? p : R(0));
    F[2] = n * vn + (dir == 1 ? p : R(0));
    F[3] = vn * (E + p);
  }
  // Right (columns: v-c, v, v, v+c with v the normal velocity) and left
  // eigenvectors of dF/dU (dir 0) or dG/dU (dir 1) at U.
  static __device__ __forceinline__ void eigen(R g, const R* U, int dir, R Rm[4][4], R Lm[4][4]) {
    // FP32 with one approximate reciprocal of rho and an approximate square
    // root; FP64 correctly rounded
    const R rho = U[0];
    const R ir = sizeof(R) == 4 ? fast_rcp(rho) : R(1);
    const R mu = sizeof(R) == 4 ? U[1] * ir : U[1] / rho;
    const R nu = sizeof(R) == 4 ? U[2] * ir : U[2] / rho;
    const R q2 = mu * mu + nu * nu;
    const R p = (g - R(1)) * (U[3] - R(0.5) * rho * q2);
    const R c = sizeof(R) == 4 ? fast_sqrt(g * p * ir) : sqrt(g * p / rho);
    const R H = sizeof(R) == 4 ? (U[3] + p) * ir : (U[3] + p) / rho;
    const R ic = fast_rcp(c);
    const R b1 = (g - R(1)) * ic * ic;
    const R b2 = R(0.5) * b1 * q2;
    const R vn = dir == 0 ? mu : nu;
    // columns
    Rm[0][0] = R(1); Rm[0][1] = R(1); Rm[0][3] = R(1);
    Rm[3][0] = H - vn * c; Rm[3][1] = R(0.5) * q2; Rm[3][3] = H + vn * c;
    if (dir == 0) {
      Rm[1][0] = mu - c; Rm[1][1] = mu; Rm[1][3] = mu + c;
      Rm[2][0] = nu;     Rm[2][1] = nu; Rm[2][3] = nu;
      Rm[0][2] = R(0); Rm[1][2] = R(0); Rm[2][2] = R(1); Rm[3][2] = nu;
    } else {
      Rm[1][0] = mu;     Rm[1][1] = mu; Rm[1][3] = mu;
      Rm[2][0] = nu - c; Rm[2][1] = nu; Rm[2][3] = nu + c;
      Rm[0][2] = R(0); Rm[1][2] = R(1); Rm[2][2] = R(0); Rm[3][2] = mu;
    }
    // rows
    const R ex = dir == 0 ? ic : R(0), ey = dir == 1 ? ic : R(0);
    Lm[0][0] = R(0.5) * (b2 + vn * ic);
    Lm[0][1] = R(-0.5) * (b1 * mu + ex);
    Lm[0][2] = R(-0.5) * (b1 * nu + ey);
    Lm[0][3] = R(0.5) * b1;
    Lm[1][0] = R(1) - b2;
    Lm[1][1] = b1 * mu;
    Lm[1][2] = b1 * nu;
    Lm[1][3] = -b1;
    if (dir == 0) {
      Lm[2][0] = -nu; Lm[2][1] = R(0); Lm[2][2] = R(1); Lm[2][3] = R(0);
    } else {
      Lm[2][0] = -mu; Lm[2][1] = R(1); Lm[2][2] = R(0); Lm[2][3] = R(0);
    }
    Lm[3][0] = R(0.5) * (b2 - vn * ic);
    Lm[3][1] = R(-0.5) * (b1 * mu - ex);
    Lm[3][2] = R(-0.5) * (b1 * nu - ey);
    Lm[3][3] = R(0.5) * b1;
  }
};

template <typename R, int C>
__device__ __forceinline__ void phys_flux2(R gas, const R* U, int dir, R* F) {
  if constexpr (C == 1) {
    F[0] = R(0.5) * U[0] * U[0];
  } else {
    Euler2D<R>::flux(gas, U, dir, F);
  }
}

// ------------------------------------------------ packed FP32 (pairs of points)

// (bcast2 and sub2: hweno1d_recon.cuh)
// The Euler flux f (dir 0) or g (dir 1) of two states at once (each component
// a pair), the arithmetic of Euler2D<float>::flux in packed FP32.
__device__ __forceinline__ void euler_flux_x2(float gas, const float2* U, int dir, float2* F) {
  const float2 rho = U[0], m = U[1], n = U[2], E = U[3];
  const float2 ir = make_float2(fast_rcp(rho.x), fast_rcp(rho.y));
  const float2 mu = __fmul2_rn(m, ir), nu = __fmul2_rn(n, ir);
  const float2 q = __ffma2_rn(n, nu, __fmul2_rn(m, mu));  // m mu + n nu
  const float2 p = __fmul2_rn(bcast2(gas - 1.0f), __ffma2_rn(bcast2(-0.5f), q, E));
  const float2 vn = dir == 0 ? mu : nu;
  F[0] = dir == 0 ? m : n;
  F[1] = dir == 0 ? __ffma2_rn(m, vn, p) : __fmul2_rn(m, vn);
  F[2] = dir == 1 ? __ffma2_rn(n, vn, p) : __fmul2_rn(n, vn);
  F[3] = __fmul2_rn(vn, __fadd2_rn(E, p));
}
// The Lax-Friedrichs flux (f(u^-) + f(u^+)) / 2 - h (u^+ - u^-) of two points.
__device__ __forceinline__ float2 lf_x2(float2 fm, float2 fp, float2 um, float2 up, float h) {
  return __ffma2_rn(bcast2(-h), sub2(up, um), __fmul2_rn(bcast2(0.5f), __fadd2_rn(fm, fp)));
}

// f(B + D) - f(B) (dir 0) or g(B + D) - g(B) (dir 1) for a base state B and
// an increment D, FP32, with rounding errors relative to the increment (no
// difference of O(|f|) terms; the float-pair precision HWENO_FP32C): with
// mu = m / rho, nu = n / rho, p = (gamma - 1)(E - (m mu + n nu) / 2),
//   dmu = (dm - mu drho) / (rho + drho), dnu likewise,
//   d(m mu) = m dmu + dm (mu + dmu), and the other products the same way,
//   dp = (gamma - 1)(dE - (d(m mu) + d(n nu)) / 2),
//   d(vn (E + p)) = dvn (E + p + dE + dp) + vn (dE + dp).
template <int C>
__device__ __forceinline__ void flux_inc2(float gas, const float* B, const float* D, int dir,
                                          float* dF) {
  if constexpr (C == 1) {
    dF[0] = D[0] * (B[0] + 0.5f * D[0]);
  } else {
    const float rho = B[0], m = B[1], n = B[2], E = B[3];
    const float dr = D[0], dm = D[1], dn = D[2], dE = D[3];
    const float ir = fast_rcp(rho), ir1 = fast_rcp(rho + dr);
    const float mu = m * ir, nu = n * ir;
    const float dmu = (dm - mu * dr) * ir1, dnu = (dn - nu * dr) * ir1;
    const float dmm = m * dmu + dm * (mu + dmu);  // d(m mu)
    const float dnn = n * dnu + dn * (nu + dnu);  // d(n nu)
    const float g1 = gas - 1.0f;
    const float p = g1 * (E - 0.5f * (m * mu + n * nu));
    const float dp = g1 * (dE - 0.5f * (dmm + dnn));
    if (dir == 0) {
      dF[0] = dm;
      dF[1] = dmm + dp;
      dF[2] = n * dmu + dn * (mu + dmu);  // d(n mu)
      dF[3] = dmu * ((E + p) + (dE + dp)) + mu * (dE + dp);
    } else {
      dF[0] = dn;
      dF[1] = m * dnu + dm * (nu + dnu);  // d(m nu)
      dF[2] = dnn + dp;
      dF[3] = dnu * ((E + p) + (dE + dp)) + nu * (dE + dp);
    }
  }
}

// flux_inc2 (Euler) for two increments D over one base B at once (each
// increment component a pair), the same arithmetic in packed FP32.
__device__ __forceinline__ void flux_inc2_x2(float gas, const float* B, const float2* D, int dir,
                                             float2* dF) {
  const float rho = B[0], m = B[1], n = B[2], E = B[3];
  const float2 dr = D[0], dm = D[1], dn = D[2], dE = D[3];
  const float ir = fast_rcp(rho);
  const float2 ir1 = make_float2(fast_rcp(rho + dr.x), fast_rcp(rho + dr.y));
  const float mu = m * ir, nu = n * ir;
  const float2 dmu = __fmul2_rn(__ffma2_rn(bcast2(-mu), dr, dm), ir1);
  const float2 dnu = __fmul2_rn(__ffma2_rn(bcast2(-nu), dr, dn), ir1);
  // d(m mu), d(n nu)
  const float2 dmm = __ffma2_rn(bcast2(m), dmu, __fmul2_rn(dm, __fadd2_rn(bcast2(mu), dmu)));
  const float2 dnn = __ffma2_rn(bcast2(n), dnu, __fmul2_rn(dn, __fadd2_rn(bcast2(nu), dnu)));
  const float g1 = gas - 1.0f;
  const float p = g1 * (E - 0.5f * (m * mu + n * nu));
  const float2 dp = __fmul2_rn(bcast2(g1), __ffma2_rn(bcast2(-0.5f), __fadd2_rn(dmm, dnn), dE));
  const float2 sE = __fadd2_rn(dE, dp);  // d(E + p)
  if (dir == 0) {
    dF[0] = dm;
    dF[1] = __fadd2_rn(dmm, dp);
    dF[2] = __ffma2_rn(bcast2(n), dmu, __fmul2_rn(dn, __fadd2_rn(bcast2(mu), dmu)));  // d(n mu)
    dF[3] = __ffma2_rn(dmu, __fadd2_rn(bcast2(E + p), sE), __fmul2_rn(bcast2(mu), sE));
  } else {
    dF[0] = dn;
    dF[1] = __ffma2_rn(bcast2(m), dnu, __fmul2_rn(dm, __fadd2_rn(bcast2(nu), dnu)));  // d(m nu)
    dF[2] = __fadd2_rn(dnn, dp);
    dF[3] = __ffma2_rn(dnu, __fadd2_rn(bcast2(E + p), sE), __fmul2_rn(bcast2(nu), sE));
  }
}

// max |f'| (dir 0) and |g'| (dir 1) at a cell average; NaN when not physical
template <typename R, int C>
__device__ __forceinline__ void wave_speeds2(R gas, const R* U, R& sx, R& sy) {
  if constexpr (C == 1) {
    sx = sy = fabs(U[0]);
  } else {
    const R rho = U[0];
    if (!(rho > R(0))) {
      sx = sy = R(NAN);
      return;
    }
    const R ir = sizeof(R) == 4 ? fast_rcp(rho) : R(1);
    const R mu = sizeof(R) == 4 ? U[1] * ir : U[1] / rho;
    const R nu = sizeof(R) == 4 ? U[2] * ir : U[2] / rho;
    const R p = (gas - R(1)) * (U[3] - R(0.5) * rho * (mu * mu + nu * nu));
    if (!(p > R(0))) {
      sx = sy = R(NAN);
      return;
    }
    const R c = sizeof(R) == 4 ? fast_sqrt(gas * p * ir) : sqrt(gas * p / rho);
    sx = fabs(mu) + c;
    sy = fabs(nu) + c;
  }
}

// ------------------------------------------------------ HWENO helpers (2D)

template <int NG, typename R>
__device__ __forceinline__ void p0_faces(const R* d, R* o) {
  if constexpr (NG == 3) hw2::p0_faces_ng3(d, o); else hw2::p0_faces_ng2(d, o);
}
template <int NG, typename R>
__device__ __forceinline__ void p0_interior(const R* d, R* o) {
  if constexpr (NG == 3) hw2::p0_interior_ng3(d, o); else hw2::p0_interior_ng2(d, o);
}
// The same two maps on two components of a cell at once (packed FP32).
template <int NG>
__device__ __forceinline__ void p0_faces_x2(const float2* d, float2* o) {
  if constexpr (NG == 3) hw2::p0_faces_ng3_x2(d, o); else hw2::p0_faces_ng2_x2(d, o);
}
template <int NG>
__device__ __forceinline__ void p0_interior_x2(const float2* d, float2* o) {
  if constexpr (NG == 3) hw2::p0_interior_ng3_x2(d, o); else hw2::p0_interior_ng2_x2(d, o);
}
template <int NG, typename R>
__device__ __forceinline__ void q_faces(int n, const R* d, R* o) {
  if constexpr (NG == 3) {
    if (n == 1) hw2::q1_faces_ng3(d, o);
    else if (n == 2) hw2::q2_faces_ng3(d, o);
    else if (n == 3) hw2::q3_faces_ng3(d, o);
    else hw2::q4_faces_ng3(d, o);
  } else {
    if (n == 1) hw2::q1_faces_ng2(d, o);
    else if (n == 2) hw2::q2_faces_ng2(d, o);
    else if (n == 3) hw2::q3_faces_ng2(d, o);
    else hw2::q4_faces_ng2(d, o);
  }
}

// HWENO values (Step 5.1) at the interface points [p_lo, p_hi) of one scalar
// field from its 19 data: tau of Eq. (tao4), weights of Eq. (99), and the
// combination omega_0 (p0/gamma_0 - sum gamma_n/gamma_0 p_n) + sum omega_n p_n
// accumulated candidate by candidate (it is linear in the candidates).
template <int NG, typename R>
__device__ __forceinline__ void hweno2d_faces(const R* d, const R* gam, R eps, int p_lo,
                                              int p_hi, R* out) {
  constexpr int NF = 4 * NG;
  R b[5];
  b[0] = hw2::beta_p0(d);
  b[1] = hw2::beta_q1(d);
  b[2] = hw2::beta_q2(d);
  b[3] = hw2::beta_q3(d);
  b[4] = hw2::beta_q4(d);
  const R s = R(0.25) * (fabs(b[0] - b[1]) + fabs(b[0] - b[2]) + fabs(b[0] - b[3]) + fabs(b[0] - b[4]));
  const R tau = s * s;
  // FP32: approximate reciprocals (the weights need a few ulp, not IEEE
  // rounding); FP64: correctly rounded quotients
  R a[5], sum = R(0);
#pragma unroll
  for (int n = 0; n < 5; ++n) {
    a[n] = gam[n] * (R(1) + (sizeof(R) == 4 ? tau * fast_rcp(b[n] + eps) : tau / (b[n] + eps)));
    sum += a[n];
  }
  const R inv = fast_rcp(sum);
  const R c0 = sizeof(R) == 4 ? a[0] * inv * fast_rcp(gam[0]) : a[0] * inv / gam[0];
  R tmp[NF];
  p0_faces<NG>(d, tmp);
#pragma unroll
  for (int p = 0; p < NF; ++p)
    if (p >= p_lo && p < p_hi) out[p] = c0 * tmp[p];
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    const R cn = a[n + 1] * inv - c0 * gam[n + 1];
    q_faces<NG>(n + 1, d, tmp);
#pragma unroll
    for (int p = 0; p < NF; ++p)
      if (p >= p_lo && p < p_hi) out[p] += cn * tmp[p];
  }
}

// The same on two fields at once (packed FP32: the smoothness indicators and
// the candidates' values in pairs, the weights of each field in scalar FP32).
template <int NG>
__device__ __forceinline__ void q_faces_x2(int n, const float2* d, float2* o) {
  if constexpr (NG == 3) {
    if (n == 1) hw2::q1_faces_ng3_x2(d, o);
    else if (n == 2) hw2::q2_faces_ng3_x2(d, o);
    else if (n == 3) hw2::q3_faces_ng3_x2(d, o);
    else hw2::q4_faces_ng3_x2(d, o);
  } else {
    if (n == 1) hw2::q1_faces_ng2_x2(d, o);
    else if (n == 2) hw2::q2_faces_ng2_x2(d, o);
    else if (n == 3) hw2::q3_faces_ng2_x2(d, o);
    else hw2::q4_faces_ng2_x2(d, o);
  }
}
template <int NG>
__device__ __forceinline__ void hweno2d_faces_x2(const float2* d, const float* gam, float eps,
                                                 int p_lo, int p_hi, float2* out) {
  constexpr int NF = 4 * NG;
  const float2 b2[5] = {hw2::beta_p0_x2(d), hw2::beta_q1_x2(d), hw2::beta_q2_x2(d),
                        hw2::beta_q3_x2(d), hw2::beta_q4_x2(d)};
  float2 c02, cn2[4];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    float b[5];
#pragma unroll
    for (int n = 0; n < 5; ++n) b[n] = h ? b2[n].y : b2[n].x;
    const float s = 0.25f * (fabsf(b[0] - b[1]) + fabsf(b[0] - b[2]) + fabsf(b[0] - b[3]) +
                             fabsf(b[0] - b[4]));
    const float tau = s * s;
    float a[5], sum = 0.0f;
#pragma unroll
    for (int n = 0; n < 5; ++n) {
      a[n] = gam[n] * (1.0f + tau * fast_rcp(b[n] + eps));
      sum += a[n];
    }
    const float inv = fast_rcp(sum);
    const float c0 = a[0] * inv * fast_rcp(gam[0]);
    if (h) c02.y = c0; else c02.x = c0;
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      const float cn = a[n + 1] * inv - c0 * gam[n + 1];
      if (h) cn2[n].y = cn; else cn2[n].x = cn;
    }
  }
  float2 tmp[NF];
  p0_faces_x2<NG>(d, tmp);
#pragma unroll
  for (int p = 0; p < NF; ++p)
    if (p >= p_lo && p < p_hi) out[p] = __fmul2_rn(c02, tmp[p]);
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    q_faces_x2<NG>(n + 1, d, tmp);
#pragma unroll
    for (int p = 0; p < NF; ++p)
      if (p >= p_lo && p < p_hi) out[p] = __ffma2_rn(cn2[n], tmp[p], out[p]);
  }
}

// Step 4 for a troubled Euler cell (lx, ly) of the flag grid: vbar from the
// x-neighbours in the x characteristic fields, wbar from the y-neighbours in
// the y fields, with the 1D Step 1 formula, written to sm.lim[slot] (S with
// kLimList) or to sm.vl / sm.wl at (lx, ly).  Rare: kept out of line so that
// its registers do not weigh on the common path.
template <typename S, typename R>
__device__ __noinline__ void limit_euler2d(S& sm, int lx, int ly, int slot, R g0, R g1, R g2,
                                           R g3, R g4, R eps, R gas) {
  const R gam[5] = {g0, g1, g2, g3, g4};  // by value: no caller array on the stack
  const int rx = lx + 1 + S::kPadX, ry = ly + 1;  // raw index of the cell
  R U[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) U[c] = sm.u[c][0][ry][rx];
#pragma unroll 1
  for (int dir = 0; dir < 2; ++dir) {
    R Rm[4][4], Lm[4][4];
    Euler2D<R>::eigen(gas, U, dir, Rm, Lm);
    const int sx = dir == 0 ? 1 : 0, sy = dir == 0 ? 0 : 1;
    const int mom = dir == 0 ? 1 : 2;
    R q[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      R wv[5];
#pragma unroll
      for (int s = 0; s < 3; ++s) {
        wv[s] = R(0);
#pragma unroll
        for (int c = 0; c < 4; ++c) wv[s] += Lm[f][c] * sm.u[c][0][ry + (s - 1) * sy][rx + (s - 1) * sx];
      }
      wv[3] = R(0);
      wv[4] = R(0);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        wv[3] += Lm[f][c] * sm.u[c][mom][ry - sy][rx - sx];
        wv[4] += Lm[f][c] * sm.u[c][mom][ry + sy][rx + sx];
      }
      q[f] = limit_first_moment(wv[0], wv[1], wv[2], wv[3], wv[4], gam, eps);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const R v = Rm[c][0] * q[0] + Rm[c][1] * q[1] + Rm[c][2] * q[2] + Rm[c][3] * q[3];
      if constexpr (S::kLimList) sm.lim[slot][c][dir] = v;
      else if (dir == 0) sm.vl[c][ly][lx] = v;
      else sm.wl[c][ly][lx] = v;
    }
  }
}

}  // namespace hw
