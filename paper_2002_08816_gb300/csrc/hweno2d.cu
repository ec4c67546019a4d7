// One fused kernel per third-order TVD Runge-Kutta stage of the 2D hybrid
// HWENO scheme (Zhao & Qiu, arXiv:2002.08816, Sec. 2.2).
//
// A CTA owns a TX x TY tile of cells.  It stages the tile and a 3-cell halo
// of the stage input in shared memory, then, on chip:
//   1. alpha_x, alpha_y from the slots the producer of the stage input left
//      (global Lax-Friedrichs fluxes); stage 1 turns them into
//      dt = CFL / (alpha_x/dx + alpha_y/dy), clipped to t_final;
//   2. Step 4 for the tile and 2 halo cells: KXRCF flags (FP32 kernels decide
//      in FP32 when the rounding-error bound allows, else with float pairs;
//      a replayed stage of the adjoint takes its recorded flags) and the
//      first moments of troubled cells modified dimension by dimension with
//      the 1D Step 1 formula (Euler: characteristic fields of the x- and of
//      the y-Jacobian at the cell average), written back into the tile once
//      every flag and limiter has read the raw ones;
//   3. Step 5.1/5.2 at the interface Gauss points of the tile's cells and of
//      the one-cell cross halo: linear p0 (the quartic on the 3x3 stencil),
//      or HWENO when the 3x3 stencil holds a troubled cell (Euler: x-faces in
//      the x characteristic fields, y-faces in the y fields);
//   4. own cells: Step 5.3 at the interior Gauss points, Lax-Friedrichs
//      fluxes at the 4 ng interface points, Eq. (ode2) and Eq. (RK);
//   5. the tile's wave-speed maxima (x and y) into the slots for the next
//      stage, the troubled count and the status bits.
// The reconstruction arithmetic is the generated straight-line code of
// hweno2d_coef.cuh (square cells); the FP32 Euler kernel runs it, the fluxes
// and the HWENO helpers on pairs (two components, two points or two
// characteristic fields) in packed FP32 (fma.rn.f32x2).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "hweno1d_recon.cuh"
#include "hweno2d_common.cuh"
#include "hweno_device.cuh"
#include "hweno.h"
#include "hweno_internal.h"

namespace hw {
namespace {

constexpr int TX = 32, TY = 8;  // cells per CTA of the stage and wave-speed kernels (a warp per row)
constexpr int NT = kThreads2D;
constexpr int NW = NT / 32;
// raw tile: a 3-cell halo, and in x one more column on the left so that the
// tile's first column bx0 - 4 is 16-byte aligned (TMA); own-tile cell (ci, cj)
// is raw (ci + OXR, cj + OYR)
constexpr int RX = TX + 8, RY = TY + 6;
constexpr int OXR = 4, OYR = 3;
constexpr int LX = TX + 4, LY = TY + 4;  // flags and modified moments, 2-cell halo
constexpr unsigned kTmaPolls = 1u << 20;  // mbarrier polls before a tile copy is given up
static_assert(TX * TY == NT, "one own cell per thread");

template <typename R, int C, int NG, bool COMP = false>
struct Smem2D {
  static constexpr int kPadX = 1;  // raw index of flag-grid column lx: lx + 2
  // the limiter's results go to `lim` by work-list slot (and are written into
  // u once every cell's flag and limiter has read the raw moments)
  static constexpr bool kLimList = true;
  // stage input (the TMA box); after Step 4 its first moments are the
  // modified ones
  alignas(128) R u[C][3][RY][RX];
  // HWENO_FP32C: the low parts of the stage input's averages (a second box)
  alignas(128) R ulo[COMP ? C : 1][COMP ? RY : 1][COMP ? RX : 1];
  R lim[C == 4 ? LX * LY : 1][C][2];  // Euler: modified x-, y-moments by list slot
  R xf[C][2 * NG][TY][TX + 2];  // x-face values (left NG, right NG) of cells -1..TX
  R yf[C][2 * NG][TY + 2][TX];  // y-face values (bottom NG, top NG) of cells -1..TY
  uint8_t fl[LY][LX];
  R red[2][NW];
  int cnt[NW];
  R amax[2][NW];
  unsigned long long bar;                        // mbarrier of the tile copy
  int ntb, nhw;                                  // lengths of the two work lists
  unsigned short tbl[LX * LY];                   // troubled cells (Euler limiter)
  unsigned short hwl[TX * TY + 2 * TX + 2 * TY]; // interface items with HWENO
};

// --------------------------------------------------------- KXRCF (2D)
// Reading: I = |dy jx + dx jy| / (h (dx + dy) max(|u0|, 1e-12)), h =
// sqrt(dx^2 + dy^2)/2, jx / jy the degree-1 trace jumps across the inflow x-
// and y-faces (left / bottom when the velocity component is >= 0).

__device__ __forceinline__ double jump64(double u0, double v0, double unb, double vnb, bool low) {
  return low ? __dsub_rn(__dsub_rn(u0, __dmul_rn(6.0, v0)), __dadd_rn(unb, __dmul_rn(6.0, vnb)))
             : __dsub_rn(__dadd_rn(u0, __dmul_rn(6.0, v0)), __dsub_rn(unb, __dmul_rn(6.0, vnb)));
}

// u0/v0/w0 the cell, (uxn, vxn) its inflow x-neighbour, (uyn, wyn) its inflow
// y-neighbour; lowx / lowy: the inflow faces are the left / bottom ones.
// FP32 data: decide in FP32 when the rounding-error bound allows, else with
// float pairs (no FP64 on the FP32 kernel's path): the two jumps as exact-to-
// ~2^-46 pairs (jump_pair), num = dy jx + dx jy from pair products (fma gives
// each product's rounding error; dx and dy carry their own low parts), and the
// threshold thr den_h max(|u0|, 1e-12) as a pair; the sign of |num| - r is then
// that of the exact values unless they agree to ~1e-13 of dy S_x + dx S_y,
// far inside the 1e-6 band around the threshold.
__device__ __forceinline__ bool kxrcf2_troubled(float u0, float v0, float w0, float uxn, float vxn,
                                                float uyn, float wyn, bool lowx, bool lowy,
                                                const Kx2& k) {
  const float jx = lowx ? (u0 - 6.0f * v0) - (uxn + 6.0f * vxn) : (u0 + 6.0f * v0) - (uxn - 6.0f * vxn);
  const float jy = lowy ? (u0 - 6.0f * w0) - (uyn + 6.0f * wyn) : (u0 + 6.0f * w0) - (uyn - 6.0f * wyn);
  const float sx = fabsf(u0) + 6.0f * fabsf(v0) + fabsf(uxn) + 6.0f * fabsf(vxn);
  const float sy = fabsf(u0) + 6.0f * fabsf(w0) + fabsf(uyn) + 6.0f * fabsf(wyn);
  const float num = fabsf(k.fdy * jx + k.fdx * jy);
  // |num - exact| <= 2^-24 (3 dy sx + 3 dx sy + 3 |num|) to first order
  const float e = 1.0e-6f * (k.fdy * sx + k.fdx * sy);
  const float nrm = fmaxf(fabsf(u0), 1e-12f);
  const float r = k.fthr_den * nrm;
  if (num - e > r * (1.0f + 4.8e-7f)) return true;
  if (num + e < r * (1.0f - 4.8e-7f)) return false;
  float jxh, jxl, jyh, jyl;
  jump_pair(u0, v0, uxn, vxn, lowx, jxh, jxl);
  jump_pair(u0, w0, uyn, wyn, lowy, jyh, jyl);
  const float p1h = __fmul_rn(k.fdy, jxh);
  const float p1l = __fadd_rn(fmaf(k.fdy, jxh, -p1h),
                              __fadd_rn(__fmul_rn(k.fdy, jxl), __fmul_rn(k.fdy_lo, jxh)));
  const float p2h = __fmul_rn(k.fdx, jyh);
  const float p2l = __fadd_rn(fmaf(k.fdx, jyh, -p2h),
                              __fadd_rn(__fmul_rn(k.fdx, jyl), __fmul_rn(k.fdx_lo, jyh)));
  float nh, nl, t;
  two_sum(p1h, p2h, nh, t);
  two_sum(nh, __fadd_rn(t, __fadd_rn(p1l, p2l)), nh, nl);
  if (nh < 0.0f) {
    nh = -nh;
    nl = -nl;
  }
  const float rh = __fmul_rn(nrm, k.fthr_den);
  const float rl = __fadd_rn(fmaf(nrm, k.fthr_den, -rh), __fmul_rn(nrm, k.fthr_den_lo));
  return __fadd_rn(__fsub_rn(nh, rh), __fsub_rn(nl, rl)) > 0.0f;
}

// FP64 data: the decision of the reading, |dy jx + dx jy| / (den_h nrm) >
// thr, in its divide-free product form (it differs from the quotient form only
// within a few ulp of the threshold).
__device__ __forceinline__ bool kxrcf2_troubled(double u0, double v0, double w0, double uxn,
                                                double vxn, double uyn, double wyn, bool lowx,
                                                bool lowy, const Kx2& k) {
  const double jx = jump64(u0, v0, uxn, vxn, lowx);
  const double jy = jump64(u0, w0, uyn, wyn, lowy);
  const double num = __dadd_rn(__dmul_rn(k.dy, jx), __dmul_rn(k.dx, jy));
  const double nrm = fmax(fabs(u0), 1e-12);
  return fabs(num) > __dmul_rn(k.thr, __dmul_rn(k.den_h, nrm));
}

// Float-pair averages (HWENO_FP32C: u0 + l0, uxn + lxn, uyn + lyn), in three
// tiers: the FP32 fast test on hi (its margins exceed what the low parts can
// change, below 2^-24 of the averages); where it cannot decide, the float-pair
// form of the FP32 kernel with the low parts added in (jump_pair_lo; the norm
// |u0 + l0| as a pair), decided when the difference clears 1e-12 (dy S_x + dx
// S_y + r), far above its rounding bound; and only inside that margin the FP64
// form on hi + lo.  The decision is the oracle's on the same state except
// within a few FP64 ulp of the threshold.
__device__ __forceinline__ bool kxrcf2_troubled_pair(float u0, float l0, float v0, float w0,
                                                     float uxn, float lxn, float vxn, float uyn,
                                                     float lyn, float wyn, bool lowx, bool lowy,
                                                     const Kx2& k) {
  const float jx = lowx ? (u0 - 6.0f * v0) - (uxn + 6.0f * vxn) : (u0 + 6.0f * v0) - (uxn - 6.0f * vxn);
  const float jy = lowy ? (u0 - 6.0f * w0) - (uyn + 6.0f * wyn) : (u0 + 6.0f * w0) - (uyn - 6.0f * wyn);
  const float sx = fabsf(u0) + 6.0f * fabsf(v0) + fabsf(uxn) + 6.0f * fabsf(vxn);
  const float sy = fabsf(u0) + 6.0f * fabsf(w0) + fabsf(uyn) + 6.0f * fabsf(wyn);
  const float num = fabsf(k.fdy * jx + k.fdx * jy);
  const float e = 1.0e-6f * (k.fdy * sx + k.fdx * sy);
  const float r = k.fthr_den * fmaxf(fabsf(u0), 1e-12f);
  if (num - e > r * (1.0f + 4.8e-7f)) return true;
  if (num + e < r * (1.0f - 4.8e-7f)) return false;
  float jxh, jxl, jyh, jyl;
  jump_pair_lo(u0, l0, v0, uxn, lxn, vxn, lowx, jxh, jxl);
  jump_pair_lo(u0, l0, w0, uyn, lyn, wyn, lowy, jyh, jyl);
  const float p1h = __fmul_rn(k.fdy, jxh);
  const float p1l = __fadd_rn(fmaf(k.fdy, jxh, -p1h),
                              __fadd_rn(__fmul_rn(k.fdy, jxl), __fmul_rn(k.fdy_lo, jxh)));
  const float p2h = __fmul_rn(k.fdx, jyh);
  const float p2l = __fadd_rn(fmaf(k.fdx, jyh, -p2h),
                              __fadd_rn(__fmul_rn(k.fdx, jyl), __fmul_rn(k.fdx_lo, jyh)));
  float mh, ml, t;
  two_sum(p1h, p2h, mh, t);
  two_sum(mh, __fadd_rn(t, __fadd_rn(p1l, p2l)), mh, ml);
  if (mh < 0.0f) {
    mh = -mh;
    ml = -ml;
  }
  float nh = fabsf(u0), nl = u0 < 0.0f ? -l0 : l0;
  if (nh < 1e-12f) {
    nh = 1e-12f;
    nl = 0.0f;
  }
  const float rh = __fmul_rn(nh, k.fthr_den);
  const float rl = __fadd_rn(fmaf(nh, k.fthr_den, -rh),
                             __fadd_rn(__fmul_rn(nh, k.fthr_den_lo), __fmul_rn(nl, k.fthr_den)));
  const float d = __fadd_rn(__fsub_rn(mh, rh), __fsub_rn(ml, rl));
  if (fabsf(d) > 1e-12f * (k.fdy * sx + k.fdx * sy + r)) return d > 0.0f;
  return kxrcf2_troubled((double)u0 + (double)l0, (double)v0, (double)w0, (double)uxn + (double)lxn,
                         (double)vxn, (double)uyn + (double)lyn, (double)wyn, lowx, lowy, k);
}

// The 19 data of component c of the cell at own-tile coordinates (ci, cj):
// ubar of cells 1..9, vbar and wbar (modified: read after Step 4) of cells
// 2, 4, 5, 6, 8.
template <typename S, typename R>
__device__ __forceinline__ void gather19(const S& sm, int c, int ci, int cj, R* d) {
#pragma unroll
  for (int k = 0; k < 9; ++k) d[k] = sm.u[c][0][cj + OYR + k / 3 - 1][ci + OXR + k % 3 - 1];
  const int mx[5] = {0, -1, 0, 1, 0}, my[5] = {-1, 0, 0, 0, 1};
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    d[9 + k] = sm.u[c][1][cj + OYR + my[k]][ci + OXR + mx[k]];
    d[14 + k] = sm.u[c][2][cj + OYR + my[k]][ci + OXR + mx[k]];
  }
}

// The 19 data as gather19 gives them, or (COMP: the float-pair averages of
// HWENO_FP32C) with the 9 averages as increments over the cell's own hi, low
// parts included: the p0 and HWENO maps are consistent (their average
// coefficients sum to one, their smoothness indicators are differences), so
// they map these increments to the point values' increments over hi.
template <bool COMP, typename S, typename R>
__device__ __forceinline__ void gather_data(const S& sm, int c, int ci, int cj, R* d) {
  gather19(sm, c, ci, cj, d);
  if constexpr (COMP) {
    const R b = d[4];
#pragma unroll
    for (int k = 0; k < 9; ++k)
      d[k] = __fadd_rn(__fsub_rn(d[k], b), sm.ulo[c][cj + OYR + k / 3 - 1][ci + OXR + k % 3 - 1]);
  }
}

// Value v of point p (order of hweno2d_coef.cuh) of component c of the cell at
// own-tile coordinates (ci, cj) into the face arrays.
template <typename S, typename R>
__device__ __forceinline__ void store_point(S& sm, int c, int p, int ci, int cj, R v) {
  constexpr int NG2 = sizeof(sm.xf[0]) / sizeof(sm.xf[0][0]);  // 2 NG
  if (p < NG2)
    sm.xf[c][p][cj][ci + 1] = v;        // left and right faces
  else
    sm.yf[c][p - NG2][cj + 1][ci] = v;  // bottom and top faces
}

// Step 5.1 for an Euler cell whose 3x3 stencil holds a troubled cell: the
// interface points [p_lo, p_hi) by HWENO in the x (x-faces) and y (y-faces)
// characteristic fields of the cell average (Remark 4).  Rare: out of line.
template <int NG, bool COMP, typename S, typename R>
__device__ __noinline__ void hweno_faces_euler2d(S& sm, int ci, int cj, int p_lo, int p_hi, R g0,
                                                 R g1, R g2, R g3, R g4, R eps, R gas,
                                                 bool mean_eigen) {
  constexpr int NF = 4 * NG;
  const R gam[5] = {g0, g1, g2, g3, g4};  // by value: no caller array on the stack
  R Uc[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) Uc[c] = sm.u[c][0][cj + OYR][ci + OXR];
  // one eigen-system per direction (the cell average), or with mean_eigen one
  // per face (the mean of the averages on its two sides): "parts" of the
  // direction's 2 NG points
  const int nparts = mean_eigen ? 2 : 1;
#pragma unroll 1
  for (int q = 0; q < 2 * nparts; ++q) {
    const int dir = q / nparts, side = q % nparts;
    const int lo = dir * 2 * NG + side * NG, hi = lo + 2 * NG / nparts;
    const int plo = p_lo > lo ? p_lo : lo, phi = p_hi < hi ? p_hi : hi;
    if (plo >= phi) continue;
    R U[4];
    if (!mean_eigen) {
#pragma unroll
      for (int c = 0; c < 4; ++c) U[c] = Uc[c];
    } else {
      const int dx = dir == 0 ? 2 * side - 1 : 0, dy = dir == 1 ? 2 * side - 1 : 0;
#pragma unroll
      for (int c = 0; c < 4; ++c) U[c] = R(0.5) * (Uc[c] + sm.u[c][0][cj + OYR + dy][ci + OXR + dx]);
    }
    R Rm[4][4], Lm[4][4];
    Euler2D<R>::eigen(gas, U, dir, Rm, Lm);
    R acc[4][NF];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int p = 0; p < NF; ++p) acc[c][p] = R(0);
    if constexpr (sizeof(R) == 4) {
      // FP32: the fields in pairs (f, f + 1) through the packed HWENO
      // helpers, the stencil data of each component gathered once per pair
#pragma unroll
      for (int f = 0; f < 4; f += 2) {
        float2 e2[19];
#pragma unroll
        for (int k = 0; k < 19; ++k) e2[k] = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          R t[19];
          gather_data<COMP>(sm, c, ci, cj, t);
#pragma unroll
          for (int k = 0; k < 19; ++k) {
            e2[k].x += Lm[f][c] * t[k];
            e2[k].y += Lm[f + 1][c] * t[k];
          }
        }
        float2 chv2[NF];
        hweno2d_faces_x2<NG>(e2, gam, eps, plo, phi, chv2);
#pragma unroll
        for (int p = 0; p < NF; ++p)
          if (p >= plo && p < phi)
#pragma unroll
            for (int c = 0; c < 4; ++c)
              acc[c][p] += Rm[c][f] * chv2[p].x + Rm[c][f + 1] * chv2[p].y;
      }
    } else {
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        R e[19], t[19];
#pragma unroll
        for (int k = 0; k < 19; ++k) e[k] = R(0);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          gather_data<COMP>(sm, c, ci, cj, t);
#pragma unroll
          for (int k = 0; k < 19; ++k) e[k] += Lm[f][c] * t[k];
        }
        R chv[NF];
        hweno2d_faces<NG>(e, gam, eps, plo, phi, chv);
#pragma unroll
        for (int p = 0; p < NF; ++p)
          if (p >= plo && p < phi)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[c][p] += Rm[c][f] * chv[p];
      }
    }
#pragma unroll
    for (int p = 0; p < NF; ++p)
      if (p >= plo && p < phi)
#pragma unroll
        for (int c = 0; c < 4; ++c) store_point(sm, c, p, ci, cj, acc[c][p]);
  }
}

template <typename R, int C, int NG, bool COMP>
__global__ void __launch_bounds__(NT, (sizeof(R) == 4 ? 2 : 1))
    stage2d_kernel(Stage2DArgs a, const __grid_constant__ CUtensorMap tile_map,
                   const __grid_constant__ CUtensorMap lo_map) {
  static_assert(!COMP || sizeof(R) == 4, "the float-pair averages are FP32");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  using SM = Smem2D<R, C, NG, COMP>;
  SM& sm = *reinterpret_cast<SM*>(smem_raw);
  constexpr int NF = 4 * NG, NI = NG * NG;
  // FP32 Euler: the linear p0 maps take two components at once (packed FP32)
  constexpr bool kPacked = C == 4 && sizeof(R) == 4;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nx = a.nx, ny = a.ny;
  const int bx0 = blockIdx.x * TX, by0 = blockIdx.y * TY;
  const size_t plane = (size_t)nx * ny;
  const R* __restrict__ w = static_cast<const R*>(a.w);

  asm volatile("griddepcontrol.wait;" ::: "memory");
  // Tiles whose halo lies inside the grid are copied by one TMA box (all 3 C
  // planes, RX x RY cells from (bx0 - 4, by0 - 3)); the others (periodic or
  // wall ghosts) by the threads, through the boundary map.
  const bool tma = a.tma && bx0 >= OXR && bx0 - OXR + RX <= nx && by0 >= OYR &&
                   by0 - OYR + RY <= ny;
  if (tma && threadIdx.x == 0) {
    mbar_init(&sm.bar, 1);
    mbar_expect_tx(&sm.bar, (unsigned)(sizeof(sm.u) + (COMP ? sizeof(sm.ulo) : 0)));
    tma_load_3d(&sm.u[0][0][0][0], &tile_map, &sm.bar, bx0 - OXR, by0 - OYR, 0);
    if constexpr (COMP) tma_load_3d(&sm.ulo[0][0][0], &lo_map, &sm.bar, bx0 - OXR, by0 - OYR, 0);
  }

  R gam[5], eps, gas, inv_dx, inv_dy;
  if constexpr (sizeof(R) == 4) {
#pragma unroll
    for (int k = 0; k < 5; ++k) gam[k] = a.f32[k];
    eps = a.f32[5]; gas = a.f32[6]; inv_dx = a.f32[7]; inv_dy = a.f32[8];
  } else {
#pragma unroll
    for (int k = 0; k < 5; ++k) gam[k] = a.gam[k];
    eps = a.eps; gas = a.gas; inv_dx = a.inv_dx; inv_dy = a.inv_dy;
  }

  // ---- 1. alpha_x, alpha_y, the time bookkeeping, the tile and its halo
  const R* a_in = static_cast<const R*>(a.a_in);
  R ax = R(0), ay = R(0);
  for (int k = tid; k < a.nin; k += NT) {
    ax = fmax(ax, a_in[k]);
    ay = fmax(ay, a_in[a.nin + k]);
  }
  // dt of the step: formed in FP64 by dt2d_kernel before stage 1
  R dt_prev = R(0);
  if (a.stage > 0) dt_prev = sc_dt<R>(a.sc);
  const int ox = tid % TX, oy = tid / TX;  // own cell of this thread
  const int gi = bx0 + ox, gj = by0 + oy;
  const bool own = gi < nx && gj < ny;
  // u^n of the own cell (stages 2 and 3): brought into L2 now and loaded in
  // phase 4, so that no registers hold it through phases 2 and 3
  if (a.stage >= 2 && own) {
    const R* u0 = static_cast<const R*>(a.u0);
#pragma unroll
    for (int c = 0; c < C; ++c) {
#pragma unroll
      for (int m = 0; m < 3; ++m)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(u0 + (3 * c + m) * plane + (size_t)gj * nx + gi));
      if constexpr (COMP)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(a.u0_lo + c * plane + (size_t)gj * nx + gi));
    }
  }
  if (!tma) {
    for (int k = tid; k < RX * RY; k += NT) {
      const int rx = k % RX, ry = k / RX;
      const int si = bc_map(bx0 - OXR + rx, nx, a.bc), sj = bc_map(by0 - OYR + ry, ny, a.bc);
      const size_t s = (size_t)sj * nx + si;
#pragma unroll
      for (int c = 0; c < C; ++c) {
#pragma unroll
        for (int m = 0; m < 3; ++m) sm.u[c][m][ry][rx] = w[(3 * c + m) * plane + s];
        if constexpr (COMP) sm.ulo[c][ry][rx] = a.w_lo[c * plane + s];
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    ax = fmax(ax, __shfl_xor_sync(0xffffffffu, ax, o));
    ay = fmax(ay, __shfl_xor_sync(0xffffffffu, ay, o));
  }
  if (lane == 0) {
    sm.amax[0][warp] = ax;
    sm.amax[1][warp] = ay;
  }
  if (tid == 0) sm.ntb = sm.nhw = 0;
  __syncthreads();
  if (tma && !mbar_wait_bounded(&sm.bar, 0, kTmaPolls)) {
    // the copy did not land: flag the stage (the host reports
    // HWENO_ERR_TIMEOUT) and give the copy, which writes this CTA's shared
    // memory, a second bounded wait; no thread leaves the common path
    atomicOr(&a.sc->status, ST_TIMEOUT);
    mbar_wait_bounded(&sm.bar, 0, kTmaPolls);
  }
  asm volatile("griddepcontrol.launch_dependents;");
  R alx = sm.amax[0][0], aly = sm.amax[1][0];
#pragma unroll
  for (int k = 1; k < NW; ++k) {
    alx = fmax(alx, sm.amax[0][k]);
    aly = fmax(aly, sm.amax[1][k]);
  }
  if (a.alpha_in) {  // replay: the recorded values (what the reduction gave)
    alx = static_cast<const R*>(a.alpha_in)[0];
    aly = static_cast<const R*>(a.alpha_in)[1];
  }
  R dt = dt_prev;
  if (a.stage == 1) {
    if (a.dt_in) {  // replay of a recorded step
      dt = *static_cast<const R*>(a.dt_in);
      if (blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) {
        a.sc->dt = (double)dt;
        a.sc->dt_f = (float)dt;
        a.sc->last = 0u;
      }
    }
    if (a.rec_dt && blockIdx.x == 0 && blockIdx.y == 0 && tid == 0)
      *static_cast<R*>(a.rec_dt) = dt;
  }
  if (a.rec_alpha && blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) {
    static_cast<R*>(a.rec_alpha)[0] = alx;
    static_cast<R*>(a.rec_alpha)[1] = aly;
  }
  if (a.stage > 0 && !(dt > R(0))) return;  // uniform over the grid
  if (a.a_zero && blockIdx.x == 0 && blockIdx.y == 0 && tid < 2 * kAlphaSlots)
    static_cast<R*>(a.a_zero)[tid] = R(0);

  // ---- 2. Step 4 on the tile plus 2 halo cells; the modified first moments
  // of the troubled cells replace the raw ones in the tile only after every
  // flag and limiter has read the raw ones
  static_assert(LX * LY <= 2 * NT, "two cells of Step 4 per thread at most");
  R hv[2][2];       // Burgers: the modified moments of this thread's troubled cells
  int hk[2] = {-1, -1};
  int it = 0;
  for (int k = tid; k < LX * LY; k += NT, ++it) {
    const int lx = k % LX, ly = k / LX;
    const int rx = lx + 1 + SM::kPadX, ry = ly + 1;  // raw index of the cell
    int flag;
    if (a.flags_in) {  // replay: the recorded decision (periodic: a ghost's is its image's)
      flag = a.flags_in[(size_t)bc_map(by0 - 2 + ly, ny, a.bc) * nx + bc_map(bx0 - 2 + lx, nx, a.bc)] != 0;
    } else if (a.mode == 1) {
      flag = 1;
    } else if (a.mode == 2) {
      flag = 0;
    } else {
      bool lowx, lowy;
      if constexpr (C == 1) {
        lowx = lowy = sm.u[0][0][ry][rx] >= R(0);
      } else {
        lowx = inflow_left(sm.u[0][0][ry][rx], sm.u[1][0][ry][rx]);
        lowy = inflow_left(sm.u[0][0][ry][rx], sm.u[2][0][ry][rx]);
      }
      const int nxx = lowx ? rx - 1 : rx + 1, nyy = lowy ? ry - 1 : ry + 1;
      const int ci = 0;
      if constexpr (COMP) {  // on hi + lo
        flag = kxrcf2_troubled_pair(sm.u[ci][0][ry][rx], sm.ulo[ci][ry][rx], sm.u[ci][1][ry][rx],
                                    sm.u[ci][2][ry][rx], sm.u[ci][0][ry][nxx], sm.ulo[ci][ry][nxx],
                                    sm.u[ci][1][ry][nxx], sm.u[ci][0][nyy][rx], sm.ulo[ci][nyy][rx],
                                    sm.u[ci][2][nyy][rx], lowx, lowy, a.kx);
        if constexpr (C == 4)
          flag = flag || kxrcf2_troubled_pair(sm.u[3][0][ry][rx], sm.ulo[3][ry][rx],
                                              sm.u[3][1][ry][rx], sm.u[3][2][ry][rx],
                                              sm.u[3][0][ry][nxx], sm.ulo[3][ry][nxx],
                                              sm.u[3][1][ry][nxx], sm.u[3][0][nyy][rx],
                                              sm.ulo[3][nyy][rx], sm.u[3][2][nyy][rx], lowx,
                                              lowy, a.kx);
      } else {
        flag = kxrcf2_troubled(sm.u[ci][0][ry][rx], sm.u[ci][1][ry][rx], sm.u[ci][2][ry][rx],
                               sm.u[ci][0][ry][nxx], sm.u[ci][1][ry][nxx], sm.u[ci][0][nyy][rx],
                               sm.u[ci][2][nyy][rx], lowx, lowy, a.kx);
        if constexpr (C == 4) {
          flag = flag || kxrcf2_troubled(sm.u[3][0][ry][rx], sm.u[3][1][ry][rx], sm.u[3][2][ry][rx],
                                         sm.u[3][0][ry][nxx], sm.u[3][1][ry][nxx],
                                         sm.u[3][0][nyy][rx], sm.u[3][2][nyy][rx], lowx, lowy, a.kx);
        }
      }
    }
    sm.fl[ly][lx] = (uint8_t)flag;
    if constexpr (C == 1) {
      if (flag) {
        hk[it] = k;
        hv[it][0] = limit_first_moment(sm.u[0][0][ry][rx - 1], sm.u[0][0][ry][rx],
                                       sm.u[0][0][ry][rx + 1], sm.u[0][1][ry][rx - 1],
                                       sm.u[0][1][ry][rx + 1], gam, eps);
        hv[it][1] = limit_first_moment(sm.u[0][0][ry - 1][rx], sm.u[0][0][ry][rx],
                                       sm.u[0][0][ry + 1][rx], sm.u[0][2][ry - 1][rx],
                                       sm.u[0][2][ry + 1][rx], gam, eps);
      }
    }
    // Euler: the troubled cells are listed and limited by consecutive threads
    // below, so a warp holding one or two of them does not run the
    // characteristic limiter for its other lanes' sake
    if constexpr (C == 4) list_append(&sm.ntb, sm.tbl, k, flag != 0, LX * LY);
  }
  // the tile's flag grid holds a troubled cell (uniform over the CTA): else
  // no interface item of the tile needs HWENO and none tests its stencil
  bool tile_troubled;
  if constexpr (C == 1) {
    tile_troubled = __syncthreads_or(hk[0] >= 0 || hk[1] >= 0);
    if (tile_troubled) {
#pragma unroll
      for (int j = 0; j < 2; ++j)
        if (hk[j] >= 0) {
          const int rx = hk[j] % LX + 1 + SM::kPadX, ry = hk[j] / LX + 1;
          sm.u[0][1][ry][rx] = hv[j][0];
          sm.u[0][2][ry][rx] = hv[j][1];
        }
      __syncthreads();
    }
  } else {
    __syncthreads();
    tile_troubled = sm.ntb > 0;
    if (tile_troubled) {
      for (int q = tid; q < sm.ntb; q += NT) {
        const int k = sm.tbl[q];
        limit_euler2d(sm, k % LX, k / LX, q, gam[0], gam[1], gam[2], gam[3], gam[4], eps, gas);
      }
      __syncthreads();
      for (int q = tid; q < sm.ntb; q += NT) {
        const int k = sm.tbl[q];
        const int rx = k % LX + 1 + SM::kPadX, ry = k / LX + 1;
#pragma unroll
        for (int c = 0; c < C; ++c) {
          sm.u[c][1][ry][rx] = sm.lim[q][c][0];
          sm.u[c][2][ry][rx] = sm.lim[q][c][1];
        }
      }
      __syncthreads();
    }
  }

  // ---- 3. interface values of the own cells (all faces) and of the cross
  //         halo (left column: right face, right column: left face, bottom
  //         row: top face, top row: bottom face)
  //         by linear p0; the items whose stencil holds a troubled cell are
  //         listed and reconstructed by HWENO on consecutive threads below
  //         (the same arithmetic, fewer warps diverging on it)
  auto item_of = [](int item, int& ci, int& cj, int& p_lo, int& p_hi) {
    if (item < TX * TY) {  // own cell: every interface point
      ci = item % TX; cj = item / TX; p_lo = 0; p_hi = NF;
    } else {               // cross halo: the one face shared with the tile
      const int h = item - TX * TY;
      if (h < TY) { ci = -1; cj = h; p_lo = NG; p_hi = 2 * NG; }
      else if (h < 2 * TY) { ci = TX; cj = h - TY; p_lo = 0; p_hi = NG; }
      else if (h < 2 * TY + TX) { ci = h - 2 * TY; cj = -1; p_lo = 3 * NG; p_hi = 4 * NG; }
      else { ci = h - 2 * TY - TX; cj = TY; p_lo = 2 * NG; p_hi = 3 * NG; }
    }
  };
  for (int item = tid; item < TX * TY + 2 * TX + 2 * TY; item += NT) {
    int ci, cj, p_lo, p_hi;  // own-tile coordinates of the cell, point range
    item_of(item, ci, cj, p_lo, p_hi);
    bool hw = false;
    if (tile_troubled) {
#pragma unroll
      for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
        for (int di = -1; di <= 1; ++di) hw |= sm.fl[cj + 2 + dj][ci + 2 + di] != 0;
    }
    if (!hw) {
      if constexpr (kPacked) {
        // FP32 Euler: components (0, 1) and (2, 3) through the packed map
#pragma unroll
        for (int c = 0; c < C; c += 2) {
          R da[19], db[19];
          gather_data<COMP>(sm, c, ci, cj, da);
          gather_data<COMP>(sm, c + 1, ci, cj, db);
          float2 d2[19], v2[NF];
#pragma unroll
          for (int k = 0; k < 19; ++k) d2[k] = make_float2(da[k], db[k]);
          p0_faces_x2<NG>(d2, v2);
#pragma unroll
          for (int p = 0; p < NF; ++p)
            if (p >= p_lo && p < p_hi) {
              store_point(sm, c, p, ci, cj, v2[p].x);
              store_point(sm, c + 1, p, ci, cj, v2[p].y);
            }
        }
      } else {
#pragma unroll
        for (int c = 0; c < C; ++c) {
          R d[19], v[NF];
          gather_data<COMP>(sm, c, ci, cj, d);
          p0_faces<NG>(d, v);
#pragma unroll
          for (int p = 0; p < NF; ++p)
            if (p >= p_lo && p < p_hi) store_point(sm, c, p, ci, cj, v[p]);
        }
      }
    }
    list_append(&sm.nhw, sm.hwl, item, hw, TX * TY + 2 * TX + 2 * TY);
  }
  __syncthreads();
  if (sm.nhw > 0) {  // uniform over the CTA
    for (int q = tid; q < sm.nhw; q += NT) {
      int ci, cj, p_lo, p_hi;
      item_of(sm.hwl[q], ci, cj, p_lo, p_hi);
      if constexpr (C == 1) {
        R d[19], v[NF];
        gather_data<COMP>(sm, 0, ci, cj, d);
        hweno2d_faces<NG>(d, gam, eps, p_lo, p_hi, v);
#pragma unroll
        for (int p = 0; p < NF; ++p)
          if (p >= p_lo && p < p_hi) store_point(sm, 0, p, ci, cj, v[p]);
      } else {
        hweno_faces_euler2d<NG, COMP>(sm, ci, cj, p_lo, p_hi, gam[0], gam[1], gam[2], gam[3],
                                      gam[4], eps, gas, (a.variant & HWENO_VARIANT_MEAN_EIGEN) != 0);
      }
    }
    __syncthreads();
  }

  // ---- 4. own cells: interior points, fluxes, Eq. (ode2), Eq. (RK)
  constexpr double r15 = 0.38729833462074168852;  // sqrt(15)/10
  constexpr double r3 = 0.28867513459481288225;   // sqrt(3)/6
  const R gw[3] = {NG == 3 ? R(5.0 / 18.0) : R(0.5), NG == 3 ? R(4.0 / 9.0) : R(0.5), R(5.0 / 18.0)};
  const R gx[3] = {NG == 3 ? R(-r15) : R(-r3), NG == 3 ? R(0) : R(r3), R(r15)};
  const int ci = ox, cj = oy;
  int myflag = 0;
  R spx = R(0), spy = R(0);
  unsigned bad = 0;
  {
    R u0c[C][3], u0l[C];
    if (a.stage >= 2 && own) {
      const R* u0 = static_cast<const R*>(a.u0);
#pragma unroll
      for (int c = 0; c < C; ++c) {
#pragma unroll
        for (int m = 0; m < 3; ++m) u0c[c][m] = u0[(3 * c + m) * plane + (size_t)gj * nx + gi];
        if constexpr (COMP) u0l[c] = a.u0_lo[c * plane + (size_t)gj * nx + gi];
      }
    }
    myflag = sm.fl[cj + 2][ci + 2];
    const R hax = R(0.5) * alx, hay = R(0.5) * aly;
    // COMP: every point value is an increment over the own cell's hi B, every
    // flux an increment over f(B) (the base cancels from Eq. (ode2) exactly)
    R B[C];
#pragma unroll
    for (int c = 0; c < C; ++c) B[c] = sm.u[c][0][cj + OYR][ci + OXR];
    auto flux = [&](const R* U, int dir, R* F) {
      if constexpr (COMP) flux_inc2<C>(gas, B, U, dir, F);
      else phys_flux2<R, C>(gas, U, dir, F);
    };
    // COMP: a neighbour's face value, held over its own hi, over B instead
    auto rebase = [&](R* v, int dx, int dy) {
      if constexpr (COMP) {
#pragma unroll
        for (int c = 0; c < C; ++c)
          v[c] = __fadd_rn(v[c], __fsub_rn(sm.u[c][0][cj + OYR + dy][ci + OXR + dx], B[c]));
      }
    };
    R Fv[C], Gv[C];
#pragma unroll
    for (int c = 0; c < C; ++c) Fv[c] = Gv[c] = R(0);
    R inter[C][NI];
    if constexpr (kPacked) {
#pragma unroll
      for (int c = 0; c < C; c += 2) {
        R da[19], db[19];
        gather_data<COMP>(sm, c, ci, cj, da);
        gather_data<COMP>(sm, c + 1, ci, cj, db);
        float2 d2[19], i2[NI];
#pragma unroll
        for (int k = 0; k < 19; ++k) d2[k] = make_float2(da[k], db[k]);
        p0_interior_x2<NG>(d2, i2);
#pragma unroll
        for (int l = 0; l < NI; ++l) {
          inter[c][l] = i2[l].x;
          inter[c + 1][l] = i2[l].y;
        }
      }
    } else {
#pragma unroll
      for (int c = 0; c < C; ++c) {
        R d[19];
        gather_data<COMP>(sm, c, ci, cj, d);
        p0_interior<NG>(d, inter[c]);
      }
    }
    // the volume integrals of Eq. (ode2) at interior point p (weight
    // gw[p % NG] gw[p / NG])
    auto interior_point = [&](int p) {
      R U[C], f[C], g[C];
#pragma unroll
      for (int c = 0; c < C; ++c) U[c] = inter[c][p];
      flux(U, 0, f);
      flux(U, 1, g);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        Fv[c] += gw[p % NG] * gw[p / NG] * f[c];
        Gv[c] += gw[p % NG] * gw[p / NG] * g[c];
      }
    };
    R sfx[C], sfs[C], sfxe[C], sgy[C], sgs[C], sgyx[C];
#pragma unroll
    for (int c = 0; c < C; ++c) sfx[c] = sfs[c] = sfxe[c] = sgy[c] = sgs[c] = sgyx[c] = R(0);
    // the Lax-Friedrichs fluxes of the four faces at Gauss point k and their
    // weighted sums
    auto face_point = [&](int k) {
      R am[C], ap[C], fa[C], fb[C], FLk[C], FRk[C], GBk[C], GTk[C];
      // x_{i-1/2}: u^- = right face of cell i-1, u^+ = own left face
#pragma unroll
      for (int c = 0; c < C; ++c) { am[c] = sm.xf[c][NG + k][cj][ci]; ap[c] = sm.xf[c][k][cj][ci + 1]; }
      rebase(am, -1, 0);
      flux(am, 0, fa); flux(ap, 0, fb);
#pragma unroll
      for (int c = 0; c < C; ++c) FLk[c] = R(0.5) * (fa[c] + fb[c]) - hax * (ap[c] - am[c]);
      // x_{i+1/2}: u^- = own right face, u^+ = left face of cell i+1
#pragma unroll
      for (int c = 0; c < C; ++c) { am[c] = sm.xf[c][NG + k][cj][ci + 1]; ap[c] = sm.xf[c][k][cj][ci + 2]; }
      rebase(ap, 1, 0);
      flux(am, 0, fa); flux(ap, 0, fb);
#pragma unroll
      for (int c = 0; c < C; ++c) FRk[c] = R(0.5) * (fa[c] + fb[c]) - hax * (ap[c] - am[c]);
      // y_{j-1/2}: u^- = top face of cell j-1, u^+ = own bottom face
#pragma unroll
      for (int c = 0; c < C; ++c) { am[c] = sm.yf[c][NG + k][cj][ci]; ap[c] = sm.yf[c][k][cj + 1][ci]; }
      rebase(am, 0, -1);
      flux(am, 1, fa); flux(ap, 1, fb);
#pragma unroll
      for (int c = 0; c < C; ++c) GBk[c] = R(0.5) * (fa[c] + fb[c]) - hay * (ap[c] - am[c]);
      // y_{j+1/2}: u^- = own top face, u^+ = bottom face of cell j+1
#pragma unroll
      for (int c = 0; c < C; ++c) { am[c] = sm.yf[c][NG + k][cj + 1][ci]; ap[c] = sm.yf[c][k][cj + 2][ci]; }
      rebase(ap, 0, 1);
      flux(am, 1, fa); flux(ap, 1, fb);
#pragma unroll
      for (int c = 0; c < C; ++c) GTk[c] = R(0.5) * (fa[c] + fb[c]) - hay * (ap[c] - am[c]);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        sfx[c] += gw[k] * (FRk[c] - FLk[c]);
        sfs[c] += gw[k] * (FLk[c] + FRk[c]);
        sfxe[c] += gw[k] * gx[k] * (FRk[c] - FLk[c]);
        sgy[c] += gw[k] * (GTk[c] - GBk[c]);
        sgs[c] += gw[k] * (GBk[c] + GTk[c]);
        sgyx[c] += gw[k] * gx[k] * (GTk[c] - GBk[c]);
      }
    };
    if constexpr (kPacked) {
      // FP32 Euler: points in pairs, (interior p, p + 1) and (Gauss k, k + 1)
      // of every face, each flux, Lax-Friedrichs flux and weighted sum in
      // packed FP32; the pairs' halves are added at the end and an odd last
      // point (3 Gauss points) runs alone.  COMP: the fluxes are increments
      // over f(B), a neighbour's face values moved onto B by one broadcast add
      auto flux_x2 = [&](const float2* U, int dir, float2* F) {
        if constexpr (COMP) flux_inc2_x2(gas, B, U, dir, F);
        else euler_flux_x2(gas, U, dir, F);
      };
      auto rebase_x2 = [&](float2* v, int dx, int dy) {
        if constexpr (COMP) {
#pragma unroll
          for (int c = 0; c < C; ++c)
            v[c] = __fadd2_rn(v[c], bcast2(__fsub_rn(sm.u[c][0][cj + OYR + dy][ci + OXR + dx], B[c])));
        }
      };
      float2 Fv2[C], Gv2[C];
#pragma unroll
      for (int c = 0; c < C; ++c) Fv2[c] = Gv2[c] = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int p = 0; p + 1 < NI; p += 2) {
        float2 U2[C], f2[C], g2[C];
#pragma unroll
        for (int c = 0; c < C; ++c) U2[c] = make_float2(inter[c][p], inter[c][p + 1]);
        flux_x2(U2, 0, f2);
        flux_x2(U2, 1, g2);
        const float2 w2 = make_float2(gw[p % NG] * gw[p / NG], gw[(p + 1) % NG] * gw[(p + 1) / NG]);
#pragma unroll
        for (int c = 0; c < C; ++c) {
          Fv2[c] = __ffma2_rn(w2, f2[c], Fv2[c]);
          Gv2[c] = __ffma2_rn(w2, g2[c], Gv2[c]);
        }
      }
#pragma unroll
      for (int c = 0; c < C; ++c) {
        Fv[c] = Fv2[c].x + Fv2[c].y;
        Gv[c] = Gv2[c].x + Gv2[c].y;
      }
      if constexpr (NI % 2 == 1) interior_point(NI - 1);
      float2 sfx2[C], sfs2[C], sfxe2[C], sgy2[C], sgs2[C], sgyx2[C];
#pragma unroll
      for (int c = 0; c < C; ++c)
        sfx2[c] = sfs2[c] = sfxe2[c] = sgy2[c] = sgs2[c] = sgyx2[c] = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int k = 0; k + 1 < NG; k += 2) {
        const float2 gw2 = make_float2(gw[k], gw[k + 1]);
        const float2 gwx2 = make_float2(gw[k] * gx[k], gw[k + 1] * gx[k + 1]);
        float2 am[C], ap[C], fa[C], fb[C], FL[C], FR[C], GB[C], GT[C];
#pragma unroll
        for (int c = 0; c < C; ++c) {
          am[c] = make_float2(sm.xf[c][NG + k][cj][ci], sm.xf[c][NG + k + 1][cj][ci]);
          ap[c] = make_float2(sm.xf[c][k][cj][ci + 1], sm.xf[c][k + 1][cj][ci + 1]);
        }
        rebase_x2(am, -1, 0);
        flux_x2(am, 0, fa); flux_x2(ap, 0, fb);
#pragma unroll
        for (int c = 0; c < C; ++c) FL[c] = lf_x2(fa[c], fb[c], am[c], ap[c], hax);
#pragma unroll
        for (int c = 0; c < C; ++c) {
          am[c] = make_float2(sm.xf[c][NG + k][cj][ci + 1], sm.xf[c][NG + k + 1][cj][ci + 1]);
          ap[c] = make_float2(sm.xf[c][k][cj][ci + 2], sm.xf[c][k + 1][cj][ci + 2]);
        }
        rebase_x2(ap, 1, 0);
        flux_x2(am, 0, fa); flux_x2(ap, 0, fb);
#pragma unroll
        for (int c = 0; c < C; ++c) FR[c] = lf_x2(fa[c], fb[c], am[c], ap[c], hax);
#pragma unroll
        for (int c = 0; c < C; ++c) {
          am[c] = make_float2(sm.yf[c][NG + k][cj][ci], sm.yf[c][NG + k + 1][cj][ci]);
          ap[c] = make_float2(sm.yf[c][k][cj + 1][ci], sm.yf[c][k + 1][cj + 1][ci]);
        }
        rebase_x2(am, 0, -1);
        flux_x2(am, 1, fa); flux_x2(ap, 1, fb);
#pragma unroll
        for (int c = 0; c < C; ++c) GB[c] = lf_x2(fa[c], fb[c], am[c], ap[c], hay);
#pragma unroll
        for (int c = 0; c < C; ++c) {
          am[c] = make_float2(sm.yf[c][NG + k][cj + 1][ci], sm.yf[c][NG + k + 1][cj + 1][ci]);
          ap[c] = make_float2(sm.yf[c][k][cj + 2][ci], sm.yf[c][k + 1][cj + 2][ci]);
        }
        rebase_x2(ap, 0, 1);
        flux_x2(am, 1, fa); flux_x2(ap, 1, fb);
#pragma unroll
        for (int c = 0; c < C; ++c) GT[c] = lf_x2(fa[c], fb[c], am[c], ap[c], hay);
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const float2 dx = sub2(FR[c], FL[c]), dy = sub2(GT[c], GB[c]);
          sfx2[c] = __ffma2_rn(gw2, dx, sfx2[c]);
          sfs2[c] = __ffma2_rn(gw2, __fadd2_rn(FL[c], FR[c]), sfs2[c]);
          sfxe2[c] = __ffma2_rn(gwx2, dx, sfxe2[c]);
          sgy2[c] = __ffma2_rn(gw2, dy, sgy2[c]);
          sgs2[c] = __ffma2_rn(gw2, __fadd2_rn(GB[c], GT[c]), sgs2[c]);
          sgyx2[c] = __ffma2_rn(gwx2, dy, sgyx2[c]);
        }
      }
#pragma unroll
      for (int c = 0; c < C; ++c) {
        sfx[c] = sfx2[c].x + sfx2[c].y;
        sfs[c] = sfs2[c].x + sfs2[c].y;
        sfxe[c] = sfxe2[c].x + sfxe2[c].y;
        sgy[c] = sgy2[c].x + sgy2[c].y;
        sgs[c] = sgs2[c].x + sgs2[c].y;
        sgyx[c] = sgyx2[c].x + sgyx2[c].y;
      }
      if constexpr (NG % 2 == 1) face_point(NG - 1);
    } else {
#pragma unroll
      for (int p = 0; p < NI; ++p) interior_point(p);
#pragma unroll
      for (int k = 0; k < NG; ++k) face_point(k);
    }
    R Uo[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const R L0 = -sfx[c] * inv_dx - sgy[c] * inv_dy;
      const R L1 = -R(0.5) * sfs[c] * inv_dx + Fv[c] * inv_dx - sgyx[c] * inv_dy;
      const R L2 = -sfxe[c] * inv_dx - R(0.5) * sgs[c] * inv_dy + Gv[c] * inv_dy;
      // the stage input the combination uses: first moments as modified by
      // Step 4 (stored, the default), or unmodified (variant)
      // (the tile holds the modified ones; the raw ones of an own cell are
      // read back from the stage input)
      const bool raw = (a.variant & HWENO_VARIANT_RAW_COMBINE) != 0;
      const size_t sw = (size_t)gj * nx + gi;
      const R W[3] = {sm.u[c][0][cj + OYR][ci + OXR],
                      raw ? (own ? w[(3 * c + 1) * plane + sw] : R(0)) : sm.u[c][1][cj + OYR][ci + OXR],
                      raw ? (own ? w[(3 * c + 2) * plane + sw] : R(0)) : sm.u[c][2][cj + OYR][ci + OXR]};
      const R Lm[3] = {L0, L1, L2};
      R o[3];
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        if (a.stage == 0) {
          o[m] = Lm[m];
        } else {
          const R s = W[m] + dt * Lm[m];
          if (a.stage == 1) o[m] = s;
          else {
            const R ca = a.stage == 2 ? R(0.75) : R(1.0 / 3.0);
            const R cb = a.stage == 2 ? R(0.25) : R(2.0 / 3.0);
            o[m] = ca * u0c[c][m] + cb * s;
          }
        }
        if (!isfinite(o[m])) bad |= ST_NONFINITE;
      }
      R olo = R(0);
      if constexpr (COMP) {
        // the average as a float pair: a u^n + b w in pair arithmetic (1/3
        // and 2/3 as pairs), then the increment b dt L
        constexpr float t1h = 1.0f / 3.0f, t2h = 2.0f / 3.0f;
        constexpr float t1l = (float)(1.0 / 3.0 - (double)t1h), t2l = (float)(2.0 / 3.0 - (double)t2h);
        const R wl = sm.ulo[c][cj + OYR][ci + OXR];
        R bh = W[0], bl = wl;
        if (a.stage == 2)
          pair_axpby(0.75f, 0.0f, u0c[c][0], u0l[c], 0.25f, 0.0f, W[0], wl, bh, bl);
        else if (a.stage == 3)
          pair_axpby(t1h, t1l, u0c[c][0], u0l[c], t2h, t2l, W[0], wl, bh, bl);
        const R cb = a.stage == 2 ? R(0.25) : a.stage == 3 ? R(2.0 / 3.0) : R(1);
        pair_add(bh, bl, (cb * dt) * L0, o[0], olo);
        if (!isfinite(o[0])) bad |= ST_NONFINITE;
      }
      if (own) {
        R* out = static_cast<R*>(a.out);
        const size_t s = (size_t)gj * nx + gi;
#pragma unroll
        for (int m = 0; m < 3; ++m) out[(3 * c + m) * plane + s] = o[m];
        if constexpr (COMP) a.out_lo[c * plane + s] = olo;
        if (a.lim_out) {  // rhs mode: the modified moments; stage 1: what stages 2-3 combine
          R* lo = static_cast<R*>(a.lim_out);
          const R M[3] = {W[0], sm.u[c][1][cj + OYR][ci + OXR], sm.u[c][2][cj + OYR][ci + OXR]};
#pragma unroll
          for (int m = 0; m < 3; ++m) lo[(3 * c + m) * plane + s] = a.stage == 0 ? M[m] : W[m];
        }
      }
      Uo[c] = o[0];
    }
    if (own) {
      if (a.flags_out) a.flags_out[(size_t)gj * nx + gi] = (uint8_t)myflag;
      if (a.stage > 0 && a.a_out) {  // (a replayed stage needs no maxima)
        wave_speeds2<R, C>(gas, Uo, spx, spy);
        if (!(spx == spx) || !(spy == spy)) {
          bad |= ST_NONPHYSICAL;
          spx = spy = R(0);
        }
      }
    } else {
      myflag = 0;
      bad = 0;
    }
  }

  // ---- 5. epilogue
  for (int o = 16; o > 0; o >>= 1) {
    spx = fmax(spx, __shfl_xor_sync(0xffffffffu, spx, o));
    spy = fmax(spy, __shfl_xor_sync(0xffffffffu, spy, o));
  }
  const int wcnt = __popc(__ballot_sync(0xffffffffu, myflag));
  if (lane == 0) {
    sm.red[0][warp] = spx;
    sm.red[1][warp] = spy;
    sm.cnt[warp] = wcnt;
  }
  if (bad) atomicOr(&a.sc->status, bad);
  __syncthreads();
  if (warp == 0) {
    R mx = lane < NW ? sm.red[0][lane] : R(0);
    R my = lane < NW ? sm.red[1][lane] : R(0);
    int cn = lane < NW ? sm.cnt[lane] : 0;
    for (int o = 16; o > 0; o >>= 1) {
      mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      my = fmax(my, __shfl_xor_sync(0xffffffffu, my, o));
      cn += __shfl_xor_sync(0xffffffffu, cn, o);
    }
    if (lane == 0) {
      const int slot = (blockIdx.y * gridDim.x + blockIdx.x) % kAlphaSlots;
      if (a.a_out) {
        atomic_max_nonneg(static_cast<R*>(a.a_out) + slot, mx);
        atomic_max_nonneg(static_cast<R*>(a.a_out) + kAlphaSlots + slot, my);
      }
      if (cn) atomicAdd(&a.sc->troubled, (unsigned long long)cn);
      if (a.stage == 3 && blockIdx.x == 0 && blockIdx.y == 0) {
        DevScalars* sc = a.sc;
        const double tf = sc->t_final;
        const double t = sc->last ? tf : sc->t + sc->dt;
        const double r = tf > 0.0 ? tf - t : (double)INFINITY;
        sc->t = t;
        sc->rem = r;
        sc->rem_f = (float)r;
        sc->steps += 1;
      }
    }
  }
}

// dt of a 2D step (Sec. 3, CFL; reading: dt = CFL / (alpha_x / dx + alpha_y /
// dy)), in FP64: one warp folds the wave-speed maxima of the step's input
// (kernel precision, so exact in FP64), forms dt and its clip to t_final,
// and leaves dt (FP64 and FP32 copies) and the last-step flag in the
// scalars, where the three stage kernels read it.
template <typename R>
__global__ void __launch_bounds__(32) dt2d_kernel(const R* __restrict__ a_in, int nin,
                                                  DevScalars* sc, double cfl, double inv_dx,
                                                  double inv_dy) {
  double ax = 0.0, ay = 0.0;
  for (int k = threadIdx.x; k < nin; k += 32) {
    ax = fmax(ax, (double)a_in[k]);
    ay = fmax(ay, (double)a_in[nin + k]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    ax = fmax(ax, __shfl_xor_sync(0xffffffffu, ax, o));
    ay = fmax(ay, __shfl_xor_sync(0xffffffffu, ay, o));
  }
  if (threadIdx.x == 0) {
    const double rem = sc->rem;
    double dt = cfl / (ax * inv_dx + ay * inv_dy);
    unsigned last = 0u;
    if (rem <= 0.0) {
      dt = 0.0;
    } else if (dt >= rem) {
      dt = rem;
      last = 1u;
    }
    if (!(ax + ay > 0.0) || !isfinite(dt)) dt = 0.0;
    sc->dt = dt;
    sc->dt_f = (float)dt;
    sc->last = last;
  }
}

template <typename R, int C>
__global__ void __launch_bounds__(NT) alpha2d_kernel(const R* __restrict__ w, R* a_out, int nx,
                                                    int ny, double gas, DevScalars* sc,
                                                    int slots) {
  __shared__ R red[2][NW];
  const int gi = blockIdx.x * TX + threadIdx.x % TX, gj = blockIdx.y * TY + threadIdx.x / TX;
  const size_t plane = (size_t)nx * ny;
  R sx = R(0), sy = R(0);
  if (gi < nx && gj < ny) {
    R U[C];
#pragma unroll
    for (int c = 0; c < C; ++c) U[c] = w[(3 * c) * plane + (size_t)gj * nx + gi];
    wave_speeds2<R, C>(R(gas), U, sx, sy);
    if (!(sx == sx) || !(sy == sy)) {
      atomicOr(&sc->status, (unsigned)ST_NONPHYSICAL);
      sx = sy = R(0);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    sx = fmax(sx, __shfl_xor_sync(0xffffffffu, sx, o));
    sy = fmax(sy, __shfl_xor_sync(0xffffffffu, sy, o));
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = sx;
    red[1][threadIdx.x >> 5] = sy;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < NW; ++k) {
      sx = fmax(sx, red[0][k]);
      sy = fmax(sy, red[1][k]);
    }
    const int b = blockIdx.y * gridDim.x + blockIdx.x;
    if (slots) {
      atomic_max_nonneg(a_out + b % kAlphaSlots, sx);
      atomic_max_nonneg(a_out + kAlphaSlots + b % kAlphaSlots, sy);
    } else {
      const int nt = gridDim.x * gridDim.y;
      a_out[b] = sx;
      a_out[nt + b] = sy;
    }
  }
}

template <typename R, int C, int NG, bool COMP>
cudaError_t launch_stage2d_t(const Stage2DArgs& a0, cudaStream_t s) {
  Stage2DArgs a = a0;
  CUtensorMap map, lo_map;
  a.tma = encode_box_map(a.w, a.nx, a.ny, 3 * C, (int)sizeof(R), RX, RY, &map) ? 1 : 0;
  memset(&lo_map, 0, sizeof(lo_map));
  if (COMP && a.tma)  // both boxes, or neither
    a.tma = encode_box_map(a.w_lo, a.nx, a.ny, C, (int)sizeof(R), RX, RY, &lo_map) ? 1 : 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)((a.nx + TX - 1) / TX), (unsigned)((a.ny + TY - 1) / TY));
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = sizeof(Smem2D<R, C, NG, COMP>);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, stage2d_kernel<R, C, NG, COMP>, a, map, lo_map);
}

template <typename R, int C, int NG, bool COMP>
cudaError_t prepare_one() {
  cudaError_t e = cudaFuncSetAttribute(stage2d_kernel<R, C, NG, COMP>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(Smem2D<R, C, NG, COMP>));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(stage2d_kernel<R, C, NG, COMP>,
                              cudaFuncAttributePreferredSharedMemoryCarveout, 100);
}
template <typename R, int C, int NG>
cudaError_t prepare_t() {
  cudaError_t e = prepare_one<R, C, NG, false>();
  if constexpr (sizeof(R) == 4) {
    if (e == cudaSuccess) e = prepare_one<R, C, NG, true>();
  }
  return e;
}

}  // namespace

int stage2d_tiles(int nx, int ny) { return ((nx + TX - 1) / TX) * ((ny + TY - 1) / TY); }

bool encode_box_map(const void* w, int nx, int ny, int planes, int esize, int box_x, int box_y,
                    CUtensorMap* map) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      fn = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }();
  memset(map, 0, sizeof(*map));
  if (!encode || !w || ((size_t)nx * esize) % 16 != 0 || ((uintptr_t)w) % 16 != 0 || nx < box_x ||
      ny < box_y || ((size_t)box_x * esize) % 16 != 0 || box_x > 256 || box_y > 256 || planes > 256)
    return false;
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)planes};
  const cuuint64_t strides[2] = {(cuuint64_t)nx * esize, (cuuint64_t)nx * ny * esize};
  const cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, (cuuint32_t)planes};
  const cuuint32_t estr[3] = {1, 1, 1};
  return encode(map, esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                3, const_cast<void*>(w), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void finish_stage2d_args(Stage2DArgs& a) {
  a.inv_dx = 1.0 / a.dx;
  a.inv_dy = 1.0 / a.dy;
  const double h = 0.5 * sqrt(a.dx * a.dx + a.dy * a.dy);
  a.kx.dx = a.dx;
  a.kx.dy = a.dy;
  a.kx.den_h = h * (a.dx + a.dy);
  a.kx.thr = a.thr;
  a.kx.fdx = (float)a.dx;
  a.kx.fdy = (float)a.dy;
  a.kx.fthr_den = (float)(a.thr * a.kx.den_h);
  a.kx.fdx_lo = (float)(a.dx - (double)a.kx.fdx);
  a.kx.fdy_lo = (float)(a.dy - (double)a.kx.fdy);
  a.kx.fthr_den_lo = (float)(a.thr * a.kx.den_h - (double)a.kx.fthr_den);
  for (int k = 0; k < 5; ++k) a.f32[k] = (float)a.gam[k];
  a.f32[5] = (float)a.eps;
  a.f32[6] = (float)a.gas;
  a.f32[7] = (float)a.inv_dx;
  a.f32[8] = (float)a.inv_dy;
  a.f32[9] = (float)a.cfl;
}

cudaError_t prepare_stage2d(int system, int fp64, int ng) {
  if (system == 0) {
    if (fp64) return ng == 2 ? prepare_t<double, 1, 2>() : prepare_t<double, 1, 3>();
    return ng == 2 ? prepare_t<float, 1, 2>() : prepare_t<float, 1, 3>();
  }
  if (fp64) return ng == 2 ? prepare_t<double, 4, 2>() : prepare_t<double, 4, 3>();
  return ng == 2 ? prepare_t<float, 4, 2>() : prepare_t<float, 4, 3>();
}

cudaError_t launch_stage2d(const Stage2DArgs& a, cudaStream_t s) {
  if (a.comp) {  // HWENO_FP32C (stages 1-3 of a step)
    if (a.system == 0)
      return a.ng == 2 ? launch_stage2d_t<float, 1, 2, true>(a, s) : launch_stage2d_t<float, 1, 3, true>(a, s);
    return a.ng == 2 ? launch_stage2d_t<float, 4, 2, true>(a, s) : launch_stage2d_t<float, 4, 3, true>(a, s);
  }
  if (a.system == 0) {
    if (a.fp64) return a.ng == 2 ? launch_stage2d_t<double, 1, 2, false>(a, s) : launch_stage2d_t<double, 1, 3, false>(a, s);
    return a.ng == 2 ? launch_stage2d_t<float, 1, 2, false>(a, s) : launch_stage2d_t<float, 1, 3, false>(a, s);
  }
  if (a.fp64) return a.ng == 2 ? launch_stage2d_t<double, 4, 2, false>(a, s) : launch_stage2d_t<double, 4, 3, false>(a, s);
  return a.ng == 2 ? launch_stage2d_t<float, 4, 2, false>(a, s) : launch_stage2d_t<float, 4, 3, false>(a, s);
}

cudaError_t launch_dt2d(const Stage2DArgs& a, cudaStream_t s) {
  if (a.fp64)
    dt2d_kernel<double><<<1, 32, 0, s>>>(static_cast<const double*>(a.a_in), a.nin, a.sc, a.cfl,
                                        a.inv_dx, a.inv_dy);
  else
    dt2d_kernel<float><<<1, 32, 0, s>>>(static_cast<const float*>(a.a_in), a.nin, a.sc, a.cfl,
                                       a.inv_dx, a.inv_dy);
  return cudaGetLastError();
}

cudaError_t launch_alpha2d(const void* w, void* a_out, int nx, int ny, int system, int fp64,
                           double gas, DevScalars* sc, int slots, cudaStream_t s) {
  dim3 grid((nx + TX - 1) / TX, (ny + TY - 1) / TY);
  if (system == 0) {
    if (fp64)
      alpha2d_kernel<double, 1><<<grid, NT, 0, s>>>(static_cast<const double*>(w), static_cast<double*>(a_out), nx, ny, gas, sc, slots);
    else
      alpha2d_kernel<float, 1><<<grid, NT, 0, s>>>(static_cast<const float*>(w), static_cast<float*>(a_out), nx, ny, gas, sc, slots);
  } else {
    if (fp64)
      alpha2d_kernel<double, 4><<<grid, NT, 0, s>>>(static_cast<const double*>(w), static_cast<double*>(a_out), nx, ny, gas, sc, slots);
    else
      alpha2d_kernel<float, 4><<<grid, NT, 0, s>>>(static_cast<const float*>(w), static_cast<float*>(a_out), nx, ny, gas, sc, slots);
  }
  return cudaGetLastError();
}

}  // namespace hw
