// Adjoint of one third-order TVD Runge-Kutta stage of the 2D hybrid HWENO
// scheme (Zhao & Qiu, arXiv:2002.08816, Sec. 2.2) with the switches of the
// forward run held fixed: the troubled cells of the stage (recorded in the
// forward pass), its Lax-Friedrichs speeds (alpha_x, alpha_y) and the step's
// dt.  Periodic boundaries.
//
// Forward, a stage maps its raw input w to W = Step 4(w) (first moments of
// troubled cells modified), to the values P_i = Step 5(D_i) at the 4 ng + ng^2
// Gauss points of every cell i (D_i: the 19 data of its 3x3 stencil), to the
// Lax-Friedrichs fluxes and L = Eq. (ode2), and to u_out = a W0 + b (W + dt L).
// Backward, lam being the adjoint of u_out:
//   kernel A, per cell i: the adjoints of the fluxes at its faces (from lam of
//     i and of its four neighbours, times b dt), of its point values (through
//     the flux Jacobians), and G_i = (dP_i/dD_i)^T lam_P, the adjoints of its
//     19 data (transposed linear p0, or the reverse of Step 5.1's nonlinear
//     combination where the stencil holds a troubled cell).  The tile sums, in
//     shared memory and in a fixed order, the entries of its cells' G_i for
//     every cell of the tile and its 1-cell ring, and writes these partial
//     sums (12 values per position) instead of the 76 per cell;
//   kernel B, per cell j: mu_j = b lam_j + the partial sums that the tiles
//     holding j's neighbours wrote for j (+ the adjoint of W0 at stage 1): the
//     adjoint of W, which passes through the moments Step 4 did not modify;
//   kernel C, only on tiles near a troubled cell: the reverse of Step 4, each
//     troubled cell sending the adjoint of its modified moments back to the
//     five data Step 1 read.
// Reverse-mode arithmetic: hweno_adj.cuh; transposed maps and smoothness-
// indicator gradients: the generated hweno2d_adj_coef.cuh.
#include <cuda_runtime.h>
#include <stdint.h>

#include "hweno2d_adj_coef.cuh"
#include "hweno_adj.cuh"
#include "hweno_device.cuh"
#include "hweno_internal.h"

namespace hw {
namespace {

constexpr int TX = kTile2DX, TY = kTile2DY;
constexpr int NT = kThreads2D;
constexpr int AX = TX + 4, AY = TY + 4;  // raw input, 2-cell halo
constexpr int BX = TX + 2, BY = TY + 2;  // 1-cell halo
// kernel A's tiles start 16-byte aligned in x (TMA): its raw input from x =
// bx0 - 4 (two columns more than the 2-cell halo needs), its lambda from x =
// bx0 - 4 (three more than the 1-cell halo), both TX + 8 wide
constexpr int AXA = TX + 8, LXA = TX + 8;
constexpr unsigned kTmaPollsA = 1u << 20;
static_assert(TX * TY == NT, "one own cell per thread");

template <typename R, int C>
struct SmemA {
  static constexpr int kPadX = 2;  // raw index of flag-grid column lx: lx + 1 + 2
  static constexpr bool kLimList = false;  // the limiter writes vl / wl
  alignas(128) R u[C][3][AY][AXA];   // raw stage input (a TMA box)
  alignas(128) R lam[C][3][BY][LXA]; // lam, the adjoint of the stage output (a TMA box;
                                     // b dt is applied where it is used)
  R vl[C][BY][BX];      // Step 4 moments
  R wl[C][BY][BX];
  // stencil adjoints of the own cells: one component's, or (FP32 Euler) a
  // pair of components' at once
  static constexpr bool kPairs = C == 4 && sizeof(R) == 4;
  R g[kPairs ? 1 : 19][TY][TX];
  float2 g2[kPairs ? 19 : 1][TY][TX];
  uint8_t fl[BY][BX];
  unsigned long long bar;  // mbarrier of the tile copies
};

// Offsets of the 19 stencil data (Fig. 1): averages of cells 1..9, then the
// x- and the y-moments of cells 2, 4, 5, 6, 8.
__device__ __forceinline__ int data_dx(int k) {
  return k < 9 ? k % 3 - 1 : ((k - 9) % 5 == 1 ? -1 : (k - 9) % 5 == 3 ? 1 : 0);
}
__device__ __forceinline__ int data_dy(int k) {
  return k < 9 ? k / 3 - 1 : ((k - 9) % 5 == 0 ? -1 : (k - 9) % 5 == 4 ? 1 : 0);
}

// The (tile, position) pairs along one axis under which the partial sums of
// kernel A hold cell j: position p of tile t is the cell t T + p - 1 (wrapped);
// j gets contributions from the cells j - 1, j, j + 1 (d = 0, 1, 2), each in
// its own tile; u[d] is false when an earlier d gave the same pair.
__device__ __forceinline__ void part_pairs(int j, int n, int T, int* t, int* p, bool* u) {
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int i = bc_map(j + d - 1, n, 0);
    t[d] = i / T;
    p[d] = i - t[d] * T - (d - 1) + 1;
    u[d] = true;
#pragma unroll
    for (int q = 0; q < d; ++q) u[d] = u[d] && !(t[q] == t[d] && p[q] == p[d]);
  }
}

template <typename R, int C>
struct SmemB {
  static constexpr int kPadX = 0;
  int nt;                          // troubled cells of the 1-halo grid, listed
  unsigned short tl[BX * BY];
  R mu[C][3][BY][BX];   // adjoint of W
  R u[C][3][AY][AX];    // raw stage input (tiles near a troubled cell)
  R cx[C][5][BY][BX];   // x-direction Step 1 of a troubled cell: adjoints of
  R cy[C][5][BY][BX];   // u_{i-1}, u_i, u_{i+1}, v_{i-1}, v_{i+1} (y: w)
  uint8_t fl[BY][BX];
};

// scalar parameters in the kernel's precision
template <typename R>
struct AdjParams {
  R gam[5], eps, gas, inv_dx, inv_dy;
  __device__ __forceinline__ explicit AdjParams(const Adj2DArgs& a) {
    if constexpr (sizeof(R) == 4) {
#pragma unroll
      for (int k = 0; k < 5; ++k) gam[k] = a.f32[k];
      eps = a.f32[5]; gas = a.f32[6]; inv_dx = a.f32[7]; inv_dy = a.f32[8];
    } else {
#pragma unroll
      for (int k = 0; k < 5; ++k) gam[k] = a.gam[k];
      eps = a.eps; gas = a.gas; inv_dx = 1.0 / a.dx; inv_dy = 1.0 / a.dy;
    }
  }
};

// Eq. (RK) weight b of the stage's W + dt L
template <typename R>
__device__ __forceinline__ R stage_b(int stage) {
  return stage == 1 ? R(1) : stage == 2 ? R(0.25) : stage == 3 ? R(2.0 / 3.0) : R(0);
}

// The 19 data of component c of the cell at own-tile coordinates (ci, cj),
// ci, cj in [-1, TX] x [-1, TY]: averages of cells 1..9, Step 4 x- and
// y-moments of cells 2, 4, 5, 6, 8 (Fig. 1).
template <typename S, typename R>
__device__ __forceinline__ void gather19a(const S& sm, int c, int ci, int cj, R* d) {
#pragma unroll
  for (int k = 0; k < 9; ++k) d[k] = sm.u[c][0][cj + 2 + k / 3 - 1][ci + 2 + S::kPadX + k % 3 - 1];
  const int mx[5] = {0, -1, 0, 1, 0}, my[5] = {-1, 0, 0, 0, 1};
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    d[9 + k] = sm.vl[c][cj + 1 + my[k]][ci + 1 + mx[k]];
    d[14 + k] = sm.wl[c][cj + 1 + my[k]][ci + 1 + mx[k]];
  }
}

// Step 5.1 interface values of an Euler cell next to a troubled cell (x-faces
// in the x characteristic fields, y-faces in the y fields of the average).
template <int NG, typename S, typename R>
__device__ __noinline__ void hw_faces_euler_vals(const S& sm, int ci, int cj, R g0, R g1, R g2,
                                                 R g3, R g4, R eps, R gas, R (*out)[4 * NG]) {
  constexpr int NF = 4 * NG;
  const R gam[5] = {g0, g1, g2, g3, g4};  // by value: the caller's parameters stay off the stack
  R D[4][19];
#pragma unroll
  for (int c = 0; c < 4; ++c) gather19a(sm, c, ci, cj, D[c]);
  R U[4] = {D[0][4], D[1][4], D[2][4], D[3][4]};
#pragma unroll 1
  for (int dir = 0; dir < 2; ++dir) {
    const int lo = dir == 0 ? 0 : 2 * NG, hi = lo + 2 * NG;
    R Rm[4][4], Lm[4][4];
    Euler2D<R>::eigen(gas, U, dir, Rm, Lm);
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int p = 0; p < NF; ++p)
        if (p >= lo && p < hi) out[c][p] = R(0);
#pragma unroll 1
    for (int f = 0; f < 4; ++f) {
      R e[19], chv[NF];
#pragma unroll
      for (int k = 0; k < 19; ++k)
        e[k] = Lm[f][0] * D[0][k] + Lm[f][1] * D[1][k] + Lm[f][2] * D[2][k] + Lm[f][3] * D[3][k];
      hweno2d_faces<NG>(e, gam, eps, lo, hi, chv);
#pragma unroll
      for (int p = 0; p < NF; ++p)
        if (p >= lo && p < hi)
#pragma unroll
          for (int c = 0; c < 4; ++c) out[c][p] += Rm[c][f] * chv[p];
    }
  }
}

// Reverse of hw_faces_euler_vals: G[c][k] += the adjoint of datum k of
// component c, given the adjoints lam[c][p] of the interface values.
template <int NG, typename S, typename R>
__device__ __noinline__ void hw_faces_euler_vjp(const S& sm, int ci, int cj, R g0, R g1, R g2,
                                                R g3, R g4, R eps, R gas, R (*lam)[4 * NG],
                                                R (*G)[19]) {
  constexpr int NF = 4 * NG;
  const R gam[5] = {g0, g1, g2, g3, g4};
  R D[4][19];
#pragma unroll
  for (int c = 0; c < 4; ++c) gather19a(sm, c, ci, cj, D[c]);
  R U[4] = {D[0][4], D[1][4], D[2][4], D[3][4]};
#pragma unroll 1
  for (int dir = 0; dir < 2; ++dir) {
    const int lo = dir == 0 ? 0 : 2 * NG, hi = lo + 2 * NG;
    R Rm[4][4], Lm[4][4], lR[4][4], lL[4][4];
    Euler2D<R>::eigen(gas, U, dir, Rm, Lm);
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) lR[r][q] = lL[r][q] = R(0);
#pragma unroll 1
    for (int f = 0; f < 4; ++f) {
      R e[19], chv[NF], lch[NF], ge[19];
#pragma unroll
      for (int k = 0; k < 19; ++k) {
        e[k] = Lm[f][0] * D[0][k] + Lm[f][1] * D[1][k] + Lm[f][2] * D[2][k] + Lm[f][3] * D[3][k];
        ge[k] = R(0);
      }
      hweno2d_faces<NG>(e, gam, eps, lo, hi, chv);
#pragma unroll
      for (int p = 0; p < NF; ++p) {
        lch[p] = R(0);
        if (p >= lo && p < hi) {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            lch[p] += Rm[c][f] * lam[c][p];
            lR[c][f] += chv[p] * lam[c][p];
          }
        }
      }
      hweno2d_faces_vjp<NG>(e, gam, eps, lch, ge);
#pragma unroll
      for (int k = 0; k < 19; ++k)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          G[c][k] += Lm[f][c] * ge[k];
          lL[f][c] += ge[k] * D[c][k];
        }
    }
    R gU[4] = {R(0), R(0), R(0), R(0)};
    euler2d_eigen_vjp(gas, U, dir, lR, lL, gU);
#pragma unroll
    for (int c = 0; c < 4; ++c) G[c][4] += gU[c];
  }
}

// Reverse of Step 4 for a troubled Euler cell (lx, ly) of the 1-halo grid:
// the adjoints mu of its modified x- and y-moments go back to the five data
// of each direction (cx, cy), including through the eigen-system of the
// cell's average.
template <typename S, typename R>
__device__ __noinline__ void limit_euler2d_vjp(S& sm, int lx, int ly, R g0, R g1, R g2, R g3, R g4,
                                               R eps, R gas) {
  const R gam[5] = {g0, g1, g2, g3, g4};
  const int rx = lx + 1, ry = ly + 1;
  R U[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) U[c] = sm.u[c][0][ry][rx];
#pragma unroll 1
  for (int dir = 0; dir < 2; ++dir) {
    const int sx = dir == 0 ? 1 : 0, sy = dir == 0 ? 0 : 1;
    const int mom = dir == 0 ? 1 : 2;
    R Rm[4][4], Lm[4][4], lR[4][4], lL[4][4], src[5][4], out[5][4], mu[4];
    Euler2D<R>::eigen(gas, U, dir, Rm, Lm);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      src[0][c] = sm.u[c][0][ry - sy][rx - sx];
      src[1][c] = U[c];
      src[2][c] = sm.u[c][0][ry + sy][rx + sx];
      src[3][c] = sm.u[c][mom][ry - sy][rx - sx];
      src[4][c] = sm.u[c][mom][ry + sy][rx + sx];
      mu[c] = sm.mu[c][mom][ly][lx];
#pragma unroll
      for (int k = 0; k < 5; ++k) out[k][c] = R(0);
#pragma unroll
      for (int q = 0; q < 4; ++q) lR[c][q] = lL[c][q] = R(0);
    }
#pragma unroll 1
    for (int f = 0; f < 4; ++f) {
      R wv[5], g5[5];
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        wv[k] = Lm[f][0] * src[k][0] + Lm[f][1] * src[k][1] + Lm[f][2] * src[k][2] +
                Lm[f][3] * src[k][3];
        g5[k] = R(0);
      }
      const R lq = Rm[0][f] * mu[0] + Rm[1][f] * mu[1] + Rm[2][f] * mu[2] + Rm[3][f] * mu[3];
      const R q = limit_first_moment_vjp(wv[0], wv[1], wv[2], wv[3], wv[4], gam, eps, lq, g5);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        lR[c][f] += mu[c] * q;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
          out[k][c] += Lm[f][c] * g5[k];
          lL[f][c] += g5[k] * src[k][c];
        }
      }
    }
    R gU[4] = {R(0), R(0), R(0), R(0)};
    euler2d_eigen_vjp(gas, U, dir, lR, lL, gU);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      out[1][c] += gU[c];
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        if (dir == 0) sm.cx[c][k][ly][lx] = out[k][c]; else sm.cy[c][k][ly][lx] = out[k][c];
      }
    }
  }
}

// ------------------------------------------------------------- kernel A

template <typename R, int C, int NG>
__global__ void __launch_bounds__(NT, (sizeof(R) == 4 ? 2 : 1))
    adj2d_points_kernel(Adj2DArgs a, const __grid_constant__ CUtensorMap u_map,
                        const __grid_constant__ CUtensorMap lam_map) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  SmemA<R, C>& sm = *reinterpret_cast<SmemA<R, C>*>(smem_raw);
  constexpr int NF = 4 * NG, NI = NG * NG, NP = NF + NI;
  const int tid = threadIdx.x;
  const int nx = a.nx, ny = a.ny;
  const int bx0 = blockIdx.x * TX, by0 = blockIdx.y * TY;
  const size_t plane = (size_t)nx * ny;
  const AdjParams<R> P_(a);
  const R* __restrict__ w = static_cast<const R*>(a.w);
  const R* __restrict__ lam = static_cast<const R*>(a.lam);
  const R ax = static_cast<const R*>(a.alpha)[0], ay = static_cast<const R*>(a.alpha)[1];
  const R scale = a.stage == 0 ? R(1) : stage_b<R>(a.stage) * *static_cast<const R*>(a.dt);

  // interior tiles: the raw input and lambda as two TMA boxes (all 3 C
  // planes each) on one mbarrier; the outermost ring of tiles (periodic
  // wrap) through the boundary map
  const bool tma = a.tma && bx0 >= 4 && bx0 - 4 + AXA <= nx && by0 >= 2 && by0 - 2 + AY <= ny;
  if (tma && tid == 0) {
    mbar_init(&sm.bar, 1);
    mbar_expect_tx(&sm.bar, (unsigned)(sizeof(sm.u) + sizeof(sm.lam)));
    tma_load_3d(&sm.u[0][0][0][0], &u_map, &sm.bar, bx0 - 4, by0 - 2, 0);
    tma_load_3d(&sm.lam[0][0][0][0], &lam_map, &sm.bar, bx0 - 4, by0 - 1, 0);
  }
  if (!tma) {
    for (int k = tid; k < AXA * AY; k += NT) {
      const int rx = k % AXA, ry = k / AXA;
      const size_t s = (size_t)bc_map(by0 - 2 + ry, ny, 0) * nx + bc_map(bx0 - 4 + rx, nx, 0);
#pragma unroll
      for (int c = 0; c < C; ++c)
#pragma unroll
        for (int m = 0; m < 3; ++m) sm.u[c][m][ry][rx] = w[(3 * c + m) * plane + s];
    }
    for (int k = tid; k < LXA * BY; k += NT) {
      const int lx = k % LXA, ly = k / LXA;
      const size_t s = (size_t)bc_map(by0 - 1 + ly, ny, 0) * nx + bc_map(bx0 - 4 + lx, nx, 0);
#pragma unroll
      for (int c = 0; c < C; ++c)
#pragma unroll
        for (int m = 0; m < 3; ++m) sm.lam[c][m][ly][lx] = lam[(3 * c + m) * plane + s];
    }
  }
  int ring_troubled = 0;
  for (int k = tid; k < BX * BY; k += NT) {
    const int lx = k % BX, ly = k / BX;
    const size_t s = (size_t)bc_map(by0 - 1 + ly, ny, 0) * nx + bc_map(bx0 - 1 + lx, nx, 0);
    sm.fl[ly][lx] = a.flags[s] != 0;
    ring_troubled |= sm.fl[ly][lx];
  }
  const bool tile_troubled = __syncthreads_or(ring_troubled);  // uniform over the CTA
  if (tile_troubled && tid == 0) {  // kernel C's work list
    const int q = atomicAdd(a.tile_list, 1);
    a.tile_list[1 + q] = blockIdx.y * gridDim.x + blockIdx.x;
  }
  if (tma && !mbar_wait_bounded(&sm.bar, 0, kTmaPollsA)) {
    // the copies did not land: flag it and give them a second bounded wait
    // (they write this CTA's shared memory); no thread leaves the common path
    if (a.sc) atomicOr(&a.sc->status, ST_TIMEOUT);
    mbar_wait_bounded(&sm.bar, 0, kTmaPollsA);
  }

  // Step 4 on the tile and its 1-cell halo (the forward values)
  for (int k = tid; k < BX * BY; k += NT) {
    const int lx = k % BX, ly = k / BX;
    const int rx = lx + 1 + SmemA<R, C>::kPadX, ry = ly + 1;
    if (!sm.fl[ly][lx]) {
#pragma unroll
      for (int c = 0; c < C; ++c) {
        sm.vl[c][ly][lx] = sm.u[c][1][ry][rx];
        sm.wl[c][ly][lx] = sm.u[c][2][ry][rx];
      }
    } else if constexpr (C == 1) {
      sm.vl[0][ly][lx] = limit_first_moment(sm.u[0][0][ry][rx - 1], sm.u[0][0][ry][rx],
                                            sm.u[0][0][ry][rx + 1], sm.u[0][1][ry][rx - 1],
                                            sm.u[0][1][ry][rx + 1], P_.gam, P_.eps);
      sm.wl[0][ly][lx] = limit_first_moment(sm.u[0][0][ry - 1][rx], sm.u[0][0][ry][rx],
                                            sm.u[0][0][ry + 1][rx], sm.u[0][2][ry - 1][rx],
                                            sm.u[0][2][ry + 1][rx], P_.gam, P_.eps);
    } else {
      limit_euler2d(sm, lx, ly, 0, P_.gam[0], P_.gam[1], P_.gam[2], P_.gam[3], P_.gam[4], P_.eps,
                    P_.gas);
    }
  }
  __syncthreads();

  const int ci = tid % TX, cj = tid / TX;
  const int gi = bx0 + ci, gj = by0 + cj;
  const bool own = gi < nx && gj < ny;
  bool hw = false;  // the cell's 3x3 stencil holds a troubled cell
  if (tile_troubled) {
#pragma unroll
    for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
      for (int di = -1; di <= 1; ++di) hw |= sm.fl[cj + 1 + dj][ci + 1 + di] != 0;
  }

  // point values (the forward's); FP32 Euler: the linear maps on pairs of
  // components in packed FP32, as the forward stage kernel
  constexpr bool kPacked = C == 4 && sizeof(R) == 4;
  R P[C][NP];
  if constexpr (kPacked) {
#pragma unroll
    for (int c = 0; c < C; c += 2) {
      R da[19], db[19];
      gather19a(sm, c, ci, cj, da);
      gather19a(sm, c + 1, ci, cj, db);
      float2 d2[19], v2[NP];
#pragma unroll
      for (int k = 0; k < 19; ++k) d2[k] = make_float2(da[k], db[k]);
      p0_faces_x2<NG>(d2, v2);
      p0_interior_x2<NG>(d2, &v2[NF]);
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        P[c][p] = v2[p].x;
        P[c + 1][p] = v2[p].y;
      }
    }
  } else {
#pragma unroll
    for (int c = 0; c < C; ++c) {
      R d[19];
      gather19a(sm, c, ci, cj, d);
      p0_faces<NG>(d, P[c]);
      p0_interior<NG>(d, &P[c][NF]);
      if constexpr (C == 1) {
        if (hw) hweno2d_faces<NG>(d, P_.gam, P_.eps, 0, NF, P[c]);
      }
    }
  }
  if constexpr (C == 4) {
    if (hw) {
      R hv[4][NF];
      hw_faces_euler_vals<NG>(sm, ci, cj, P_.gam[0], P_.gam[1], P_.gam[2], P_.gam[3], P_.gam[4],
                              P_.eps, P_.gas, hv);
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int p = 0; p < NF; ++p) P[c][p] = hv[c][p];
    }
  }

  // adjoints of the point values, in place
  constexpr double r15 = 0.38729833462074168852;  // sqrt(15)/10
  constexpr double r3 = 0.28867513459481288225;   // sqrt(3)/6
  const R gw[3] = {NG == 3 ? R(5.0 / 18.0) : R(0.5), NG == 3 ? R(4.0 / 9.0) : R(0.5), R(5.0 / 18.0)};
  const R gx[3] = {NG == 3 ? R(-r15) : R(-r3), NG == 3 ? R(0) : R(r3), R(r15)};
  const R hax = R(0.5) * ax, hay = R(0.5) * ay;
  const int lx = ci + 1, ly = cj + 1;
  // sm.lam holds lambda itself (from x = bx0 - 4); b dt enters the weights
#define LAM(c, m, di, dj) sm.lam[c][m][ly + (dj)][lx + 3 + (di)]
  // the adjoints of the four faces' point values at Gauss point k
  auto face_point = [&](int k) {
    const R wxk = gw[k] * P_.inv_dx * scale, wyk = gw[k] * P_.inv_dy * scale;
    R lf[C], U[C], o[C];
    // x_{i-1/2}: own left point k is u^+
#pragma unroll
    for (int c = 0; c < C; ++c) {
      lf[c] = wxk * (LAM(c, 0, 0, 0) - R(0.5) * LAM(c, 1, 0, 0) + gx[k] * LAM(c, 2, 0, 0) -
                     LAM(c, 0, -1, 0) - R(0.5) * LAM(c, 1, -1, 0) - gx[k] * LAM(c, 2, -1, 0));
      U[c] = P[c][k];
    }
    flux_jt2<R, C>(P_.gas, U, 0, lf, o);
#pragma unroll
    for (int c = 0; c < C; ++c) P[c][k] = R(0.5) * o[c] - hax * lf[c];
    // x_{i+1/2}: own right point NG+k is u^-
#pragma unroll
    for (int c = 0; c < C; ++c) {
      lf[c] = wxk * (-LAM(c, 0, 0, 0) - R(0.5) * LAM(c, 1, 0, 0) - gx[k] * LAM(c, 2, 0, 0) +
                     LAM(c, 0, 1, 0) - R(0.5) * LAM(c, 1, 1, 0) + gx[k] * LAM(c, 2, 1, 0));
      U[c] = P[c][NG + k];
    }
    flux_jt2<R, C>(P_.gas, U, 0, lf, o);
#pragma unroll
    for (int c = 0; c < C; ++c) P[c][NG + k] = R(0.5) * o[c] + hax * lf[c];
    // y_{j-1/2}: own bottom point 2NG+k is u^+
#pragma unroll
    for (int c = 0; c < C; ++c) {
      lf[c] = wyk * (LAM(c, 0, 0, 0) + gx[k] * LAM(c, 1, 0, 0) - R(0.5) * LAM(c, 2, 0, 0) -
                     LAM(c, 0, 0, -1) - gx[k] * LAM(c, 1, 0, -1) - R(0.5) * LAM(c, 2, 0, -1));
      U[c] = P[c][2 * NG + k];
    }
    flux_jt2<R, C>(P_.gas, U, 1, lf, o);
#pragma unroll
    for (int c = 0; c < C; ++c) P[c][2 * NG + k] = R(0.5) * o[c] - hay * lf[c];
    // y_{j+1/2}: own top point 3NG+k is u^-
#pragma unroll
    for (int c = 0; c < C; ++c) {
      lf[c] = wyk * (-LAM(c, 0, 0, 0) - gx[k] * LAM(c, 1, 0, 0) - R(0.5) * LAM(c, 2, 0, 0) +
                     LAM(c, 0, 0, 1) + gx[k] * LAM(c, 1, 0, 1) - R(0.5) * LAM(c, 2, 0, 1));
      U[c] = P[c][3 * NG + k];
    }
    flux_jt2<R, C>(P_.gas, U, 1, lf, o);
#pragma unroll
    for (int c = 0; c < C; ++c) P[c][3 * NG + k] = R(0.5) * o[c] + hay * lf[c];
  };
  // interior point p: the volume integrals of Eq. (ode2)'s moment equations
  auto interior_point = [&](int p) {
    const int k = (p - NF) % NG, l = (p - NF) / NG;
    const R wk = gw[k] * gw[l];
    R U[C], l1[C], l2[C], o1[C], o2[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      U[c] = P[c][p];
      l1[c] = wk * P_.inv_dx * scale * LAM(c, 1, 0, 0);
      l2[c] = wk * P_.inv_dy * scale * LAM(c, 2, 0, 0);
    }
    flux_jt2<R, C>(P_.gas, U, 0, l1, o1);
    flux_jt2<R, C>(P_.gas, U, 1, l2, o2);
#pragma unroll
    for (int c = 0; c < C; ++c) P[c][p] = o1[c] + o2[c];
  };
  if constexpr (kPacked) {
    // FP32 Euler: points in pairs (Gauss k, k + 1 of each face; interior p,
    // p + 1) through the packed Jacobian transposes; a face's lambda
    // combination is A + gx_k B with A and B formed once for both points
#pragma unroll
    for (int k = 0; k + 1 < NG; k += 2) {
      const float2 wx2 = make_float2(gw[k] * P_.inv_dx * scale, gw[k + 1] * P_.inv_dx * scale);
      const float2 wy2 = make_float2(gw[k] * P_.inv_dy * scale, gw[k + 1] * P_.inv_dy * scale);
      const float2 gx2 = make_float2(gx[k], gx[k + 1]);
      // one face: sign s of the own cell's side (-1: u^+ at the low face, +1:
      // u^- at the high face), the neighbour's offset, the moment m1 that
      // carries 1/2 and m2 that carries gx; writes the points p0, p0 + 1
      auto face_pair = [&](int p0, int dir, float sgn, int di, int dj, int m1, int m2) {
        float2 lf[C], U2[C], o2[C];
#pragma unroll
        for (int c = 0; c < C; ++c) {
          // -s (own - nb) terms: A = -s (L0 - L0nb) - (L1 + L1nb) / 2 (m1), B = -s (L2 - L2nb) (m2)
          const float A = -sgn * (LAM(c, 0, 0, 0) - LAM(c, 0, di, dj)) -
                          0.5f * (LAM(c, m1, 0, 0) + LAM(c, m1, di, dj));
          const float B = -sgn * (LAM(c, m2, 0, 0) - LAM(c, m2, di, dj));
          lf[c] = __fmul2_rn(dir == 0 ? wx2 : wy2, __ffma2_rn(gx2, bcast2(B), bcast2(A)));
          U2[c] = make_float2(P[c][p0], P[c][p0 + 1]);
        }
        flux_jt2_x2(P_.gas, U2, dir, lf, o2);
        const float h = dir == 0 ? hax : hay;
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const float2 r = __ffma2_rn(bcast2(sgn * h), lf[c], __fmul2_rn(bcast2(0.5f), o2[c]));
          P[c][p0] = r.x;
          P[c][p0 + 1] = r.y;
        }
      };
      face_pair(k, 0, -1.0f, -1, 0, 1, 2);           // x_{i-1/2}
      face_pair(NG + k, 0, 1.0f, 1, 0, 1, 2);        // x_{i+1/2}
      face_pair(2 * NG + k, 1, -1.0f, 0, -1, 2, 1);  // y_{j-1/2}
      face_pair(3 * NG + k, 1, 1.0f, 0, 1, 2, 1);    // y_{j+1/2}
    }
    if constexpr (NG % 2 == 1) face_point(NG - 1);
#pragma unroll
    for (int p = NF; p + 1 < NP; p += 2) {
      const int k0 = (p - NF) % NG, l0 = (p - NF) / NG, k1 = (p + 1 - NF) % NG, l1i = (p + 1 - NF) / NG;
      const float2 w2 = make_float2(gw[k0] * gw[l0], gw[k1] * gw[l1i]);
      float2 U2[C], la[C], lb[C], oa[C], ob[C];
#pragma unroll
      for (int c = 0; c < C; ++c) {
        U2[c] = make_float2(P[c][p], P[c][p + 1]);
        la[c] = __fmul2_rn(w2, bcast2(P_.inv_dx * scale * LAM(c, 1, 0, 0)));
        lb[c] = __fmul2_rn(w2, bcast2(P_.inv_dy * scale * LAM(c, 2, 0, 0)));
      }
      flux_jt2_x2(P_.gas, U2, 0, la, oa);
      flux_jt2_x2(P_.gas, U2, 1, lb, ob);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const float2 r = __fadd2_rn(oa[c], ob[c]);
        P[c][p] = r.x;
        P[c][p + 1] = r.y;
      }
    }
    if constexpr (NI % 2 == 1) interior_point(NP - 1);
  } else {
#pragma unroll
    for (int k = 0; k < NG; ++k) face_point(k);
#pragma unroll
    for (int p = NF; p < NP; ++p) interior_point(p);
  }
#undef LAM

  // adjoints of the 19 data, summed per target cell over the tile's own cells
  R Gl[C == 4 ? 4 : 1][19];
  if constexpr (C == 4) {
    if (own && hw) {
      R lamF[4][NF];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
#pragma unroll
        for (int p = 0; p < NF; ++p) lamF[c][p] = P[c][p];
#pragma unroll
        for (int k = 0; k < 19; ++k) Gl[c][k] = R(0);
      }
      hw_faces_euler_vjp<NG>(sm, ci, cj, P_.gam[0], P_.gam[1], P_.gam[2], P_.gam[3], P_.gam[4],
                             P_.eps, P_.gas, lamF, Gl);
    }
  }
  R* __restrict__ part = static_cast<R*>(a.G) + (size_t)(blockIdx.y * gridDim.x + blockIdx.x) * (C * 3 * BX * BY);
  if constexpr (kPacked) {
#pragma unroll
    for (int c = 0; c < C; c += 2) {
      float2 g2[19];
#pragma unroll
      for (int k = 0; k < 19; ++k) g2[k] = make_float2(0.0f, 0.0f);
      if (own) {
        float2 l2[NP];
#pragma unroll
        for (int p = 0; p < NP; ++p) l2[p] = make_float2(P[c][p], P[c + 1][p]);
        if (!hw) {
          p0_faces_T_x2<NG>(l2, g2);
        } else {
#pragma unroll
          for (int k = 0; k < 19; ++k) g2[k] = make_float2(Gl[c][k], Gl[c + 1][k]);
        }
        p0_interior_T_x2<NG>(&l2[NF], g2);
      }
      // both components' tile sums at once (each in the fixed order of the
      // single-component exchange)
#pragma unroll
      for (int k = 0; k < 19; ++k) sm.g2[k][cj][ci] = g2[k];
      __syncthreads();
      for (int t = tid; t < BX * BY; t += NT) {
        const int tx = t % BX - 1, ty = t / BX - 1;  // tile coordinates of the target
        float2 m[3] = {make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};
#pragma unroll
        for (int k = 0; k < 19; ++k) {
          const int sx = tx - data_dx(k), sy = ty - data_dy(k);
          if (sx >= 0 && sx < TX && sy >= 0 && sy < TY) {
            const int q = k < 9 ? 0 : (k < 14 ? 1 : 2);
            m[q] = __fadd2_rn(m[q], sm.g2[k][sy][sx]);
          }
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          part[(c * 3 + q) * (BX * BY) + t] = m[q].x;
          part[((c + 1) * 3 + q) * (BX * BY) + t] = m[q].y;
        }
      }
      __syncthreads();
    }
  } else {
    // the tile's sums of its cells' stencil adjoints g for component c, in a
    // fixed order (deterministic)
    auto exchange = [&](int c, const R* g) {
#pragma unroll
      for (int k = 0; k < 19; ++k) sm.g[k][cj][ci] = g[k];
      __syncthreads();
      for (int t = tid; t < BX * BY; t += NT) {
        const int tx = t % BX - 1, ty = t / BX - 1;  // tile coordinates of the target
        R m[3] = {R(0), R(0), R(0)};
#pragma unroll
        for (int k = 0; k < 19; ++k) {
          const int sx = tx - data_dx(k), sy = ty - data_dy(k);
          if (sx >= 0 && sx < TX && sy >= 0 && sy < TY) m[k < 9 ? 0 : (k < 14 ? 1 : 2)] += sm.g[k][sy][sx];
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) part[(c * 3 + q) * (BX * BY) + t] = m[q];
      }
      __syncthreads();
    };
#pragma unroll
    for (int c = 0; c < C; ++c) {
      R g[19];
#pragma unroll
      for (int k = 0; k < 19; ++k) g[k] = R(0);
      if (own) {
        if (!hw) {
          p0_faces_T<NG>(P[c], g);
        } else if constexpr (C == 1) {
          R d[19];
          gather19a(sm, c, ci, cj, d);
          hweno2d_faces_vjp<NG>(d, P_.gam, P_.eps, P[c], g);
        } else {
#pragma unroll
          for (int k = 0; k < 19; ++k) g[k] = Gl[c][k];
        }
        p0_interior_T<NG>(&P[c][NF], g);
      }
      exchange(c, g);
    }
  }
}

// ------------------------------------------------------------- kernels B, C

// m[c][q] += the partial sums kernel A's tiles wrote for cell (gi, gj).
template <typename R, int C>
__device__ __forceinline__ void part_sums(const Adj2DArgs& a, int gi, int gj, R (*m)[3]) {
  const R* __restrict__ part = static_cast<const R*>(a.G);
  int tx[3], px[3], ty[3], py[3];
  bool ux[3], uy[3];
  part_pairs(gi, a.nx, TX, tx, px, ux);
  part_pairs(gj, a.ny, TY, ty, py, uy);
  const int ntx = (a.nx + TX - 1) / TX;
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      if (!(uy[b] && ux[q])) continue;
      const R* pt = part + (size_t)(ty[b] * ntx + tx[q]) * (C * 3 * BX * BY) + py[b] * BX + px[q];
#pragma unroll
      for (int c = 0; c < C; ++c)
#pragma unroll
        for (int r = 0; r < 3; ++r) m[c][r] += pt[(c * 3 + r) * (BX * BY)];
    }
}

// mu = b lam + (stage 1: the adjoint of W0) + the partial sums, every
// component (the same sums as kernel B's).
template <typename R, int C>
__device__ __forceinline__ void mu_at(const Adj2DArgs& a, int gi, int gj, R (*m)[3]) {
  const size_t plane = (size_t)a.nx * a.ny, s = (size_t)gj * a.nx + gi;
  const R* __restrict__ lam = static_cast<const R*>(a.lam);
  const R bco = stage_b<R>(a.stage);
#pragma unroll
  for (int c = 0; c < C; ++c)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      m[c][q] = a.stage > 0 ? bco * lam[(3 * c + q) * plane + s] : R(0);
      if (a.stage == 1) m[c][q] += static_cast<const R*>(a.acc)[(3 * c + q) * plane + s];
    }
  part_sums<R, C>(a, gi, gj, m);
}

// Kernel B, one cell per thread: the adjoint of the stage input where Step 4
// changed nothing (mu itself; zero for the first moments of a troubled cell),
// and the adjoint of W0 (formed at stage 2: lam3 / 3 + 3 lam2 / 4; stage 1 adds it).
template <typename R, int C>
__global__ void __launch_bounds__(NT) adj2d_pass_kernel(Adj2DArgs a) {
  const int gi = blockIdx.x * TX + threadIdx.x % TX, gj = blockIdx.y * TY + threadIdx.x / TX;
  if (gi >= a.nx || gj >= a.ny) return;
  const size_t plane = (size_t)a.nx * a.ny, s = (size_t)gj * a.nx + gi;
  const bool t0 = a.flags[s] != 0;
  R* __restrict__ out = static_cast<R*>(a.lam_in);
  const R* __restrict__ lam = static_cast<const R*>(a.lam);
  R* __restrict__ acc = static_cast<R*>(a.acc);
  // every load first, then the stores.  av: stage 1 the adjoint of W0 that
  // stage 2 left; stage 2 lam3 / 3, lam3 (the adjoint of stage 3's output)
  // still being in this kernel's output buffer, which stage 3 only read
  R lv[C][3], m[C][3], av[C][3];
#pragma unroll
  for (int c = 0; c < C; ++c)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      lv[c][q] = lam[(3 * c + q) * plane + s];
      av[c][q] = a.stage == 1 ? acc[(3 * c + q) * plane + s]
                 : a.stage == 2 ? R(1.0 / 3.0) * out[(3 * c + q) * plane + s] : R(0);
    }
  const R bco = stage_b<R>(a.stage);
#pragma unroll
  for (int c = 0; c < C; ++c)
#pragma unroll
    for (int q = 0; q < 3; ++q) m[c][q] = (a.stage > 0 ? bco * lv[c][q] : R(0)) + (a.stage == 1 ? av[c][q] : R(0));
  part_sums<R, C>(a, gi, gj, m);
#pragma unroll
  for (int c = 0; c < C; ++c) {
    out[(3 * c) * plane + s] = m[c][0];
    out[(3 * c + 1) * plane + s] = t0 ? R(0) : m[c][1];
    out[(3 * c + 2) * plane + s] = t0 ? R(0) : m[c][2];
    if (a.stage == 2) {
#pragma unroll
      for (int q = 0; q < 3; ++q) acc[(3 * c + q) * plane + s] = av[c][q] + R(0.75) * lv[c][q];
    }
  }
}

// One tile of kernel C (a tile with a troubled cell in its 1-cell ring): adds
// the reverse of Step 4 (each troubled cell's modified moments back to the
// five data Step 1 read) to the adjoints kernel B wrote.
template <typename R, int C>
__device__ __noinline__ void fix_tile(const Adj2DArgs& a, int tile) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmemB<R, C>& sm = *reinterpret_cast<SmemB<R, C>*>(smem_raw);
  const int tid = threadIdx.x;
  const int nx = a.nx, ny = a.ny;
  const int ntx = (nx + TX - 1) / TX;
  const int bx0 = (tile % ntx) * TX, by0 = (tile / ntx) * TY;
  const size_t plane = (size_t)nx * ny;
  if (tid == 0) sm.nt = 0;
  __syncthreads();
  for (int k = tid; k < BX * BY; k += NT) {
    const int lx = k % BX, ly = k / BX;
    const size_t s = (size_t)bc_map(by0 - 1 + ly, ny, 0) * nx + bc_map(bx0 - 1 + lx, nx, 0);
    sm.fl[ly][lx] = a.flags[s] != 0;
    list_append(&sm.nt, sm.tl, k, sm.fl[ly][lx] != 0, BX * BY);
  }
  const AdjParams<R> P_(a);
  for (int k = tid; k < BX * BY; k += NT) {
    const int lx = k % BX, ly = k / BX;
    R m[C][3];
    mu_at<R, C>(a, bc_map(bx0 - 1 + lx, nx, 0), bc_map(by0 - 1 + ly, ny, 0), m);
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
      for (int q = 0; q < 3; ++q) sm.mu[c][q][ly][lx] = m[c][q];
  }
  const R* __restrict__ w = static_cast<const R*>(a.w);
  for (int k = tid; k < AX * AY; k += NT) {
    const int rx = k % AX, ry = k / AX;
    const size_t s = (size_t)bc_map(by0 - 2 + ry, ny, 0) * nx + bc_map(bx0 - 2 + rx, nx, 0);
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
      for (int m = 0; m < 3; ++m) sm.u[c][m][ry][rx] = w[(3 * c + m) * plane + s];
  }
  __syncthreads();
  // the troubled cells on consecutive threads (listed above)
  for (int q = tid; q < sm.nt; q += NT) {
    const int k = sm.tl[q];
    const int lx = k % BX, ly = k / BX;
    const int rx = lx + 1, ry = ly + 1;
    if constexpr (C == 1) {
      R g[5] = {R(0), R(0), R(0), R(0), R(0)};
      limit_first_moment_vjp(sm.u[0][0][ry][rx - 1], sm.u[0][0][ry][rx], sm.u[0][0][ry][rx + 1],
                             sm.u[0][1][ry][rx - 1], sm.u[0][1][ry][rx + 1], P_.gam, P_.eps,
                             sm.mu[0][1][ly][lx], g);
#pragma unroll
      for (int q = 0; q < 5; ++q) sm.cx[0][q][ly][lx] = g[q];
#pragma unroll
      for (int q = 0; q < 5; ++q) g[q] = R(0);
      limit_first_moment_vjp(sm.u[0][0][ry - 1][rx], sm.u[0][0][ry][rx], sm.u[0][0][ry + 1][rx],
                             sm.u[0][2][ry - 1][rx], sm.u[0][2][ry + 1][rx], P_.gam, P_.eps,
                             sm.mu[0][2][ly][lx], g);
#pragma unroll
      for (int q = 0; q < 5; ++q) sm.cy[0][q][ly][lx] = g[q];
    } else {
      limit_euler2d_vjp(sm, lx, ly, P_.gam[0], P_.gam[1], P_.gam[2], P_.gam[3], P_.gam[4], P_.eps,
                        P_.gas);
    }
  }
  __syncthreads();
  const int ci = tid % TX, cj = tid / TX;
  const int gi = bx0 + ci, gj = by0 + cj;
  if (gi >= nx || gj >= ny) return;
  const int lx = ci + 1, ly = cj + 1;
  const bool fl = sm.fl[ly][lx - 1] || sm.fl[ly][lx + 1] || sm.fl[ly - 1][lx] || sm.fl[ly + 1][lx] ||
                  sm.fl[ly][lx];
  if (!fl) return;
  const size_t s = (size_t)gj * nx + gi;
  R* __restrict__ out = static_cast<R*>(a.lam_in);
#pragma unroll
  for (int c = 0; c < C; ++c) {
    R g0 = R(0), g1 = R(0), g2 = R(0);
    if (sm.fl[ly][lx - 1]) { g0 += sm.cx[c][2][ly][lx - 1]; g1 += sm.cx[c][4][ly][lx - 1]; }
    if (sm.fl[ly][lx + 1]) { g0 += sm.cx[c][0][ly][lx + 1]; g1 += sm.cx[c][3][ly][lx + 1]; }
    if (sm.fl[ly - 1][lx]) { g0 += sm.cy[c][2][ly - 1][lx]; g2 += sm.cy[c][4][ly - 1][lx]; }
    if (sm.fl[ly + 1][lx]) { g0 += sm.cy[c][0][ly + 1][lx]; g2 += sm.cy[c][3][ly + 1][lx]; }
    if (sm.fl[ly][lx]) g0 += sm.cx[c][1][ly][lx] + sm.cy[c][1][ly][lx];
    out[(3 * c) * plane + s] += g0;
    out[(3 * c + 1) * plane + s] += g1;
    out[(3 * c + 2) * plane + s] += g2;
  }
}

// Kernel C: a grid-stride loop over the tiles kernel A listed (tiles without a
// troubled cell in their ring have nothing to add).
template <typename R, int C>
__global__ void __launch_bounds__(NT) adj2d_fix_kernel(Adj2DArgs a) {
  const int count = a.tile_list[0];
  for (int i = blockIdx.x; i < count; i += gridDim.x) {
    fix_tile<R, C>(a, a.tile_list[1 + i]);
    __syncthreads();
  }
}

template <typename R, int C, int NG>
cudaError_t launch_t(const Adj2DArgs& a, cudaStream_t s) {
  const dim3 grid((unsigned)((a.nx + TX - 1) / TX), (unsigned)((a.ny + TY - 1) / TY));
  cudaError_t e = cudaMemsetAsync(a.tile_list, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  Adj2DArgs b = a;
  CUtensorMap um, lm;
  b.tma = encode_box_map(a.w, a.nx, a.ny, 3 * C, (int)sizeof(R), AXA, AY, &um) &&
          encode_box_map(a.lam, a.nx, a.ny, 3 * C, (int)sizeof(R), LXA, BY, &lm);
  adj2d_points_kernel<R, C, NG><<<grid, NT, sizeof(SmemA<R, C>), s>>>(b, um, lm);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  adj2d_pass_kernel<R, C><<<grid, NT, 0, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const unsigned ntile = grid.x * grid.y, gc = 2u * (unsigned)nsm;
  adj2d_fix_kernel<R, C><<<ntile < gc ? ntile : gc, NT, sizeof(SmemB<R, C>), s>>>(a);
  return cudaGetLastError();
}

template <typename R, int C, int NG>
cudaError_t prepare_t() {
  cudaError_t e = cudaFuncSetAttribute(adj2d_points_kernel<R, C, NG>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(SmemA<R, C>));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(adj2d_fix_kernel<R, C>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(SmemB<R, C>));
}

}  // namespace

void finish_adj2d_args(Adj2DArgs& a) {
  for (int k = 0; k < 5; ++k) a.f32[k] = (float)a.gam[k];
  a.f32[5] = (float)a.eps;
  a.f32[6] = (float)a.gas;
  a.f32[7] = (float)(1.0 / a.dx);
  a.f32[8] = (float)(1.0 / a.dy);
}

cudaError_t prepare_adj2d(int system, int fp64, int ng) {
  if (system == 0) {
    if (fp64) return ng == 2 ? prepare_t<double, 1, 2>() : prepare_t<double, 1, 3>();
    return ng == 2 ? prepare_t<float, 1, 2>() : prepare_t<float, 1, 3>();
  }
  if (fp64) return ng == 2 ? prepare_t<double, 4, 2>() : prepare_t<double, 4, 3>();
  return ng == 2 ? prepare_t<float, 4, 2>() : prepare_t<float, 4, 3>();
}

cudaError_t launch_adj2d(const Adj2DArgs& a, cudaStream_t s) {
  if (a.system == 0) {
    if (a.fp64) return a.ng == 2 ? launch_t<double, 1, 2>(a, s) : launch_t<double, 1, 3>(a, s);
    return a.ng == 2 ? launch_t<float, 1, 2>(a, s) : launch_t<float, 1, 3>(a, s);
  }
  if (a.fp64) return a.ng == 2 ? launch_t<double, 4, 2>(a, s) : launch_t<double, 4, 3>(a, s);
  return a.ng == 2 ? launch_t<float, 4, 2>(a, s) : launch_t<float, 4, 3>(a, s);
}

}  // namespace hw
