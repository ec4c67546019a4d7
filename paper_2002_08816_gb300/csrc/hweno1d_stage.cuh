// The body of one third-order TVD Runge-Kutta stage of the 1D hybrid HWENO
// scheme (Zhao & Qiu, arXiv:2002.08816, Sec. 2.1) on one tile, shared by the
// per-stage kernel and the persistent kernel (hweno1d.cu).
//
// A CTA of NTH + 32 threads owns T = NTH - 6 consecutive cells: NTH cell
// threads and one scalar warp.  The cell threads stage the cells plus a
// 3-cell halo of the stage input in shared memory (coalesced loads of each
// structure-of-arrays row), then, all on chip:
//   1. (scalar warp, concurrently with steps 2-3 of the cell threads, all in
//      FP64) alpha = max |f'(ubar)| over the maxima the producer of the stage
//      input left in kAlphaSlots FP64 slots (global Lax-Friedrichs flux);
//      stage 1 also turns alpha into dt = CFL dx / alpha, clipped to t_final;
//      the lead tile records dt and, in stage 3, the time.  The per-cell
//      wave speeds are bulk arithmetic in the kernel's precision; their
//      maximum, dt, the clipping and the time are FP64, off the cell
//      threads' critical path (a dependent FP64 operation costs tens of
//      cycles on GB300, a division hundreds);
//   2. KXRCF flags and the modified first moments (Step 1) for the cells and
//      2 halo cells per side, in characteristic fields for Euler (out-of-line
//      work of the troubled lanes); an FP32 kernel decides a flag in FP32 when
//      its rounding-error bound allows and by an error-free float-pair
//      evaluation otherwise, so flags equal the FP64 decision off the threshold;
//   3. interface values (Steps 2.1/2.2) for the cells and 1 halo cell per
//      side: linear p0 unless a cell of S0 = {i-1, i, i+1} is troubled;
//   4. for the own cells: interior Gauss-Lobatto values (Step 2.3), the
//      Lax-Friedrichs fluxes at x_{i-+1/2}, F_i, the right-hand sides of
//      Eq. (odeH) and the Runge-Kutta combination of Eq. (RK);
//   5. the maximum wave speed of the output, folded by FP64 atomic max into
//      the tile's one of kAlphaSlots slots that the next stage reads for its alpha
//      (warp by warp, or after a CTA reduction on large grids), the troubled
//      count and the status bits (non-finite, non-physical).
// The limited stage input is what the RK combination uses (the first moment
// of a troubled cell is modified in the state, as a DG limiter would).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "hweno1d_recon.cuh"
#include "hweno_device.cuh"
#include "hweno.h"
#include "hweno_internal.h"

namespace hw {
namespace s1d {

constexpr int H = 3;  // halo cells per side
// grids of at most this many tiles fold the wave-speed maxima warp by warp
constexpr int kWarpAtomicTiles = 2048;

// Named barriers: kBarCells among the NTH cell threads only; kBarAll for the
// cell threads and the scalar warp (which only arrives) before step 4.
constexpr int kBarCells = 1, kBarAll = 2;
__device__ __forceinline__ void bar_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive(int id, int count) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// A load of data another CTA may have written earlier in the same launch
// (the persistent kernel): through L2, never from a stale L1 line.
template <typename T>
__device__ __forceinline__ T ldx(const T* p) {
  return __ldcg(p);
}

template <typename R, int C, int NTH>
struct Smem1D {
  static constexpr int T = NTH - 2 * H, NW = NTH / 32;
  R u[C][2][T + 2 * H];  // stage input, cells base-3 .. base+T+2
  R vl[C][T + 4];        // modified first moments, cells base-2 .. base+T+1
  R fm[C][T + 2];        // u^+_{i-1/2}, cells base-1 .. base+T
  R fp[C][T + 2];        // u^-_{i+1/2}
  R ffm[C][T + 2];       // f(u^+_{i-1/2})
  R ffp[C][T + 2];       // f(u^-_{i+1/2})
  uint8_t fl[T + 4];     // flags, cells base-2 .. base+T+1
  R red[NW];
  int cnt[NW];
  R alpha, dt;           // from the scalar warp, in the kernel's precision
};

template <typename R, int C>
__device__ __forceinline__ void phys_flux(R gas, const R* U, R* F) {
  if constexpr (C == 1) {
    F[0] = R(0.5) * U[0] * U[0];
  } else {
    // f(rho, m, E) of Eq. (euler1); FP32 uses an approximate reciprocal of rho
    const R rho = U[0], m = U[1], E = U[2];
    const R mu = sizeof(R) == 4 ? m * fast_rcp(rho) : m / rho;
    const R p = (gas - R(1)) * (E - R(0.5) * m * mu);
    F[0] = m;
    F[1] = m * mu + p;
    F[2] = mu * (E + p);
  }
}

// max |f'(u)| at a cell average, in the kernel's precision (NaN when the
// state is not physical); the maxima are reduced in FP64.
template <typename R, int C>
__device__ __forceinline__ R wave_speed(R gas, const R* U) {
  if constexpr (C == 1) {
    return fabs(U[0]);
  } else {
    return euler1d_speed_r<R>(gas, U[0], U[1], U[2]);
  }
}

// Euler troubled-cell work for one cell (Remark 2: the characteristic fields
// of the Jacobian at a cell average).  Out of line, with scalar arguments and
// results: compiled once per precision, so every tile size runs the same
// instructions on a cell (the execution choice cannot change a result through
// a multiply-add the optimiser contracts differently in another
// instantiation), the kernel body keeps few registers, and no array of the
// caller has its address taken.  The three fields are independent chains
// that the one thread interleaves.
template <typename R>
struct ConsVec {
  R v[3];
};
template <typename R>
struct ConsFaces {
  R L[3], Rt[3], fL[3], fR[3];
};

// Step 1 for cell i: the modified first moments, from the averages of cells
// i-1, i, i+1 (am*, a0*, ap*) and the first moments of i-1, i+1 (vm*, vp*),
// limited field by field and mapped back to the conserved variables.
template <typename R>
__device__ __noinline__ ConsVec<R> char_limit(R gas, R g0, R g1, R g2, R eps, R am0, R am1, R am2,
                                              R a00, R a01, R a02, R ap0, R ap1, R ap2, R vm0,
                                              R vm1, R vm2, R vp0, R vp1, R vp2) {
  const R U[3] = {a00, a01, a02};
  const R gam[3] = {g0, g1, g2};
  R Rm[3][3], Lm[3][3];
  Euler1D<R>::eigen(gas, U, Rm, Lm);
  R q[3];
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    const R* l = Lm[f];
    q[f] = limit_first_moment(l[0] * am0 + l[1] * am1 + l[2] * am2,
                              l[0] * a00 + l[1] * a01 + l[2] * a02,
                              l[0] * ap0 + l[1] * ap1 + l[2] * ap2,
                              l[0] * vm0 + l[1] * vm1 + l[2] * vm2,
                              l[0] * vp0 + l[1] * vp1 + l[2] * vp2, gam, eps);
  }
  ConsVec<R> o;
#pragma unroll
  for (int c = 0; c < 3; ++c) o.v[c] = Rm[c][0] * q[0] + Rm[c][1] * q[1] + Rm[c][2] * q[2];
  return o;
}

// Step 2.1 for cell i: the HWENO values at x_{i-1/2} and x_{i+1/2} from the
// averages of cells i-1, i, i+1 and their modified first moments (vm*, v0*,
// vp*), in the characteristic fields of the state (b0, b1, b2), mapped back
// to the conserved variables, with their physical fluxes.
template <typename R>
__device__ __noinline__ ConsFaces<R> char_faces(R gas, R g0, R g1, R g2, R eps, R b0, R b1, R b2,
                                                R am0, R am1, R am2, R a00, R a01, R a02, R ap0,
                                                R ap1, R ap2, R vm0, R vm1, R vm2, R v00, R v01,
                                                R v02, R vp0, R vp1, R vp2) {
  const R U[3] = {b0, b1, b2};
  const R gam[3] = {g0, g1, g2};
  R Rm[3][3], Lm[3][3];
  Euler1D<R>::eigen(gas, U, Rm, Lm);
  R cl[3], cr[3];
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    const R* l = Lm[f];
    hweno_faces(l[0] * am0 + l[1] * am1 + l[2] * am2, l[0] * a00 + l[1] * a01 + l[2] * a02,
                l[0] * ap0 + l[1] * ap1 + l[2] * ap2, l[0] * vm0 + l[1] * vm1 + l[2] * vm2,
                l[0] * v00 + l[1] * v01 + l[2] * v02, l[0] * vp0 + l[1] * vp1 + l[2] * vp2, gam,
                eps, cl[f], cr[f]);
  }
  ConsFaces<R> o;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    o.L[c] = Rm[c][0] * cl[0] + Rm[c][1] * cl[1] + Rm[c][2] * cl[2];
    o.Rt[c] = Rm[c][0] * cr[0] + Rm[c][1] * cr[1] + Rm[c][2] * cr[2];
  }
  phys_flux<R, 3>(gas, o.L, o.fL);
  phys_flux<R, 3>(gas, o.Rt, o.fR);
  return o;
}

// Step 2 at the interfaces of the cell in slot e = k + 2 of sm.u (k = 0 is
// the first halo cell that needs them): the traces u^+_{i-1/2}, u^-_{i+1/2}
// (linear p0, Step 2.2, or Step 2.1 when the stencil S0 holds a troubled
// cell; Euler in the characteristic fields of Remark 2) into sm.fm, sm.fp,
// and their physical fluxes into sm.ffm, sm.ffp.
template <typename R, int C, int NTH>
__device__ __forceinline__ void faces_of_cell(Smem1D<R, C, NTH>& sm, int k, R gas, const R* gam,
                                              R eps, int variant) {
  const int e = k + 2;  // sm.u index e; sm.vl / sm.fl index of cell e is e - 1
  const bool hw = sm.fl[k] | sm.fl[k + 1] | sm.fl[k + 2];
  R L[C], Rt[C], fL[C], fR[C];
  if (!hw || C == 1) {
    if (!hw) {
      if constexpr (C == 3 && sizeof(R) == 4) {
        // FP32 Euler: density and momentum as a pair through the packed map
        float2 l2, r2;
        auto p2 = [&](int m, int j) { return make_float2(m == 0 ? sm.u[0][0][j] : sm.vl[0][j],
                                                         m == 0 ? sm.u[1][0][j] : sm.vl[1][j]); };
        linear_faces_x2(p2(0, e - 1), p2(0, e), p2(0, e + 1), p2(1, e - 2), p2(1, e - 1),
                        p2(1, e), l2, r2);
        L[0] = l2.x; L[1] = l2.y; Rt[0] = r2.x; Rt[1] = r2.y;
        linear_faces(sm.u[2][0][e - 1], sm.u[2][0][e], sm.u[2][0][e + 1], sm.vl[2][e - 2],
                     sm.vl[2][e - 1], sm.vl[2][e], L[2], Rt[2]);
      } else {
#pragma unroll
        for (int c = 0; c < C; ++c)
          linear_faces(sm.u[c][0][e - 1], sm.u[c][0][e], sm.u[c][0][e + 1], sm.vl[c][e - 2],
                       sm.vl[c][e - 1], sm.vl[c][e], L[c], Rt[c]);
      }
    } else {
      hweno_faces(sm.u[0][0][e - 1], sm.u[0][0][e], sm.u[0][0][e + 1], sm.vl[0][e - 2],
                  sm.vl[0][e - 1], sm.vl[0][e], gam, eps, L[0], Rt[0]);
    }
    phys_flux<R, C>(gas, L, fL);
    phys_flux<R, C>(gas, Rt, fR);
  } else {
    // Default: both faces in the fields of the cell average (Remark 2).
    // Variant: u^+_{i-1/2} in the fields of the mean of the averages of
    // cells i-1, i; u^-_{i+1/2} in those of cells i, i+1.
    const bool mean = variant & HWENO_VARIANT_MEAN_EIGEN;
    for (int side = 0; side < (mean ? 2 : 1); ++side) {
      R B[3];
#pragma unroll
      for (int c = 0; c < 3; ++c)
        B[c] = !mean ? sm.u[c][0][e]
               : side ? R(0.5) * (sm.u[c][0][e] + sm.u[c][0][e + 1])
                      : R(0.5) * (sm.u[c][0][e - 1] + sm.u[c][0][e]);
      const ConsFaces<R> o = char_faces<R>(
          gas, gam[0], gam[1], gam[2], eps, B[0], B[1], B[2], sm.u[0][0][e - 1],
          sm.u[1][0][e - 1], sm.u[2][0][e - 1], sm.u[0][0][e], sm.u[1][0][e], sm.u[2][0][e],
          sm.u[0][0][e + 1], sm.u[1][0][e + 1], sm.u[2][0][e + 1], sm.vl[0][e - 2],
          sm.vl[1][e - 2], sm.vl[2][e - 2], sm.vl[0][e - 1], sm.vl[1][e - 1], sm.vl[2][e - 1],
          sm.vl[0][e], sm.vl[1][e], sm.vl[2][e]);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        if (!mean || side == 0) {
          L[c] = o.L[c];
          fL[c] = o.fL[c];
        }
        if (!mean || side == 1) {
          Rt[c] = o.Rt[c];
          fR[c] = o.fR[c];
        }
      }
    }
  }
#pragma unroll
  for (int c = 0; c < C; ++c) {
    sm.fm[c][k] = L[c];
    sm.fp[c][k] = Rt[c];
    sm.ffm[c][k] = fL[c];
    sm.ffp[c][k] = fR[c];
  }
}

// Step 2.3 of the cell in sm.u slot e (FP32 Euler: density and momentum as a
// pair through the packed map).
template <typename R, int C, int NTH>
__device__ __forceinline__ void interior_values(const Smem1D<R, C, NTH>& sm, int e, R* gm, R* gp) {
  if constexpr (C == 3 && sizeof(R) == 4) {
    auto p2 = [&](int m, int j) { return make_float2(m == 0 ? sm.u[0][0][j] : sm.vl[0][j],
                                                     m == 0 ? sm.u[1][0][j] : sm.vl[1][j]); };
    float2 m2, q2;
    linear_interior_x2(p2(0, e - 1), p2(0, e), p2(0, e + 1), p2(1, e - 2), p2(1, e - 1), p2(1, e),
                       m2, q2);
    gm[0] = m2.x; gm[1] = m2.y; gp[0] = q2.x; gp[1] = q2.y;
    linear_interior(sm.u[2][0][e - 1], sm.u[2][0][e], sm.u[2][0][e + 1], sm.vl[2][e - 2],
                    sm.vl[2][e - 1], sm.vl[2][e], gm[2], gp[2]);
  } else {
#pragma unroll
    for (int c = 0; c < C; ++c)
      linear_interior(sm.u[c][0][e - 1], sm.u[c][0][e], sm.u[c][0][e + 1], sm.vl[c][e - 2],
                      sm.vl[c][e - 1], sm.vl[c][e], gm[c], gp[c]);
  }
}

// Eq. (odeH) for the own cell of thread tid (sm.u slot e = tid + 3): the
// interior Gauss-Lobatto values (Step 2.3) and their fluxes, the
// Lax-Friedrichs fluxes at x_{i-+1/2} (each from the traces and trace fluxes
// the two cells beside the interface stored, so both cells use the same
// number and the averages stay conservative), the four-point Gauss-Lobatto
// F_i and the two right-hand sides
//   Lu = -(fhat_{i+1/2} - fhat_{i-1/2}) / dx,
//   Lv = (F_i - (fhat_{i-1/2} + fhat_{i+1/2}) / 2) / dx.
template <typename R, int C, int NTH>
__device__ __forceinline__ void rhs_of_cell(const Smem1D<R, C, NTH>& sm, int tid, R gas, R alpha,
                                            R inv_dx, R* Lu, R* Lv) {
  const int e = tid + H, k = tid + 1;  // sm.u slot; sm.fm/fp slot of the cell
  const R half_alpha = R(0.5) * alpha;
  R gm[C], gp[C], f2[C], f3[C];
  interior_values<R, C, NTH>(sm, e, gm, gp);
  phys_flux<R, C>(gas, gm, f2);
  phys_flux<R, C>(gas, gp, f3);
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const R ql = R(0.5) * (sm.ffp[c][k - 1] + sm.ffm[c][k]) -
                 half_alpha * (sm.fm[c][k] - sm.fp[c][k - 1]);
    const R qr = R(0.5) * (sm.ffp[c][k] + sm.ffm[c][k + 1]) -
                 half_alpha * (sm.fm[c][k + 1] - sm.fp[c][k]);
    // four-point Gauss-Lobatto F_i; the end points are the cell's own traces
    const R F = R(1.0 / 12.0) * (sm.ffm[c][k] + sm.ffp[c][k]) + R(5.0 / 12.0) * (f2[c] + f3[c]);
    Lu[c] = -(qr - ql) * inv_dx;
    Lv[c] = (F - R(0.5) * (ql + qr)) * inv_dx;
  }
}

// Eq. (odeH) as above, split by its dependence on alpha: the Lax-Friedrichs
// fluxes are linear in alpha, so Lu = L0u - alpha Du and Lv = L0v - alpha Dv
// with L0 from the traces' fluxes and F_i and D from the trace jumps.  A
// caller that learns alpha late computes the four parts first.
template <typename R, int C, int NTH>
__device__ __forceinline__ void rhs_parts_of_cell(const Smem1D<R, C, NTH>& sm, int tid, R gas,
                                                  R inv_dx, R* L0u, R* Du, R* L0v, R* Dv) {
  const int e = tid + H, k = tid + 1;  // sm.u slot; sm.fm/fp slot of the cell
  R gm[C], gp[C], f2[C], f3[C];
  interior_values<R, C, NTH>(sm, e, gm, gp);
  phys_flux<R, C>(gas, gm, f2);
  phys_flux<R, C>(gas, gp, f3);
#pragma unroll
  for (int c = 0; c < C; ++c) {
    // central parts and jumps of the fluxes at x_{i-1/2} and x_{i+1/2}
    const R cl = R(0.5) * (sm.ffp[c][k - 1] + sm.ffm[c][k]);
    const R cr = R(0.5) * (sm.ffp[c][k] + sm.ffm[c][k + 1]);
    const R jl = sm.fm[c][k] - sm.fp[c][k - 1];
    const R jr = sm.fm[c][k + 1] - sm.fp[c][k];
    const R F = R(1.0 / 12.0) * (sm.ffm[c][k] + sm.ffp[c][k]) + R(5.0 / 12.0) * (f2[c] + f3[c]);
    L0u[c] = -(cr - cl) * inv_dx;
    Du[c] = R(-0.5) * (jr - jl) * inv_dx;
    L0v[c] = (F - R(0.5) * (cl + cr)) * inv_dx;
    Dv[c] = R(-0.25) * (jl + jr) * inv_dx;
  }
}

// One stage on one tile of T = NTH - 6 cells, by a CTA of NTH + 32 threads.  The
// per-stage kernel calls it once; the persistent kernel calls it for each of
// its tiles of each stage, between grid barriers, so every load of data
// produced in the same launch goes through L2 (ldx).
template <typename R, int C, bool BATCH, int NTH>
__device__ __forceinline__ void stage1d_tile(Stage1DArgs a, const int tile, Smem1D<R, C, NTH>& sm) {
  constexpr int T = NTH - 2 * H, NT = NTH, NW = NTH / 32;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  int n = a.n;
  int base = tile * T;
  int inst = 0;
  bool lead = tile == 0;  // the tile that keeps the (instance's) time
  if constexpr (BATCH) {
    // a batch of independent instances: this tile's instance and first cell
    inst = a.tile_inst[tile];
    base = a.tile_base[tile];
    const BatchInst& bi = a.binst[inst];
    n = bi.n;
    lead = base == 0;
    const long long off = bi.off;
    a.w = static_cast<const R*>(a.w) + off;
    if (a.u0) a.u0 = static_cast<const R*>(a.u0) + off;
    a.out = static_cast<R*>(a.out) + off;
    if (a.lim_out) a.lim_out = static_cast<R*>(a.lim_out) + off;
    if (a.flags_out) a.flags_out += off / (2 * C);
    a.a_in = static_cast<const double*>(a.a_in) + inst;
    a.nin = 1;
    a.inv_dx = bi.inv_dx;
    a.h = bi.h;
    a.cfl_dx = bi.cfl_dx;
    a.hthr = bi.hthr_f;
    a.hthr_lo = bi.hthr_lo_f;
    a.f32[5] = bi.inv_dx_f;
    a.f32[6] = bi.cfl_dx_f;
  }
  const R* __restrict__ w = static_cast<const R*>(a.w);

  // The producer of the stage input may still be finishing (programmatic
  // dependent launch): wait for its completion and memory before any read.
  asm volatile("griddepcontrol.wait;" ::: "memory");

  // Parameters in the kernel's precision (FP32 copies made on the host).
  R gam[3], eps, gas, inv_dx;
  if constexpr (sizeof(R) == 4) {
    gam[0] = a.f32[0]; gam[1] = a.f32[1]; gam[2] = a.f32[2];
    eps = a.f32[3]; gas = a.f32[4]; inv_dx = a.f32[5];
  } else {
    gam[0] = a.gam[0]; gam[1] = a.gam[1]; gam[2] = a.gam[2];
    eps = a.eps; gas = a.gas; inv_dx = a.inv_dx;
  }

  if (tid >= NT) {
    // ---- the scalar warp: alpha, dt and the time, in FP64 ----------------
    // its own loads go out first, concurrently with the cell threads' tile
    const unsigned long long* a_in = static_cast<const unsigned long long*>(a.a_in);
    unsigned long long am = 0ull;  // bit patterns of non-negative doubles: the
                                   // integer order is the numeric order
    for (int k = lane; k < a.nin; k += 32) {
      const unsigned long long v = ldx(a_in + k);
      am = v > am ? v : am;
    }
    double rem = 0.0, dt = 0.0, tf = 0.0, t = 0.0;
    unsigned last = 0u;
    unsigned long long steps = 0ull;
    const bool keep = a.stage == 3 && lead && lane == 0;  // the time keeper
    if constexpr (BATCH) {
      const BatchScalars& bs = a.bsc[inst];
      if (a.stage == 1) rem = ldx(&bs.rem);
      else if (a.stage > 1) dt = ldx(&bs.dt);
      if (keep) {
        last = ldx(&bs.last);
        t = ldx(&bs.t);
      }
    } else {
      if (a.stage == 1) rem = ldx(&a.sc->rem);
      else if (a.stage > 1) dt = ldx(&a.sc->dt);
      if (keep) {
        last = ldx(&a.sc->last);
        t = ldx(&a.sc->t);
      }
    }
    if (keep) {
      tf = ldx(&a.sc->t_final);
      steps = ldx(&a.sc->steps);
    }
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long v = __shfl_xor_sync(0xffffffffu, am, o);
      am = v > am ? v : am;
    }
    asm volatile("griddepcontrol.launch_dependents;");
    const double alpha = __longlong_as_double((long long)am);
    if (a.stage == 1) {
      // dt = CFL dx / alpha(u^n), clipped to the remaining time (the clipped
      // step is the last one and ends exactly at t_final); 0 once t_final
      // has been reached
      dt = a.cfl_dx / alpha;
      last = 0u;
      if (rem <= 0.0) {
        dt = 0.0;
      } else if (dt >= rem) {
        dt = rem;
        last = 1u;
      }
      if (!(alpha > 0.0) || !isfinite(dt)) dt = 0.0;
      if (lead && lane == 0) {
        if constexpr (BATCH) {
          BatchScalars& bs = a.bsc[inst];
          bs.dt = dt;
          bs.dt_f = (float)dt;
          bs.last = last;
        } else {
          a.sc->dt = dt;
          a.sc->dt_f = (float)dt;
          a.sc->last = last;
        }
      }
    }
    if (lane == 0) {
      sm.alpha = R(alpha);
      sm.dt = R(dt);
    }
    if (a.stage > 0 && dt > 0.0) {
      // the slots of the stage after next (read two stages ago, now free)
      if constexpr (BATCH) {
        if (a.a_zero && lead && lane == 0) static_cast<double*>(a.a_zero)[inst] = 0.0;
      } else {
        if (a.a_zero && tile == 0)
          for (int k = lane; k < kAlphaSlots; k += 32) static_cast<double*>(a.a_zero)[k] = 0.0;
      }
      if (keep) {  // stage 3 of the lead tile: the step is complete
        const double tn = last ? tf : t + dt;
        const double r = tf > 0.0 ? tf - tn : (double)INFINITY;
        if constexpr (BATCH) {
          BatchScalars& bs = a.bsc[inst];
          bs.t = tn;
          bs.rem = r;
          bs.rem_f = (float)r;
          if (inst == 0) a.sc->steps = steps + 1ull;
        } else {
          a.sc->t = tn;
          a.sc->rem = r;
          a.sc->rem_f = (float)r;
          a.sc->steps = steps + 1ull;
        }
      }
    }
    bar_arrive(kBarAll, NT + 32);
    return;
  }

  // ---- the cell threads --------------------------------------------------
  // 2. in one round trip: the tile-plus-halo element of each thread and, in
  //    stages 2 and 3, the modified u^n of its own cell
  R u0c[C][2];
  if (a.stage >= 2 && tid < T && base + tid < n) {
    const R* u0 = static_cast<const R*>(a.u0);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      u0c[c][0] = ldx(u0 + (2 * c + 0) * n + base + tid);
      u0c[c][1] = ldx(u0 + (2 * c + 1) * n + base + tid);
    }
  }
  if (tid < T + 2 * H) {
    if (a.bc == 2) {
      bool mir;
      const int g = bc_map_wall(base - H + tid, n, &mir);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        sm.u[c][0][tid] = ldx(w + (2 * c + 0) * n + g) * (mir ? R(mirror_sign(c, 0)) : R(1));
        sm.u[c][1][tid] = ldx(w + (2 * c + 1) * n + g) * (mir ? R(mirror_sign(c, 1)) : R(1));
      }
    } else {
      const int g = bc_map(base - H + tid, n, a.bc);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        sm.u[c][0][tid] = ldx(w + (2 * c + 0) * n + g);
        sm.u[c][1][tid] = ldx(w + (2 * c + 1) * n + g);
      }
    }
  }
  bar_sync(kBarCells, NT);
  // the next stage's CTAs may be scheduled now; they wait for this grid above
  asm volatile("griddepcontrol.launch_dependents;");

  // 3. troubled cells and modified first moments (Step 1), cells base-2 ..
  //    base+T+1; Euler limits in the characteristic fields of the cell
  //    average (Remark 2)
  int flag = 0;
  if (tid < T + 4) {
    const int k = tid, e = k + 1;
    const double h = a.h;
    const float hthr = a.hthr, hthr_lo = a.hthr_lo;
    if (a.mode == 1) {
      flag = 1;
    } else if (a.mode == 2) {
      flag = 0;
    } else if constexpr (C == 1) {
      const R u0 = sm.u[0][0][e];
      flag = kxrcf_troubled(sm.u[0][0][e - 1], u0, sm.u[0][0][e + 1], sm.u[0][1][e - 1],
                            sm.u[0][1][e], sm.u[0][1][e + 1], u0 >= R(0), h, a.thr, hthr, hthr_lo);
    } else {
      const bool left = inflow_left(sm.u[0][0][e], sm.u[1][0][e]);
      flag = kxrcf_troubled(sm.u[0][0][e - 1], sm.u[0][0][e], sm.u[0][0][e + 1],
                            sm.u[0][1][e - 1], sm.u[0][1][e], sm.u[0][1][e + 1], left, h, a.thr,
                            hthr, hthr_lo) ||
             kxrcf_troubled(sm.u[2][0][e - 1], sm.u[2][0][e], sm.u[2][0][e + 1],
                            sm.u[2][1][e - 1], sm.u[2][1][e], sm.u[2][1][e + 1], left, h, a.thr,
                            hthr, hthr_lo);
    }
    sm.fl[k] = (uint8_t)flag;
    if (!flag) {
#pragma unroll
      for (int c = 0; c < C; ++c) sm.vl[c][k] = sm.u[c][1][e];
    } else if constexpr (C == 1) {
      sm.vl[0][k] = limit_first_moment(sm.u[0][0][e - 1], sm.u[0][0][e], sm.u[0][0][e + 1],
                                       sm.u[0][1][e - 1], sm.u[0][1][e + 1], gam, eps);
    } else {
      const ConsVec<R> o = char_limit<R>(
          gas, gam[0], gam[1], gam[2], eps, sm.u[0][0][e - 1], sm.u[1][0][e - 1],
          sm.u[2][0][e - 1], sm.u[0][0][e], sm.u[1][0][e], sm.u[2][0][e], sm.u[0][0][e + 1],
          sm.u[1][0][e + 1], sm.u[2][0][e + 1], sm.u[0][1][e - 1], sm.u[1][1][e - 1],
          sm.u[2][1][e - 1], sm.u[0][1][e + 1], sm.u[1][1][e + 1], sm.u[2][1][e + 1]);
#pragma unroll
      for (int c = 0; c < 3; ++c) sm.vl[c][k] = o.v[c];
    }
  }
  bar_sync(kBarCells, NT);

  // 4. interface values (Steps 2.1, 2.2) and their physical fluxes, cells
  //    base-1 .. base+T
  if (tid < T + 2) faces_of_cell<R, C, NTH>(sm, tid, gas, gam, eps, a.variant);
  // alpha and dt from the scalar warp; a zero dt (t_final reached) is
  // uniform over the grid (the instance), and the stage then writes nothing
  bar_sync(kBarAll, NT + 32);
  const R alpha = sm.alpha, dt = sm.dt;
  if (a.stage > 0 && !(dt > R(0))) return;

  // 5. own cells: fluxes, F_i, right-hand side, RK combination
  const int i = base + tid;
  const bool own = tid < T && i < n;
  int myflag = 0;
  R speed = R(0);
  unsigned bad = 0;
  if (own) {
    const int e = tid + H;  // sm.u index
    myflag = sm.fl[tid + 2];
    R Lus[C], Lvs[C];
    rhs_of_cell<R, C, NTH>(sm, tid, gas, alpha, inv_dx, Lus, Lvs);
    R Uo[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const R Lu = Lus[c], Lv = Lvs[c];
      const R wu = sm.u[c][0][e];
      // the stage input the combination uses: first moments as modified by
      // Step 1 (stored, the default), or unmodified (variant)
      const R wvm = sm.vl[c][e - 1];
      const R wv = (a.variant & HWENO_VARIANT_RAW_COMBINE) ? sm.u[c][1][e] : wvm;
      R ou, ov;
      if (a.stage == 0) {
        ou = Lu;
        ov = Lv;
      } else {
        const R rdt = dt;
        const R su = wu + rdt * Lu, sv = wv + rdt * Lv;
        if (a.stage == 1) {
          ou = su;
          ov = sv;
        } else {
          const R ca = a.stage == 2 ? R(0.75) : R(1.0 / 3.0);
          const R cb = a.stage == 2 ? R(0.25) : R(2.0 / 3.0);
          ou = ca * u0c[c][0] + cb * su;
          ov = ca * u0c[c][1] + cb * sv;
        }
      }
      R* out = static_cast<R*>(a.out);
      out[(2 * c + 0) * n + i] = ou;
      out[(2 * c + 1) * n + i] = ov;
      if (a.lim_out) {
        R* lo = static_cast<R*>(a.lim_out);
        lo[(2 * c + 0) * n + i] = wu;
        lo[(2 * c + 1) * n + i] = a.stage == 0 ? wvm : wv;  // rhs mode: the modified moment
      }
      if (!isfinite(ou) || !isfinite(ov)) bad |= ST_NONFINITE;
      Uo[c] = ou;
    }
    if (a.flags_out) a.flags_out[i] = (uint8_t)myflag;
    if (a.stage > 0) {
      speed = wave_speed<R, C>(gas, Uo);
      if (!(speed == speed)) {
        bad |= ST_NONPHYSICAL;
        speed = R(0);
      }
    }
  }
  // 6. epilogue: the maximum wave speed of the output into the tile's slot
  //    for the next alpha (a maximum does not depend on the order of the
  //    atomics), the troubled count, the status bits.  Batches and grids of up
  //    to kWarpAtomicTiles tiles fold each warp's values directly (no CTA
  //    barrier on the latency-bound path); larger grids reduce over the CTA
  //    first, so that the slots' atomic queues stay short.
  R wmax = speed;
  for (int o = 16; o > 0; o >>= 1) wmax = fmax(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
  const int wcnt = __popc(__ballot_sync(0xffffffffu, myflag));
  if (bad) atomicOr(&a.sc->status, bad);
  double* const slot = static_cast<double*>(a.a_out) + (BATCH ? inst : tile % kAlphaSlots);
  if (BATCH || a.ntile <= kWarpAtomicTiles) {
    if (lane == 0) {
      if (a.a_out) atomic_max_nonneg(slot, (double)wmax);
      if (wcnt) atomicAdd(&a.sc->troubled, (unsigned long long)wcnt);
    }
    return;
  }
  if (lane == 0) {
    sm.red[warp] = wmax;
    sm.cnt[warp] = wcnt;
  }
  bar_sync(kBarCells, NT);
  if (warp == 0) {
    R m = lane < NW ? sm.red[lane] : R(0);
    int c = lane < NW ? sm.cnt[lane] : 0;
    for (int o = 16; o > 0; o >>= 1) {
      m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
      c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if (lane == 0) {
      if (a.a_out) atomic_max_nonneg(slot, (double)m);
      if (c) atomicAdd(&a.sc->troubled, (unsigned long long)c);
    }
  }
}

}  // namespace s1d
}  // namespace hw
