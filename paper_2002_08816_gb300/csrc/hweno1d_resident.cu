// The resident 1D run: a whole run of third-order TVD Runge-Kutta steps of the
// hybrid HWENO scheme (Zhao & Qiu, arXiv:2002.08816, Sec. 2.1, Eq. (odeH),
// Eq. (RK)) in one cooperative launch in which every CTA keeps its tile of
// the state on chip for all stages.
//
// A CTA of NTH + 32 threads owns T <= NTH - 6 consecutive cells (T chosen on
// the host so that the tiles cover the grid with one or a few CTAs per SM).
// Between stages nothing of the tile leaves the SM: each thread keeps its own
// cell's stage output and the limited u^n in registers and writes the output
// into the shared-memory stage input at the start of the next stage.  Only
// two things cross CTAs per stage, both as 64-bit words that carry their
// stage in the high half and an FP32 value in the low half, written with
// relaxed stores and polled with relaxed loads (an aligned 64-bit access is
// single-copy atomic, so a word with the expected tag holds that stage's
// value: no fence, flag or counter is needed, and every exchange costs one
// round trip to L2):
//   * the 3-cell halo: each CTA publishes its first and last three outputs
//     (two generations, by stage parity); the six halo threads of a
//     neighbour poll exactly the words they need;
//   * alpha (global Lax-Friedrichs flux, Sec. 2.1) and, in stage 1, dt: each
//     CTA publishes the maximum wave speed of its outputs in a word of its own
//     cache line (two generations); the scalar warp of CTA 0 polls them all,
//     reduces them exactly and publishes alpha in one word, which the scalar
//     warp of every other CTA polls (two hops instead of every CTA polling
//     every entry, which made the entries' few cache lines a hot spot); each
//     forms dt = CFL dx / alpha in FP64 with the clip to t_final and hands
//     both to the cell threads through shared memory, all while the cell
//     threads compute the troubled flags, the limiter and the interface
//     values, which do not need alpha.
// Both buffers are zeroed before each launch (tags start at 1).
// Every wait is bounded (r.polls polls; the library passes 2^21, about a
// second): a CTA whose wait runs out sets ST_TIMEOUT and leaves, so the others
// run out too and the launch ends with a status the host reads.  A self-test
// (hweno_check_resident) names a CTA that never publishes its maximum.  The arithmetic of a cell is that of the
// per-stage kernel (hweno1d_stage.cuh): the same helpers in the same order.
#include <cuda_runtime.h>
#include <stdint.h>

#include "hweno1d_comp.cuh"

namespace hw {
namespace {

using s1d::bar_arrive;
using s1d::bar_sync;
using s1d::ConsVec;
using s1d::H;
using s1d::kBarAll;
using s1d::kBarCells;
using s1d::ldx;
using s1d::Smem1D;


constexpr int kMaxEnt = 10;            // entries a scalar-warp lane polls (ncta <= 320)
constexpr int kEntStride = 16;         // words between two CTAs' entries: one cache line each

typedef unsigned long long u64;
__device__ __forceinline__ u64 ld_relaxed(const u64* p) {
  u64 v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(u64* p, u64 v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ u64 tagged(unsigned tag, float v) {
  return ((u64)tag << 32) | (u64)__float_as_uint(v);
}
__device__ __forceinline__ unsigned tag_of(u64 w) { return (unsigned)(w >> 32); }
__device__ __forceinline__ float value_of(u64 w) { return __uint_as_float((unsigned)w); }

// The maximum of the ncta entries (kEntStride words apart) once all carry
// `tag` (the warp's lanes poll up to kMaxEnt entries each, every round's loads
// in flight together); false after `polls` rounds.
__device__ __forceinline__ bool gather_max(const u64* ent, int ncta, unsigned tag, int lane,
                                           float* out, unsigned polls) {
  u64 w[kMaxEnt];
#pragma unroll
  for (int j = 0; j < kMaxEnt; ++j) w[j] = 0ull;
  bool ok = false;
  for (unsigned it = 0; it < polls; ++it) {
    bool mine = true;
#pragma unroll
    for (int j = 0; j < kMaxEnt; ++j) {
      const int k = lane + 32 * j;
      if (k < ncta && tag_of(w[j]) != tag) w[j] = ld_relaxed(ent + (size_t)k * kEntStride);
    }
#pragma unroll
    for (int j = 0; j < kMaxEnt; ++j) {
      const int k = lane + 32 * j;
      if (k < ncta && tag_of(w[j]) != tag) mine = false;
    }
    if (__all_sync(0xffffffffu, mine)) {
      ok = true;
      break;
    }
  }
  float m = 0.0f;
#pragma unroll
  for (int j = 0; j < kMaxEnt; ++j)
    if (lane + 32 * j < ncta) m = fmaxf(m, value_of(w[j]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  *out = m;
  return ok;
}

// One word polled by one thread until it carries `tag`; false after `polls`
// polls.
__device__ __forceinline__ bool poll_word(const u64* p, unsigned tag, u64* out, unsigned polls) {
  for (unsigned it = 0; it < polls; ++it) {
    const u64 w = ld_relaxed(p);
    if (tag_of(w) == tag) {
      *out = w;
      return true;
    }
  }
  return false;
}

template <typename R, int C, int NTH, bool COMP>
struct SmemRes {
  Smem1D<R, C, NTH> w;  // the stage's working arrays (as the per-stage kernel)
  // float-pair averages (COMP): low parts of the stage input's averages (sm.u
  // slots) and the flux increments f(hi_{e+1}) - f(hi_e) (sm.fm slots)
  R ulo[COMP ? C : 1][COMP ? NTH : 1];
  R fb[COMP ? C : 1][COMP ? NTH : 1];
  int abort;            // a wait ran out: every thread leaves
  unsigned red_max[2];  // the CTA's maximum wave speed (bits), per stage parity
  unsigned arrived[2];  // warps that have folded theirs in
  unsigned trb;         // troubled cell-stages of the run
};

// Source of halo slot j (0..2 left, 3..5 right) of the tile of Tq cells from
// base (tiles of T cells; the last one may be shorter): the CTA that owns the
// cell and the slot in that CTA's published cells (0..2 its first three
// cells, 3..5 its last three), and the mirror flag of a reflective ghost.
struct HaloSrc {
  int cta, slot;
  bool mirror;
};
__device__ __forceinline__ HaloSrc halo_source(int j, int base, int Tq, int T, int n, int bc,
                                               int ncta) {
  const int g = j < 3 ? base - 3 + j : base + Tq + (j - 3);
  int src;
  bool mir = false;
  if (bc == 2) src = bc_map_wall(g, n, &mir);
  else src = bc_map(g, n, bc);
  HaloSrc h;
  h.cta = src / T;
  if (h.cta >= ncta) h.cta = ncta - 1;
  const int first = h.cta * T;
  const int last = min(first + T, n);  // one past the owner's last cell
  const int lo = src - first;
  h.slot = lo < 3 ? lo : 3 + (src - (last - 3));
  h.mirror = mir;
  return h;
}

template <typename R, int C, int NTH, bool COMP>
__global__ void __launch_bounds__(NTH + 32, NTH == 256 ? 2 : 1) resident1d_kernel(Resident1DArgs r) {
  static_assert(sizeof(R) == 4, "the exchange words carry FP32 values");
  __shared__ SmemRes<R, C, NTH, COMP> S;
  Smem1D<R, C, NTH>& sm = S.w;
  const Stage1DArgs& a = r.a;
  const int tid = threadIdx.x, lane = tid & 31;
  constexpr int NT = NTH, NW = NTH / 32;
  const int T = r.tile, n = a.n, ncta = gridDim.x, q = blockIdx.x;
  const int base = q * T;
  const int Tq = min(T, n - base);  // this CTA's cells (the last tile may be short)
  u64* const hal = r.halo;                 // [cta][parity][6 slots][C][NV]
  constexpr int NV = COMP ? 3 : 2;         // words per cell and component: average, first
                                           // moment (, low part of the average)
  constexpr int HS = 6 * C * NV;           // values of one CTA's published cells

  if (tid == 0) {
    S.abort = 0;
    S.red_max[0] = S.red_max[1] = 0u;
    S.arrived[0] = S.arrived[1] = 0u;
    S.trb = 0u;
  }
  __syncthreads();

  if (tid >= NT) {
    // ---- the scalar warp ------------------------------------------------
    double t = 0.0, rem = 0.0, tf = 0.0, dt = 0.0;
    unsigned last = 0u;
    unsigned long long steps = 0ull;
    const bool lead = q == 0 && lane == 0;
    tf = ldx(&a.sc->t_final);
    t = ldx(&a.sc->t);
    rem = ldx(&a.sc->rem);
    steps = ldx(&a.sc->steps);
    const u64* ent = r.entries;
    int done_steps = 0;
    int s_end = 3 * r.nsteps;  // stages whose outputs exist at the end
    bool ok = true;
    for (int s = 0; s < 3 * r.nsteps; ++s) {
      const int stage = s % 3 + 1;
      double alpha = 0.0;
      if (s == 0) {
        const unsigned long long* p0 = static_cast<const unsigned long long*>(r.part0);
        unsigned long long am = 0ull;
        for (int k = lane; k < kAlphaSlots; k += 32) {
          const unsigned long long v = ldx(p0 + k);
          am = v > am ? v : am;
        }
        for (int o = 16; o > 0; o >>= 1) {
          const unsigned long long v = __shfl_xor_sync(0xffffffffu, am, o);
          am = v > am ? v : am;
        }
        alpha = __longlong_as_double((long long)am);
      } else {
        // every CTA has published stage s - 1 (tag s): CTA 0 gathers the
        // entries and publishes alpha, the others read that one word
        float m = 0.0f;
        bool got;
        if (q == 0) {
          got = gather_max(ent + (size_t)((s - 1) & 1) * ncta * kEntStride, ncta, (unsigned)s,
                           lane, &m, r.polls);
          if (got && lane == 0) st_relaxed(r.alpha_word + ((s - 1) & 1), tagged((unsigned)s, m));
        } else {
          u64 w = 0ull;
          if (lane == 0) poll_word(r.alpha_word + ((s - 1) & 1), (unsigned)s, &w, r.polls);
          w = __shfl_sync(0xffffffffu, w, 0);
          got = tag_of(w) == (unsigned)s;
          m = value_of(w);
        }
        if (!got) {
          if (lane == 0) {
            atomicOr(&a.sc->status, (unsigned)ST_TIMEOUT);
            S.abort = 1;
          }
          ok = false;
        }
        alpha = (double)m;
      }
      if (stage == 1) {
        dt = a.cfl_dx / alpha;
        last = 0u;
        if (rem <= 0.0) {
          dt = 0.0;
        } else if (dt >= rem) {
          dt = rem;
          last = 1u;
        }
        if (!(alpha > 0.0) || !isfinite(dt)) dt = 0.0;
      }
      if (lane == 0) {
        sm.alpha = R(alpha);
        sm.dt = R(ok ? dt : 0.0);
      }
      bar_arrive(kBarAll, NT + 32);
      if (!ok || !(dt > 0.0)) {
        s_end = s;
        break;
      }
      if (stage == 3) {
        t = last ? tf : t + dt;
        rem = tf > 0.0 ? tf - t : (double)INFINITY;
        ++done_steps;
      }
    }
    // alpha of the final state for the next call (slot 0 of the first
    // buffer, the other slots and the second buffer zero, as the per-stage
    // launches leave them), once every CTA has published its last stage
    if (q == 0 && ok && s_end > 0) {
      float m = 0.0f;
      if (gather_max(ent + (size_t)((s_end - 1) & 1) * ncta * kEntStride, ncta, (unsigned)s_end,
                     lane, &m, r.polls)) {
        const double am = (double)m;
        double* p0 = static_cast<double*>(r.part0);
        double* p1 = static_cast<double*>(r.part1);
        for (int k = lane; k < kAlphaSlots; k += 32) {
          p0[k] = k == 0 ? am : 0.0;
          p1[k] = 0.0;
        }
      } else if (lane == 0) {
        atomicOr(&a.sc->status, (unsigned)ST_TIMEOUT);
      }
    }
    if (lead) {
      a.sc->t = t;
      a.sc->rem = rem;
      a.sc->rem_f = (float)rem;
      a.sc->dt = dt;
      a.sc->dt_f = (float)dt;
      a.sc->last = last;
      a.sc->steps = steps + (unsigned long long)done_steps;
    }
    return;
  }

  // ---- the cell threads ----------------------------------------------------
  R gam[3], eps, gas, inv_dx;
  if constexpr (sizeof(R) == 4) {
    gam[0] = a.f32[0]; gam[1] = a.f32[1]; gam[2] = a.f32[2];
    eps = a.f32[3]; gas = a.f32[4]; inv_dx = a.f32[5];
  } else {
    gam[0] = a.gam[0]; gam[1] = a.gam[1]; gam[2] = a.gam[2];
    eps = a.eps; gas = a.gas; inv_dx = a.inv_dx;
  }
  const bool own = tid < Tq;
  const int i = base + tid;
  // this thread's cell between stages: the stage output, and u^n as limited
  // by stage 1 (the Runge-Kutta combination's u^n); COMP: the low parts of
  // their averages
  R cur[C][2], u0c[C][2], curl[C], u0l[C];
  // the first stage input: tile and halo from global memory
  {
    const R* w = static_cast<const R*>(a.w);
    if (tid < Tq + 2 * H) {
      if (a.bc == 2) {
        bool mir;
        const int g = bc_map_wall(base - H + tid, n, &mir);
#pragma unroll
        for (int c = 0; c < C; ++c) {
          sm.u[c][0][tid] = w[(2 * c + 0) * n + g] * (mir ? R(mirror_sign(c, 0)) : R(1));
          sm.u[c][1][tid] = w[(2 * c + 1) * n + g] * (mir ? R(mirror_sign(c, 1)) : R(1));
          if constexpr (COMP) S.ulo[c][tid] = r.lo[c * n + g] * (mir ? R(mirror_sign(c, 0)) : R(1));
        }
      } else {
        const int g = bc_map(base - H + tid, n, a.bc);
#pragma unroll
        for (int c = 0; c < C; ++c) {
          sm.u[c][0][tid] = w[(2 * c + 0) * n + g];
          sm.u[c][1][tid] = w[(2 * c + 1) * n + g];
          if constexpr (COMP) S.ulo[c][tid] = r.lo[c * n + g];
        }
      }
    }
  }
  // halo sources of the six halo threads (tid 0..2: left, Tq+3..Tq+5: right)
  const int hj = tid < 3 ? tid : (tid >= Tq + 3 && tid < Tq + 6 ? tid - Tq : -1);
  HaloSrc hs = {0, 0, false};
  if (hj >= 0) hs = halo_source(hj, base, Tq, T, n, a.bc, ncta);
  unsigned bad = 0u;
  int done = 0;  // stages completed

#pragma unroll 1
  for (int s = 0; s < 3 * r.nsteps; ++s) {
    const int stage = s % 3 + 1;
    if (s > 0) {
      // the stage input: own cells from registers, the halo from the
      // neighbours' published cells of stage s - 1
      if (own) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
          sm.u[c][0][tid + H] = cur[c][0];
          sm.u[c][1][tid + H] = cur[c][1];
          if constexpr (COMP) S.ulo[c][tid + H] = curl[c];
        }
      }
      if (hj >= 0) {
        const u64* src = hal + ((size_t)hs.cta * 2 + ((s - 1) & 1)) * HS + hs.slot * (C * NV);
        u64 w[C * NV];
#pragma unroll
        for (int j = 0; j < C * NV; ++j) w[j] = 0ull;
        bool got = false;
        for (unsigned it = 0; it < r.polls && !got; ++it) {
          got = true;
#pragma unroll
          for (int j = 0; j < C * NV; ++j)
            if (tag_of(w[j]) != (unsigned)s) w[j] = ld_relaxed(src + j);
#pragma unroll
          for (int j = 0; j < C * NV; ++j)
            if (tag_of(w[j]) != (unsigned)s) got = false;
        }
        if (!got) {
          atomicOr(&a.sc->status, (unsigned)ST_TIMEOUT);
          S.abort = 1;
        } else {
          const int e = hj < 3 ? hj : Tq + hj;
#pragma unroll
          for (int c = 0; c < C; ++c) {
            const R s0 = hs.mirror ? R(mirror_sign(c, 0)) : R(1);
            sm.u[c][0][e] = R(value_of(w[NV * c + 0])) * s0;
            sm.u[c][1][e] = R(value_of(w[NV * c + 1])) * (hs.mirror ? R(mirror_sign(c, 1)) : R(1));
            if constexpr (COMP) S.ulo[c][e] = R(value_of(w[NV * c + 2])) * s0;
          }
        }
      }
    }
    bar_sync(kBarCells, NT);
    if (S.abort) break;
    if (s == 0 && own) {
#pragma unroll
      for (int c = 0; c < C; ++c) {
        cur[c][0] = sm.u[c][0][tid + H];
        cur[c][1] = sm.u[c][1][tid + H];
        curl[c] = COMP ? S.ulo[c][tid + H] : R(0);
      }
    }

    // Step 1: troubled cells and modified first moments, cells base-2 .. base+Tq+1
    int flag = 0;
    if (tid < Tq + 4) {
      const int k = tid, e = k + 1;
      const double h = a.h;
      const float hthr = a.hthr, hthr_lo = a.hthr_lo;
      if (a.mode == 1) {
        flag = 1;
      } else if (a.mode == 2) {
        flag = 0;
      } else if constexpr (COMP) {
        // the decision on hi + lo (the FP64 form where FP32 on hi cannot decide)
        const bool left = C == 1 ? sm.u[0][0][e] >= R(0) : inflow_left(sm.u[0][0][e], sm.u[1][0][e]);
        flag = c1d::kxrcf_troubled_pair(sm.u[0][0][e - 1], S.ulo[0][e - 1], sm.u[0][0][e],
                                        S.ulo[0][e], sm.u[0][0][e + 1], S.ulo[0][e + 1],
                                        sm.u[0][1][e - 1], sm.u[0][1][e], sm.u[0][1][e + 1], left,
                                        h, a.thr, hthr, hthr_lo);
        if constexpr (C == 3)
          flag = flag || c1d::kxrcf_troubled_pair(sm.u[2][0][e - 1], S.ulo[2][e - 1],
                                                  sm.u[2][0][e], S.ulo[2][e], sm.u[2][0][e + 1],
                                                  S.ulo[2][e + 1], sm.u[2][1][e - 1],
                                                  sm.u[2][1][e], sm.u[2][1][e + 1], left, h,
                                                  a.thr, hthr, hthr_lo);
      } else if constexpr (C == 1) {
        const R uc = sm.u[0][0][e];
        flag = kxrcf_troubled(sm.u[0][0][e - 1], uc, sm.u[0][0][e + 1], sm.u[0][1][e - 1],
                              sm.u[0][1][e], sm.u[0][1][e + 1], uc >= R(0), h, a.thr, hthr,
                              hthr_lo);
      } else {
        const bool left = inflow_left(sm.u[0][0][e], sm.u[1][0][e]);
        flag = kxrcf_troubled(sm.u[0][0][e - 1], sm.u[0][0][e], sm.u[0][0][e + 1],
                              sm.u[0][1][e - 1], sm.u[0][1][e], sm.u[0][1][e + 1], left, h,
                              a.thr, hthr, hthr_lo) ||
               kxrcf_troubled(sm.u[2][0][e - 1], sm.u[2][0][e], sm.u[2][0][e + 1],
                              sm.u[2][1][e - 1], sm.u[2][1][e], sm.u[2][1][e + 1], left, h,
                              a.thr, hthr, hthr_lo);
      }
      sm.fl[k] = (uint8_t)flag;
      if (!flag) {
#pragma unroll
        for (int c = 0; c < C; ++c) sm.vl[c][k] = sm.u[c][1][e];
      } else if constexpr (C == 1) {
        sm.vl[0][k] = limit_first_moment(sm.u[0][0][e - 1], sm.u[0][0][e], sm.u[0][0][e + 1],
                                         sm.u[0][1][e - 1], sm.u[0][1][e + 1], gam, eps);
      } else {
        const ConsVec<R> o = s1d::char_limit<R>(
            gas, gam[0], gam[1], gam[2], eps, sm.u[0][0][e - 1], sm.u[1][0][e - 1],
            sm.u[2][0][e - 1], sm.u[0][0][e], sm.u[1][0][e], sm.u[2][0][e], sm.u[0][0][e + 1],
            sm.u[1][0][e + 1], sm.u[2][0][e + 1], sm.u[0][1][e - 1], sm.u[1][1][e - 1],
            sm.u[2][1][e - 1], sm.u[0][1][e + 1], sm.u[1][1][e + 1], sm.u[2][1][e + 1]);
#pragma unroll
        for (int c = 0; c < 3; ++c) sm.vl[c][k] = o.v[c];
      }
    }
    bar_sync(kBarCells, NT);

    // Step 2: interface values and their physical fluxes, cells base-1 .. base+Tq
    // (COMP: their increments over the cell's hi)
    if (tid < Tq + 2) {
      if constexpr (COMP)
        c1d::faces_of_cell_inc<C, NTH>(sm, S.ulo, S.fb, tid, gas, gam, eps, a.variant);
      else
        s1d::faces_of_cell<R, C, NTH>(sm, tid, gas, gam, eps, a.variant);
    }
    bar_sync(kBarCells, NT);

    // own cells: Eq. (odeH) up to its alpha-linear part, before alpha is known;
    // COMP: also the alpha-independent part of the averages' combination
    int myflag = 0;
    R speed = R(0);
    R L0u[C], Du[C], L0v[C], Dv[C], bh[C], bl[C];
    if (own) {
      myflag = sm.fl[tid + 2];
      if constexpr (COMP) {
        c1d::rhs_parts_inc<C, NTH>(sm, S.ulo, S.fb, tid, gas, inv_dx, L0u, Du, L0v, Dv);
        // 1/3 and 2/3 as float pairs
        constexpr float t1h = 1.0f / 3.0f, t2h = 2.0f / 3.0f;
        constexpr float t1l = (float)(1.0 / 3.0 - (double)t1h), t2l = (float)(2.0 / 3.0 - (double)t2h);
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const R wh = cur[c][0], wl = curl[c];
          if (stage == 1) {
            bh[c] = wh;
            bl[c] = wl;
          } else if (stage == 2) {
            pair_axpby(0.75f, 0.0f, u0c[c][0], u0l[c], 0.25f, 0.0f, wh, wl, bh[c], bl[c]);
          } else {
            pair_axpby(t1h, t1l, u0c[c][0], u0l[c], t2h, t2l, wh, wl, bh[c], bl[c]);
          }
        }
      } else {
        s1d::rhs_parts_of_cell<R, C, NTH>(sm, tid, gas, inv_dx, L0u, Du, L0v, Dv);
      }
    }
    // alpha and dt from the scalar warp
    bar_sync(kBarAll, NT + 32);
    if (S.abort) break;
    const R alpha = sm.alpha, dt = sm.dt;
    if (!(dt > R(0))) break;  // t_final reached: uniform over the grid

    // the Runge-Kutta combination; the output stays in registers, the first
    // and last three are published for the neighbours
    if (own) {
      const int e = tid + H;
      R Uo[C];
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const R Lu = L0u[c] - alpha * Du[c], Lv = L0v[c] - alpha * Dv[c];
        const R wu = sm.u[c][0][e];
        const R wv = (a.variant & HWENO_VARIANT_RAW_COMBINE) ? sm.u[c][1][e] : sm.vl[c][e - 1];
        const R su = wu + dt * Lu, sv = wv + dt * Lv;
        R ou, ov;
        if (stage == 1) {
          u0c[c][0] = wu;
          u0c[c][1] = wv;
          if constexpr (COMP) u0l[c] = curl[c];
          ou = su;
          ov = sv;
        } else {
          const R ca = stage == 2 ? R(0.75) : R(1.0 / 3.0);
          const R cb = stage == 2 ? R(0.25) : R(2.0 / 3.0);
          ou = ca * u0c[c][0] + cb * su;
          ov = ca * u0c[c][1] + cb * sv;
        }
        if constexpr (COMP) {
          // the averages: the pair formed before alpha plus the stage's increment
          const R cb = stage == 1 ? R(1) : stage == 2 ? R(0.25) : R(2.0 / 3.0);
          pair_add(bh[c], bl[c], (cb * dt) * Lu, ou, curl[c]);
        }
        cur[c][0] = ou;
        cur[c][1] = ov;
        if (!isfinite(ou) || !isfinite(ov)) bad |= ST_NONFINITE;
        Uo[c] = ou;
      }
      speed = s1d::wave_speed<R, C>(gas, Uo);
      if (!(speed == speed)) {
        bad |= ST_NONPHYSICAL;
        speed = R(0);
      }
      // publish the first and last three cells (the neighbours' halo)
      const int pslot = tid < 3 ? tid : (tid >= Tq - 3 ? 3 + tid - (Tq - 3) : -1);
      if (pslot >= 0) {
        u64* dst = hal + ((size_t)q * 2 + (s & 1)) * HS + pslot * (C * NV);
#pragma unroll
        for (int c = 0; c < C; ++c) {
          st_relaxed(dst + NV * c + 0, tagged((unsigned)(s + 1), float(cur[c][0])));
          st_relaxed(dst + NV * c + 1, tagged((unsigned)(s + 1), float(cur[c][1])));
          if constexpr (COMP) st_relaxed(dst + NV * c + 2, tagged((unsigned)(s + 1), float(curl[c])));
        }
      }
    }
    // the CTA's maximum wave speed (non-negative floats order as their bit
    // patterns: one warp reduction instruction) and troubled count; the last
    // warp to fold its own in publishes the CTA's (no CTA barrier: the next
    // stage's first barrier orders the shared memory)
    const unsigned wm = __reduce_max_sync(0xffffffffu, __float_as_uint((float)speed));
    const int wc = __popc(__ballot_sync(0xffffffffu, myflag));
    if (lane == 0) {
      const int g = s & 1;
      atomicMax(&S.red_max[g], wm);
      if (wc) atomicAdd(&S.trb, (unsigned)wc);
      __threadfence_block();
      if (atomicAdd(&S.arrived[g], 1u) == (unsigned)(NW - 1)) {
        const unsigned m = atomicExch(&S.red_max[g], 0u);  // read, and reset for stage s + 2
        S.arrived[g] = 0u;
        if (q != r.silent_cta)
          st_relaxed(r.entries + ((size_t)g * ncta + q) * kEntStride,
                     tagged((unsigned)(s + 1), __uint_as_float(m)));
      }
    }
    ++done;
  }

  // the final state, the status bits and the troubled count
  if (own && !S.abort && done > 0) {
    R* out = static_cast<R*>(a.out);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      out[(2 * c + 0) * n + i] = cur[c][0];
      out[(2 * c + 1) * n + i] = cur[c][1];
      if constexpr (COMP) r.lo[c * n + i] = curl[c];
    }
  }
  if (bad) atomicOr(&a.sc->status, bad);
  bar_sync(kBarCells, NT);  // every warp's troubled count is in
  if (tid == 0 && S.trb) atomicAdd(&a.sc->troubled, (unsigned long long)S.trb);
}

template <typename R, int C, int NTH, bool COMP>
cudaError_t resident_occupancy(int* per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      per_sm, resident1d_kernel<R, C, NTH, COMP>, NTH + 32, 0);
}

template <typename R, int C, int NTH, bool COMP>
cudaError_t resident_launch(const Resident1DArgs& r, int ncta, cudaStream_t s) {
  Resident1DArgs rc = r;
  void* args[] = {&rc};
  return cudaLaunchCooperativeKernel((const void*)resident1d_kernel<R, C, NTH, COMP>, dim3(ncta),
                                     dim3(NTH + 32), args, 0, s);
}

template <typename R, int C, bool COMP>
cudaError_t resident_c(int nth, const Resident1DArgs* r, int ncta, cudaStream_t s, int* per) {
  if (r) return nth == 512 ? resident_launch<R, C, 512, COMP>(*r, ncta, s)
                           : resident_launch<R, C, 256, COMP>(*r, ncta, s);
  return nth == 512 ? resident_occupancy<R, C, 512, COMP>(per)
                    : resident_occupancy<R, C, 256, COMP>(per);
}

// comp: the float-pair averages (HWENO_FP32C)
cudaError_t resident_dispatch(int system, int nth, bool comp, const Resident1DArgs* r, int ncta,
                              cudaStream_t s, int* per) {
  if (comp)
    return system == 0 ? resident_c<float, 1, true>(nth, r, ncta, s, per)
                       : resident_c<float, 3, true>(nth, r, ncta, s, per);
  return system == 0 ? resident_c<float, 1, false>(nth, r, ncta, s, per)
                     : resident_c<float, 3, false>(nth, r, ncta, s, per);
}

// HWENO_FP32C state conversions: an FP64 state [C][M][n] (M moments, n cells)
// into hi (the state in FP32) and the low parts of its averages [C][n]; and
// back, hi + lo.
__global__ void split_pairs_kernel(const double* __restrict__ src, float* __restrict__ hi,
                                   float* __restrict__ lo, int C, int M, int n) {
  const size_t total = (size_t)C * M * n;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total;
       k += (size_t)gridDim.x * blockDim.x) {
    const double x = src[k];
    const float h = (float)x;
    hi[k] = h;
    const size_t c = k / ((size_t)M * n), m = (k / n) % M, i = k % n;
    if (m == 0) lo[c * n + i] = (float)(x - (double)h);
  }
}
__global__ void join_pairs_kernel(const float* __restrict__ hi, const float* __restrict__ lo,
                                  double* __restrict__ out, int C, int M, int n) {
  const size_t total = (size_t)C * M * n;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total;
       k += (size_t)gridDim.x * blockDim.x) {
    const size_t c = k / ((size_t)M * n), m = (k / n) % M, i = k % n;
    out[k] = (double)hi[k] + (m == 0 ? (double)lo[c * n + i] : 0.0);
  }
}

}  // namespace

cudaError_t launch_split_pairs(const void* src, void* hi, float* lo, int C, int M, int n,
                               cudaStream_t s) {
  const size_t total = (size_t)C * M * n;
  size_t blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  split_pairs_kernel<<<(unsigned)blocks, 256, 0, s>>>(static_cast<const double*>(src),
                                                      static_cast<float*>(hi), lo, C, M, n);
  return cudaGetLastError();
}

cudaError_t launch_join_pairs(const void* hi, const float* lo, double* out, int C, int M, int n,
                              cudaStream_t s) {
  const size_t total = (size_t)C * M * n;
  size_t blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  join_pairs_kernel<<<(unsigned)blocks, 256, 0, s>>>(static_cast<const float*>(hi), lo, out, C,
                                                     M, n);
  return cudaGetLastError();
}

cudaError_t resident1d_geometry(int system, int nth, bool comp, int n, int* tile, int* ncta) {
  *tile = 0;
  *ncta = 0;
  if (nth != 256 && nth != 512) return cudaErrorInvalidValue;
  int dev = 0, nsm = 0, per = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = resident_dispatch(system, nth, comp, nullptr, 0, nullptr, &per);
  if (e != cudaSuccess) return e;
  if (per < 1 || n < 6) return cudaSuccess;  // not possible: *tile = 0
  // the fewest cells per CTA with all CTAs co-resident; every tile (the
  // last one too) at least 6 cells so that the published first and last
  // three cells do not overlap
  long long slots = (long long)per * nsm;
  if (slots > 32 * kMaxEnt) slots = 32 * kMaxEnt;  // the scalar warp polls at most this many
  int t = (int)((n + slots - 1) / slots);
  if (t < 6) t = 6;
  for (; t <= nth - 6; ++t) {
    const int c = (n + t - 1) / t;
    if (c <= slots && n - (c - 1) * t >= 6) {
      *tile = t;
      *ncta = c;
      return cudaSuccess;
    }
  }
  return cudaSuccess;
}

size_t resident1d_entry_words(int ncta) { return (size_t)2 * ncta * kEntStride + 2; }

size_t resident1d_halo_words(int system, int ncta) {
  return (size_t)ncta * 2 * 6 * (system == 0 ? 1 : 3) * 3;
}

cudaError_t launch_resident1d(const Resident1DArgs& r, int nth, int ncta, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(r.halo, 0,
                                  sizeof(unsigned long long) * resident1d_halo_words(r.a.system, ncta), s);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(r.entries, 0, sizeof(unsigned long long) * resident1d_entry_words(ncta), s);
  if (e != cudaSuccess) return e;
  return resident_dispatch(r.a.system, nth, r.lo != nullptr, &r, ncta, s, nullptr);
}

}  // namespace hw
