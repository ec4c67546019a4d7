// Device helpers shared by the 1D and 2D kernels: ghost-cell index maps,
// block reductions, status bits and the Euler physics (Eq. (euler1),
// Eq. (euler2)).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hw {

// FP32 reciprocal and square root by the approximate PTX instructions
// (rcp.approx, sqrt.approx, flushing subnormals: within about 1 ulp, ~20
// cycles of latency on GB300 against 45-65 for the correctly rounded forms);
// FP64 keeps the correctly rounded forms.  Zero gives +inf, a negative
// square root NaN, as the non-physical-state checks expect.
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
template <typename R>
__device__ __forceinline__ R fast_rcp(R x) {
  if constexpr (sizeof(R) == 4) return rcp_approx(x); else return R(1) / x;
}
template <typename R>
__device__ __forceinline__ R fast_sqrt(R x) {
  if constexpr (sizeof(R) == 4) return sqrt_approx(x); else return sqrt(x);
}

// bits of the device status word
enum : unsigned { ST_NONFINITE = 1u, ST_NONPHYSICAL = 2u, ST_TIMEOUT = 4u };

// Scalars of one time integration, resident in device memory.
struct DevScalars {
  double t;          // time reached
  double dt;         // dt of the step in flight (written by stage 1)
  double t_final;    // clip time (<= 0: none)
  double rem;        // t_final - t (+inf without clipping)
  float dt_f;        // dt as the FP32 kernels use it
  float rem_f;       // rem rounded to FP32
  unsigned status;   // ST_* bits
  unsigned last;     // 1: the step in flight was clipped to t_final (its last)
  unsigned long long steps;     // completed steps
  unsigned long long troubled;  // troubled cell-stages
};
static_assert(sizeof(DevScalars) == 64, "one 64-byte block");

// dt and rem in the kernel's precision
template <typename R>
__device__ __forceinline__ R& sc_dt(DevScalars* s) {
  if constexpr (sizeof(R) == 4) return s->dt_f; else return s->dt;
}
template <typename R>
__device__ __forceinline__ R sc_rem(const DevScalars* s) {
  if constexpr (sizeof(R) == 4) return s->rem_f; else return s->rem;
}

// Maximum of a non-negative value into a slot: for x >= 0 the order of the
// IEEE bit patterns is the numeric order.
__device__ __forceinline__ void atomic_max_nonneg(float* slot, float x) {
  atomicMax(reinterpret_cast<unsigned int*>(slot), __float_as_uint(x));
}
__device__ __forceinline__ void atomic_max_nonneg(double* slot, double x) {
  atomicMax(reinterpret_cast<unsigned long long*>(slot),
            (unsigned long long)__double_as_longlong(x));
}

// Ghost cells: periodic wraps, outflow copies the boundary cell.  Any g
// (a tile's halo may span several periods when n is smaller than a tile).
__device__ __forceinline__ int bc_map(int g, int n, int bc) {
  if (bc == 0) {
    if (g >= 0 && g < n) return g;
    int r = g % n;
    return r < 0 ? r + n : r;
  }
  return g < 0 ? 0 : (g >= n ? n - 1 : g);
}

// Reflective walls (1D Euler): a ghost is the mirror image of an interior
// cell; *mirror tells the caller to apply mirror_sign.  Tiles may stage cells
// far beyond the domain when n is small; those (never used by an own cell) are
// clamped into range.
__device__ __forceinline__ int bc_map_wall(int g, int n, bool* mirror) {
  *mirror = g < 0 || g >= n;
  if (g < 0) return min(-1 - g, n - 1);
  if (g >= n) return max(2 * n - 1 - g, 0);
  return g;
}

// q(x) -> s q(2 x_w - x) keeps the average times s and the first moment times
// -s; s = -1 for the momentum (component 1), +1 for density and energy.
__device__ __forceinline__ float mirror_sign(int c, int m) {
  const float s = c == 1 ? -1.0f : 1.0f;
  return m == 0 ? s : -s;
}

// Tensor-memory-accelerator (TMA) copies of a tile into shared memory,
// completed on an mbarrier (PTX ISA: cp.async.bulk.tensor, mbarrier).  One
// thread initialises the barrier, announces the bytes and issues the copy;
// every thread waits on phase 0 with a bounded number of polls.
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
  // the initialised barrier, visible to the copy engine
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// box of the 3D tensor map at element coordinates (x, y, z): x * element size
// must be a multiple of 16 bytes
__device__ __forceinline__ void tma_load_3d(void* dst, const void* map, unsigned long long* bar,
                                            int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// true once phase `parity` completed, false after `polls` unsuccessful polls
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity,
                                                  unsigned polls) {
  for (unsigned it = 0; it < polls; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Appends `item` to a shared-memory work list when `need`: the converged
// threads of the warp vote (ballot), one of them reserves the warp's entries
// with a single shared atomic, and each voter writes its entry at its rank
// among the voters.  Called by every thread of the loop iteration; returns
// the entry's index (-1 without an entry).  Entries past `cap` are counted
// but not written.
__device__ __forceinline__ int list_append(int* count, unsigned short* list, int item, bool need,
                                           int cap) {
  const unsigned act = __activemask();
  const unsigned vote = __ballot_sync(act, need);
  if (!vote) return -1;
  const int lane = threadIdx.x & 31, leader = __ffs(act) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(count, __popc(vote));
  base = __shfl_sync(act, base, leader);
  if (!need) return -1;
  const int q = base + __popc(vote & ((1u << lane) - 1u));
  if (q < cap) list[q] = (unsigned short)item;
  return q;
}

template <int NT>
__device__ __forceinline__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  v = (threadIdx.x < NT / 32) ? red[threadIdx.x] : 0.0;
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (threadIdx.x == 0) red[0] = v;
  __syncthreads();
  v = red[0];
  __syncthreads();
  return v;
}

template <typename R>
__device__ __forceinline__ bool finite(R x) {
  return isfinite(x);
}

// ---------------------------------------------------------------- physics

template <typename R>
struct Euler1D {
  // flux of (rho, m, E)
  static __device__ __forceinline__ void flux(R g, const R* U, R* F) {
    const R rho = U[0], m = U[1], E = U[2];
    const R mu = m / rho;
    const R p = (g - R(1)) * (E - R(0.5) * m * mu);
    F[0] = m;
    F[1] = m * mu + p;
    F[2] = mu * (E + p);
  }
  // Velocity, pressure, sound speed, enthalpy and 1/c at U; FP32 with one
  // approximate reciprocal of rho and an approximate square root.
  static __device__ __forceinline__ void primitive(R g, const R* U, R& mu, R& p, R& c, R& H,
                                                   R& ic) {
    const R rho = U[0];
    if constexpr (sizeof(R) == 4) {
      const R ir = fast_rcp(rho);
      mu = U[1] * ir;
      p = (g - R(1)) * (U[2] - R(0.5) * rho * mu * mu);
      c = fast_sqrt(g * p * ir);
      H = (U[2] + p) * ir;
      ic = fast_rcp(c);
    } else {
      mu = U[1] / U[0];
      p = (g - R(1)) * (U[2] - R(0.5) * rho * mu * mu);
      c = sqrt(g * p / rho);
      H = (U[2] + p) / rho;
      ic = R(1) / c;
    }
  }
  // Left eigenvectors (rows) of dF/dU at U, and the velocity mu, sound speed
  // c and enthalpy H that fix the right ones.
  static __device__ __forceinline__ void left(R g, const R* U, R Lm[3][3], R& mu_, R& c_, R& H_) {
    R mu, p, c, H, ic;
    primitive(g, U, mu, p, c, H, ic);
    const R rho = U[0];
    const R b1 = (g - R(1)) * ic * ic;
    const R b2 = R(0.5) * b1 * mu * mu;
    Lm[0][0] = R(0.5) * (b2 + mu * ic);
    Lm[0][1] = R(-0.5) * (b1 * mu + ic);
    Lm[0][2] = R(0.5) * b1;
    Lm[1][0] = R(1) - b2;
    Lm[1][1] = b1 * mu;
    Lm[1][2] = -b1;
    Lm[2][0] = R(0.5) * (b2 - mu * ic);
    Lm[2][1] = R(-0.5) * (b1 * mu - ic);
    Lm[2][2] = R(0.5) * b1;
    mu_ = mu;
    c_ = c;
    H_ = H;
  }
  // Right eigenvectors (columns: mu-c, mu, mu+c) from mu, c and H.
  static __device__ __forceinline__ void right(R mu, R c, R H, R Rm[3][3]) {
    Rm[0][0] = R(1);        Rm[0][1] = R(1);              Rm[0][2] = R(1);
    Rm[1][0] = mu - c;      Rm[1][1] = mu;                Rm[1][2] = mu + c;
    Rm[2][0] = H - mu * c;  Rm[2][1] = R(0.5) * mu * mu;  Rm[2][2] = H + mu * c;
  }
  // Right and left eigenvectors of dF/dU at U.
  static __device__ __forceinline__ void eigen(R g, const R* U, R Rm[3][3], R Lm[3][3]) {
    R mu, c, H;
    left(g, U, Lm, mu, c, H);
    right(mu, c, H, Rm);
  }
};

// |mu| + c from cell averages; NaN marks a non-physical state.
template <typename R>
__device__ __forceinline__ R euler1d_speed_r(R g, R rho, R m, R E) {
  if (!(rho > R(0))) return R(NAN);
  if constexpr (sizeof(R) == 4) {
    const R ir = fast_rcp(rho);
    const R mu = m * ir;
    const R p = (g - R(1)) * (E - R(0.5) * m * mu);
    if (!(p > R(0))) return R(NAN);
    return fabs(mu) + fast_sqrt(g * p * ir);
  } else {
    const R ir = R(1) / rho;  // one divide for both quotients
    const R mu = m * ir;
    const R p = (g - R(1)) * (E - R(0.5) * m * mu);
    if (!(p > R(0))) return R(NAN);
    return fabs(mu) + sqrt(g * p * ir);
  }
}

}  // namespace hw
