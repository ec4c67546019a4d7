// The 1D kernels: one launch per third-order TVD Runge-Kutta stage (captured
// in CUDA graphs by the C ABI, with programmatic dependent launch), or a whole
// run in one persistent cooperative launch; both inline the same stage body
// (hweno1d_stage.cuh).  Also the wave-speed kernels that start a
// run and small helpers (conversions, device scalars).
#include <cuda_runtime.h>
#include <stdint.h>

#include "hweno1d_stage.cuh"

namespace hw {
namespace {

using s1d::H;
using s1d::Smem1D;
using s1d::wave_speed;
constexpr int NT = kThreads1D;  // threads of the wave-speed kernels
constexpr int T = kTile1D;      // their cells per CTA
constexpr int NW = NT / 32;

// Every CTA has NTH cell threads and one scalar warp (hweno1d_stage.cuh).
// The 128-thread tiles are the high-occupancy choice: 8 CTAs per SM in FP32
// (at most 51 registers), 6 in FP64, which hides the stage's dependent
// load and arithmetic chains on large states and batches; on small states,
// which sit at the per-stage latency floor, the 256-thread tiles at the
// register count the compiler picks are faster.  hweno_autotune chooses.
template <typename R, int C, bool BATCH, int NTH>
__global__ void __launch_bounds__(NTH + 32, NTH == 128 ? (sizeof(R) == 4 ? 8 : 6) : 1)
    stage1d_kernel(Stage1DArgs a) {
  __shared__ Smem1D<R, C, NTH> sm;
  s1d::stage1d_tile<R, C, BATCH, NTH>(a, blockIdx.x, sm);
}

// ------------------------------------------------------------ persistent run
// A whole run of Runge-Kutta steps in one cooperative launch: each CTA applies
// the stage body to its tiles of a stage, then all CTAs meet at a grid barrier
// before the next stage reads their outputs and the alpha slots they filled.
// The barrier's wait is bounded: after kBarrierPolls polls (about a second)
// the CTA sets ST_TIMEOUT in the status word and returns, and the others give
// up at their own bounded waits, so a lost arrival cannot hang the GPU
// (hweno_check_barrier exercises exactly that).

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// All CTAs of the (co-resident) grid meet here; false when the wait timed out.
// bar[0] counts the arrivals of the whole launch (zeroed by the host before
// it), so the k-th meeting is over once it reaches target = k * gridDim.x:
// each CTA publishes its writes (fence), adds its arrival without waiting for
// a reply, and polls; nobody resets the counter or bumps a generation, which
// would put two more round trips to L2 on the last arriver's path.
// At most `limit` polls: the persistent kernel passes kBarrierPolls (about a
// second of polling); a CTA whose wait runs out sets ST_TIMEOUT and returns,
// so that a lost arrival ends the launch with a status the host reads.
__device__ __forceinline__ bool grid_sync(unsigned* bar, unsigned target, DevScalars* sc,
                                          unsigned limit) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int good = 1;
    __threadfence();
    atomicAdd(bar, 1u);
    unsigned it = 0;
    while (static_cast<int>(ld_acquire_gpu(bar) - target) < 0) {
      if (++it >= limit) {
        atomicOr(&sc->status, (unsigned)ST_TIMEOUT);
        good = 0;
        break;
      }
      __nanosleep(32);
    }
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

constexpr unsigned kBarrierPolls = 1u << 21;  // ~0.5-1 us a poll: about a second

// Self-test of grid_sync: `meetings` meetings of the grid, each waiting for
// gridDim.x + missing arrivals (missing > 0: arrivals that never come, so every
// wait runs out after `limit` polls).
__global__ void __launch_bounds__(128) barrier_check_kernel(unsigned* bar, int meetings,
                                                            unsigned missing, unsigned limit,
                                                            DevScalars* sc) {
  unsigned meet = 0;
  for (int m = 0; m < meetings; ++m) {
    meet += gridDim.x + missing;
    if (!grid_sync(bar, meet, sc, limit)) return;
  }
}

template <typename R, int C, bool BATCH, int NTH>
__global__ void __launch_bounds__(NTH + 32) run1d_kernel(Run1DArgs r) {
  __shared__ Smem1D<R, C, NTH> sm;
  unsigned meet = 0;  // arrivals that end the next meeting
  for (int step = 0; step < r.nsteps; ++step) {
#pragma unroll 1
    for (int stage = 1; stage <= 3; ++stage) {
      Stage1DArgs a = r.a;
      a.stage = stage;
      const int pi = stage - 1, po = stage % 3, pz = (stage + 1) % 3;
      a.a_in = r.part[pi];
      a.a_out = r.part[po];
      a.a_zero = r.part[pz];
      a.w = r.U[stage - 1];
      a.out = r.U[stage % 3];
      a.u0 = stage == 1 ? nullptr : r.W0;
      a.lim_out = stage == 1 ? r.W0 : nullptr;
      for (int tile = blockIdx.x; tile < a.ntile; tile += gridDim.x) {
        s1d::stage1d_tile<R, C, BATCH, NTH>(a, tile, sm);
        __syncthreads();
      }
      meet += gridDim.x;
      if (!grid_sync(r.bar, meet, r.a.sc, kBarrierPolls)) return;
    }
  }
}

template <typename R, int C, bool BATCH, int NTH>
cudaError_t max_ctas_t(int* ctas) {
  int dev = 0, nsm = 0, per = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, run1d_kernel<R, C, BATCH, NTH>, NTH + 32, 0);
  *ctas = per * nsm;
  return e;
}

template <typename R, int C, bool BATCH, int NTH>
cudaError_t run_t(const Run1DArgs& r, cudaStream_t s) {
  int ctas = 0;
  cudaError_t e = max_ctas_t<R, C, BATCH, NTH>(&ctas);
  if (e != cudaSuccess) return e;
  if (ctas < 1) return cudaErrorCooperativeLaunchTooLarge;
  const int grid = r.a.ntile < ctas ? r.a.ntile : ctas;
  e = cudaMemsetAsync(r.bar, 0, 2 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  Run1DArgs rc = r;
  void* args[] = {&rc};
  return cudaLaunchCooperativeKernel((const void*)run1d_kernel<R, C, BATCH, NTH>, dim3(grid),
                                     dim3(NTH + 32), args, 0, s);
}

template <typename R, int C, bool BATCH>
cudaError_t run_b(const Run1DArgs& r, cudaStream_t s) {
  if (r.a.nth == 128) return run_t<R, C, BATCH, 128>(r, s);
  if (r.a.nth == 512) return run_t<R, C, BATCH, 512>(r, s);
  return run_t<R, C, BATCH, 256>(r, s);
}

template <typename R, int C>
cudaError_t run_c(const Run1DArgs& r, cudaStream_t s) {
  return r.a.tile_inst ? run_b<R, C, true>(r, s) : run_b<R, C, false>(r, s);
}

template <typename R, int C, bool BATCH>
cudaError_t max_b(int nth, int* ctas) {
  if (nth == 128) return max_ctas_t<R, C, BATCH, 128>(ctas);
  if (nth == 512) return max_ctas_t<R, C, BATCH, 512>(ctas);
  return max_ctas_t<R, C, BATCH, 256>(ctas);
}

template <typename R, int C>
cudaError_t max_c(int batch, int nth, int* ctas) {
  return batch ? max_b<R, C, true>(nth, ctas) : max_b<R, C, false>(nth, ctas);
}


// Wave-speed maxima in FP64 slots (the per-cell speeds in the kernel's
// precision, as the stage kernels compute them).
template <typename R, int C>
__global__ void __launch_bounds__(NT) alpha1d_kernel(const R* __restrict__ w, double* a_out,
                                                    int n, double gas, DevScalars* sc, int slots) {
  __shared__ R red[NW];
  const int i = blockIdx.x * T + threadIdx.x;
  R s = R(0);
  if (threadIdx.x < T && i < n) {
    R U[C];
#pragma unroll
    for (int c = 0; c < C; ++c) U[c] = w[(2 * c) * n + i];
    s = wave_speed<R, C>(R(gas), U);
    if (!(s == s)) {
      atomicOr(&sc->status, (unsigned)ST_NONPHYSICAL);
      s = R(0);
    }
  }
  for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < NW; ++k) s = fmax(s, red[k]);
    if (slots)
      atomic_max_nonneg(a_out + blockIdx.x % kAlphaSlots, (double)s);
    else
      a_out[blockIdx.x] = (double)s;
  }
}

// Wave-speed maxima of every instance of a batch, one slot per instance (the
// batch's tiles: NTH threads, NTH - 6 cells).
template <typename R, int C, int NTH>
__global__ void __launch_bounds__(NTH) alpha1d_batch_kernel(Stage1DArgs a) {
  constexpr int T = NTH - 2 * H, NW = NTH / 32;
  __shared__ R red[NW];
  const int inst = a.tile_inst[blockIdx.x];
  const BatchInst& bi = a.binst[inst];
  const int i = a.tile_base[blockIdx.x] + threadIdx.x;
  const R* w = static_cast<const R*>(a.w) + bi.off;
  const int n = bi.n;
  R s = R(0);
  if (threadIdx.x < T && i < n) {
    R U[C];
#pragma unroll
    for (int c = 0; c < C; ++c) U[c] = w[(2 * c) * n + i];
    s = wave_speed<R, C>(R(a.gas), U);
    if (!(s == s)) {
      atomicOr(&a.sc->status, (unsigned)ST_NONPHYSICAL);
      s = R(0);
    }
  }
  for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < NW; ++k) s = fmax(s, red[k]);
    atomic_max_nonneg(static_cast<double*>(a.a_out) + inst, (double)s);
  }
}

__global__ void batch_scalars_kernel(BatchScalars* bsc, int n_inst, int reset, double t_final) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < n_inst; b += gridDim.x * blockDim.x) {
    BatchScalars& s = bsc[b];
    if (reset) {
      s.t = 0.0;
      s.dt = 0.0;
      s.dt_f = 0.0f;
      s.last = 0u;
    }
    const double r = t_final > 0.0 ? t_final - s.t : (double)INFINITY;
    s.rem = r;
    s.rem_f = (float)r;
  }
}

template <typename S, typename D>
__global__ void convert_kernel(const S* __restrict__ src, D* __restrict__ dst, size_t count) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < count;
       k += (size_t)gridDim.x * blockDim.x)
    dst[k] = (D)src[k];
}

// Sums in FP64 of the cell averages of each component: n cells from base,
// component c at base + c * comp_stride.  Pass 1: one FP64 partial per block and
// component, in a fixed order; pass 2 (one block): the partials, in order.
template <typename R>
__global__ void __launch_bounds__(256) totals_kernel(const R* __restrict__ base, long long comp_stride,
                                                     int C, long long n, double* partials) {
  __shared__ double red[8];
  for (int c = 0; c < C; ++c) {
    double s = 0.0;
    for (long long i = blockIdx.x * 256ll + threadIdx.x; i < n; i += (long long)gridDim.x * 256)
      s += (double)base[c * comp_stride + i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int k = 0; k < 8; ++k) t += red[k];
      partials[c * gridDim.x + blockIdx.x] = t;
    }
    __syncthreads();
  }
}

__global__ void totals_finish_kernel(const double* partials, int nblocks, int C, double* out) {
  if (threadIdx.x < C) {
    double t = 0.0;
    for (int b = 0; b < nblocks; ++b) t += partials[threadIdx.x * nblocks + b];
    out[threadIdx.x] = t;
  }
}

__global__ void set_scalars_kernel(DevScalars* sc, int reset, double t_final) {
  if (reset) {
    sc->t = 0.0;
    sc->dt = 0.0;
    sc->dt_f = 0.0f;
    sc->last = 0u;
    sc->status = 0u;
    sc->steps = 0ull;
    sc->troubled = 0ull;
  }
  sc->t_final = t_final;
  const double r = t_final > 0.0 ? t_final - sc->t : (double)INFINITY;
  sc->rem = r;
  sc->rem_f = (float)r;
}

// Stage launches allow programmatic dependent launch: a stage's CTAs can be
// resident before the previous stage ends and start at its completion.
template <typename R, int C, int NTH>
cudaError_t launch_stage1d_n(const Stage1DArgs& a, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)a.ntile);
  cfg.blockDim = dim3(NTH + 32);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (a.tile_inst) return cudaLaunchKernelEx(&cfg, stage1d_kernel<R, C, true, NTH>, a);
  return cudaLaunchKernelEx(&cfg, stage1d_kernel<R, C, false, NTH>, a);
}

template <typename R, int C>
cudaError_t launch_stage1d_t(const Stage1DArgs& a, cudaStream_t s) {
  if (a.nth == 128) return launch_stage1d_n<R, C, 128>(a, s);
  if (a.nth == 512) return launch_stage1d_n<R, C, 512>(a, s);
  return launch_stage1d_n<R, C, 256>(a, s);
}

template <typename R, int C>
void alpha1d_batch_t(const Stage1DArgs& a, cudaStream_t s) {
  if (a.nth == 128) alpha1d_batch_kernel<R, C, 128><<<a.ntile, 128, 0, s>>>(a);
  else if (a.nth == 512) alpha1d_batch_kernel<R, C, 512><<<a.ntile, 512, 0, s>>>(a);
  else alpha1d_batch_kernel<R, C, 256><<<a.ntile, 256, 0, s>>>(a);
}

}  // namespace

cudaError_t run1d_max_ctas(int system, int fp64, int batch, int nth, int* ctas) {
  if (system == 0) return fp64 ? max_c<double, 1>(batch, nth, ctas) : max_c<float, 1>(batch, nth, ctas);
  return fp64 ? max_c<double, 3>(batch, nth, ctas) : max_c<float, 3>(batch, nth, ctas);
}

cudaError_t launch_run1d(const Run1DArgs& r, cudaStream_t s) {
  if (r.a.system == 0) return r.a.fp64 ? run_c<double, 1>(r, s) : run_c<float, 1>(r, s);
  return r.a.fp64 ? run_c<double, 3>(r, s) : run_c<float, 3>(r, s);
}

cudaError_t launch_barrier_check(int ctas, int meetings, int missing, unsigned polls,
                                 unsigned* bar, DevScalars* sc, cudaStream_t s, bool* too_many) {
  int dev = 0, nsm = 0, per = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, barrier_check_kernel, 128, 0);
  if (e != cudaSuccess) return e;
  *too_many = ctas > per * nsm;
  if (*too_many) return cudaSuccess;
  e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  unsigned um = (unsigned)missing;
  void* args[] = {&bar, &meetings, &um, &polls, &sc};
  return cudaLaunchCooperativeKernel((const void*)barrier_check_kernel, dim3(ctas), dim3(128),
                                     args, 0, s);
}

cudaError_t launch_stage1d(const Stage1DArgs& a, cudaStream_t s) {
  if (a.system == 0) return a.fp64 ? launch_stage1d_t<double, 1>(a, s) : launch_stage1d_t<float, 1>(a, s);
  return a.fp64 ? launch_stage1d_t<double, 3>(a, s) : launch_stage1d_t<float, 3>(a, s);
}

cudaError_t launch_alpha1d(const void* w, void* a_out, int n, int ntile, int system, int fp64,
                           double gas, DevScalars* sc, int slots, cudaStream_t s) {
  const double* wd = static_cast<const double*>(w);
  const float* wf = static_cast<const float*>(w);
  double* od = static_cast<double*>(a_out);
  if (system == 0) {
    if (fp64)
      alpha1d_kernel<double, 1><<<ntile, NT, 0, s>>>(wd, od, n, gas, sc, slots);
    else
      alpha1d_kernel<float, 1><<<ntile, NT, 0, s>>>(wf, od, n, gas, sc, slots);
  } else {
    if (fp64)
      alpha1d_kernel<double, 3><<<ntile, NT, 0, s>>>(wd, od, n, gas, sc, slots);
    else
      alpha1d_kernel<float, 3><<<ntile, NT, 0, s>>>(wf, od, n, gas, sc, slots);
  }
  return cudaGetLastError();
}

cudaError_t launch_alpha1d_batch(const Stage1DArgs& a, cudaStream_t s) {
  if (a.system == 0) {
    if (a.fp64) alpha1d_batch_t<double, 1>(a, s);
    else alpha1d_batch_t<float, 1>(a, s);
  } else {
    if (a.fp64) alpha1d_batch_t<double, 3>(a, s);
    else alpha1d_batch_t<float, 3>(a, s);
  }
  return cudaGetLastError();
}

cudaError_t launch_batch_scalars(BatchScalars* bsc, int n_inst, int reset, double t_final,
                                 cudaStream_t s) {
  int blocks = (n_inst + 255) / 256;
  if (blocks < 1) blocks = 1;
  batch_scalars_kernel<<<blocks, 256, 0, s>>>(bsc, n_inst, reset, t_final);
  return cudaGetLastError();
}

cudaError_t launch_convert(const void* src, int src_fp64, void* dst, int dst_fp64, size_t count,
                           cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  const int threads = 256;
  size_t blocks = (count + threads - 1) / threads;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (src_fp64 && dst_fp64)
    convert_kernel<<<(unsigned)blocks, threads, 0, s>>>(static_cast<const double*>(src), static_cast<double*>(dst), count);
  else if (src_fp64)
    convert_kernel<<<(unsigned)blocks, threads, 0, s>>>(static_cast<const double*>(src), static_cast<float*>(dst), count);
  else if (dst_fp64)
    convert_kernel<<<(unsigned)blocks, threads, 0, s>>>(static_cast<const float*>(src), static_cast<double*>(dst), count);
  else
    convert_kernel<<<(unsigned)blocks, threads, 0, s>>>(static_cast<const float*>(src), static_cast<float*>(dst), count);
  return cudaGetLastError();
}

cudaError_t launch_totals(const void* base, int fp64, long long comp_stride, int C, long long n,
                          double* partials, int nblocks, double* out, cudaStream_t s) {
  if (fp64)
    totals_kernel<double><<<nblocks, 256, 0, s>>>(static_cast<const double*>(base), comp_stride, C, n, partials);
  else
    totals_kernel<float><<<nblocks, 256, 0, s>>>(static_cast<const float*>(base), comp_stride, C, n, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  totals_finish_kernel<<<1, 32, 0, s>>>(partials, nblocks, C, out);
  return cudaGetLastError();
}

cudaError_t launch_set_scalars(DevScalars* sc, int reset, double t_final, cudaStream_t s) {
  set_scalars_kernel<<<1, 1, 0, s>>>(sc, reset, t_final);
  return cudaGetLastError();
}

}  // namespace hw
