// hweno_fma_peak: the FP32 or FP64 fused multiply-add throughput of the GPU,
// measured by a kernel of independent FMA chains, for the arithmetic
// roofline of the stage kernels (the paper names no hardware); and the same
// with packed FP32 (fma.rn.f32x2, two FMAs per instruction), which shows
// whether the packed form raises the FP32 flop rate or only saves issue
// slots.
//
// Every thread of a grid that fills each SM runs kChains independent chains
// of FMAs (x = x * a + b, a and b chosen so the values stay bounded and
// normal) for `iters` iterations; the flops (2 per FMA) over the time of the
// launch, taken with CUDA events on a private stream after one untimed
// launch, are the achieved peak at the clock the GPU runs at.  The chains'
// results are stored so that nothing is optimised away.
#include <cuda_runtime.h>

#include "hweno.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename R>
__global__ void __launch_bounds__(kThreads) fma_peak_kernel(R* sink, int iters, R a, R b) {
  R x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = R(threadIdx.x + k) * R(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
    }
  }
  R s = R(0);
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  sink[blockIdx.x * kThreads + threadIdx.x] = s;
}

// kChains independent chains of packed pairs (2 kChains FMAs per step)
__global__ void __launch_bounds__(kThreads) fma_peak_x2_kernel(float2* sink, int iters, float a,
                                                              float b) {
  float2 x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = make_float2((threadIdx.x + k) * 1e-3f, (threadIdx.x - k) * 1e-3f);
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) x[k] = __ffma2_rn(x[k], a2, b2);
    }
  }
  float2 s = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int k = 0; k < kChains; ++k) s = __fadd2_rn(s, x[k]);
  sink[blockIdx.x * kThreads + threadIdx.x] = s;
}

template <typename R, bool X2>
hweno_status measure(int iters, double* flops_per_s) {
  int dev = 0, nsm = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HWENO_ERR_CUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return HWENO_ERR_CUDA;
  const void* kern = X2 ? (const void*)fma_peak_x2_kernel : (const void*)fma_peak_kernel<R>;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kThreads, 0) != cudaSuccess)
    return HWENO_ERR_CUDA;
  if (per < 1) per = 1;
  const int grid = nsm * per;
  void* sink = nullptr;
  const size_t esize = X2 ? sizeof(float2) : sizeof(R);
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  hweno_status st = HWENO_ERR_CUDA;
  float ms = 0.0f;
  // x -> 0.5 x + 0.25 stays in [0, 1): no overflow, no subnormals
  const R a = R(0.5), b = R(0.25);
  if (cudaMalloc(&sink, esize * (size_t)grid * kThreads) == cudaSuccess &&
      cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
      cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
    for (int rep = 0; rep < 2; ++rep) {  // one untimed launch, then the timed one
      if (rep == 1) cudaEventRecord(e0, s);
      if constexpr (X2)
        fma_peak_x2_kernel<<<grid, kThreads, 0, s>>>(static_cast<float2*>(sink), iters, float(a),
                                                     float(b));
      else
        fma_peak_kernel<R><<<grid, kThreads, 0, s>>>(static_cast<R*>(sink), iters, a, b);
    }
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
        cudaGetLastError() == cudaSuccess && ms > 0.0f) {
      const double fmas = (double)grid * kThreads * (double)iters * 16.0 * kChains * (X2 ? 2 : 1);
      *flops_per_s = 2.0 * fmas / (ms * 1e-3);
      st = HWENO_OK;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (sink) cudaFree(sink);
  return st;
}

}  // namespace

extern "C" hweno_status hweno_fma_peak(int kind, int iters, double* flops_per_s) {
  if (!flops_per_s || iters < 1 || iters > (1 << 24) || kind < 0 || kind > 2) return HWENO_ERR_ARG;
  if (kind == 1) return measure<double, false>(iters, flops_per_s);
  if (kind == 2) return measure<float, true>(iters, flops_per_s);
  return measure<float, false>(iters, flops_per_s);
}
