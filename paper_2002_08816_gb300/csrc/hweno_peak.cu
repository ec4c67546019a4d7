// hweno_fma_peak: the FP32 or FP64 fused multiply-add throughput of the GPU,
// measured by a kernel of independent FMA chains, for the arithmetic
// roofline of the stage kernels (the paper names no hardware).
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

template <typename R>
hweno_status measure(int iters, double* flops_per_s) {
  int dev = 0, nsm = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HWENO_ERR_CUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return HWENO_ERR_CUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fma_peak_kernel<R>, kThreads, 0) !=
      cudaSuccess)
    return HWENO_ERR_CUDA;
  if (per < 1) per = 1;
  const int grid = nsm * per;
  R* sink = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  hweno_status st = HWENO_ERR_CUDA;
  float ms = 0.0f;
  // x -> 0.5 x + 0.25 stays in [0, 1): no overflow, no subnormals
  const R a = R(0.5), b = R(0.25);
  if (cudaMalloc(&sink, sizeof(R) * (size_t)grid * kThreads) == cudaSuccess &&
      cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
      cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
    fma_peak_kernel<R><<<grid, kThreads, 0, s>>>(sink, iters, a, b);
    cudaEventRecord(e0, s);
    fma_peak_kernel<R><<<grid, kThreads, 0, s>>>(sink, iters, a, b);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
        cudaGetLastError() == cudaSuccess && ms > 0.0f) {
      const double fmas = (double)grid * kThreads * (double)iters * 16.0 * kChains;
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

extern "C" hweno_status hweno_fma_peak(int fp64, int iters, double* flops_per_s) {
  if (!flops_per_s || iters < 1 || iters > (1 << 24)) return HWENO_ERR_ARG;
  return fp64 ? measure<double>(iters, flops_per_s) : measure<float>(iters, flops_per_s);
}
