// Host-side plumbing shared by the C-ABI layer and the kernel translation
// units (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hweno_device.cuh"

namespace hw {

// Everything one 1D stage launch needs.  Pointers are device pointers.
struct Stage1DArgs {
  const void* w;         // stage input [C][2][n]
  const void* u0;        // limited u^n (stages 2, 3)
  void* out;             // stage output (or L in rhs mode)
  void* lim_out;         // stage 1: limited u^n; rhs mode: limited input (nullable)
  const double* a_in;    // per-tile partial maxima of the wave speed of w
  double* a_out;         // per-tile partial maxima of the wave speed of out (nullable)
  DevScalars* sc;        // t, dt, t_final, status, counters
  uint8_t* flags_out;    // troubled flags of the own cells (nullable)
  int n;                 // cells
  int ntile;             // tiles (= CTAs)
  int stage;             // 1, 2, 3; 0 = rhs mode
  int bc;                // 0 periodic, 1 outflow
  int mode;              // 0 hybrid, 1 all, 2 none
  int system;            // 0 Burgers, 1 Euler
  int fp64;              // 0 FP32, 1 FP64
  double dx, cfl, eps, thr, gas;
  double gam[3];
  // derived on the host so that no thread spends FP64 work on them
  double inv_dx;         // 1 / dx
  double h;              // dx / 2, the KXRCF cell size
  float hthr;            // (float)(thr * h)
};

constexpr int kTile1D = 250;     // cells per CTA of the 1D kernels
constexpr int kThreads1D = 256;  // threads per CTA (tile + 3-cell halo per side)

cudaError_t launch_stage1d(const Stage1DArgs& a, cudaStream_t s);
cudaError_t launch_alpha1d(const void* w, double* a_out, int n, int ntile, int system, int fp64,
                           double gas, DevScalars* sc, cudaStream_t s);
cudaError_t launch_convert(const void* src, int src_fp64, void* dst, int dst_fp64, size_t count,
                           cudaStream_t s);
cudaError_t launch_set_scalars(DevScalars* sc, int reset, double t_final, cudaStream_t s);

}  // namespace hw
