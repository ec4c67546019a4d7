// hweno_rhs1d_noalloc: a 1D right-hand-side evaluation that allocates no
// device memory.
//
// hweno_rhs needs scratch memory beside its inputs and outputs (the per-tile
// partial maxima of the wave speed that give the Lax-Friedrichs alpha, and a
// status word), which hweno_create obtains with cudaMalloc.  Some callers
// cannot let a library call cudaMalloc: a framework that has handed the
// device memory to its own pool allocator (a library allocation bypasses the
// pool's accounting and can fail once the pool has reserved the memory), a
// process whose device memory is budgeted allocation by allocation, or a
// latency-bound loop that cannot afford the device synchronisation
// cudaMalloc and cudaFree may imply.  For them this entry point keeps its
// scratch in a fixed file-scope __device__ array instead.
//
// The array holds one partial maximum per tile of the 1D stage kernel plus
// the status word, so one call handles at most HWENO_NOALLOC_MAX_CELLS cells.
// Every GPU that loads the library holds the array (about 131 KiB) until the
// process exits.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include "hweno.h"
#include "hweno_internal.h"

namespace {

constexpr int kNoallocMaxTiles = (HWENO_NOALLOC_MAX_CELLS + hw::kTile1D - 1) / hw::kTile1D;
// layout of the scratch, in doubles: [0, 8) the status word and counters of
// one call (hw::DevScalars), [8, 8 + kNoallocMaxTiles) the per-tile maxima
// of |f'(ubar)| that give alpha
constexpr int kScalarSlots = 8;
static_assert(sizeof(hw::DevScalars) <= kScalarSlots * sizeof(double), "scalars fit");
constexpr int kNoallocScratchDoubles = kScalarSlots + kNoallocMaxTiles;

}  // namespace

// The scratch of every call, on every device that loads the library
// (kNoallocScratchDoubles doubles, about 131 KiB).  In host code this name
// is only a host-side stand-in: the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) double g_noalloc_scratch[kNoallocScratchDoubles];

namespace {

// Device address of the scratch on the current device, looked up on every
// call (cheap next to the call's stream synchronisation), so that a device
// reset or a re-created context never leaves a stale address behind.
hweno_status scratch_on_current_device(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) return HWENO_ERR_CUDA;
  *out = static_cast<double*>(p);
  return HWENO_OK;
}

// hweno_create's checks, plus the two this entry point adds: one dimension,
// and no more cells than the scratch holds.
hweno_status check_config(const hweno_config* c) {
  if (!c) return HWENO_ERR_ARG;
  if (c->dim != 1) return HWENO_ERR_ARG;
  if (c->nx > HWENO_NOALLOC_MAX_CELLS) return HWENO_ERR_TOO_LARGE;
  return hw::validate_config(c);
}

}  // namespace

extern "C" {

hweno_status hweno_rhs1d_noalloc(const hweno_config* cfg, void* cuda_stream, const void* in,
                                 void* out, uint8_t* flags_out, void* ulim_out) {
  hweno_status st = check_config(cfg);
  if (st != HWENO_OK) return st;
  if (!in || !out) return HWENO_ERR_ARG;
  if (in == out || (ulim_out && (ulim_out == in || ulim_out == out)))
    return HWENO_ERR_ARG;
  double* scr = nullptr;
  st = scratch_on_current_device(&scr);
  if (st != HWENO_OK) return st;
  hw::DevScalars* sc = reinterpret_cast<hw::DevScalars*>(scr);
  double* partial = scr + kScalarSlots;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int n = cfg->nx;
  const int ntile = (n + hw::kTile1D - 1) / hw::kTile1D;
  const int fp64 = cfg->precision == HWENO_FP64;
  // the previous call's status bits and counters must not leak into this one
  cudaError_t e = hw::launch_set_scalars(sc, 1, -1.0, s);
  if (e == cudaSuccess)
    e = hw::launch_alpha1d(in, partial, n, ntile, cfg->system, fp64, cfg->gas_gamma, sc, 0, s);
  if (e == cudaSuccess) {
    hw::Stage1DArgs a;
    memset(&a, 0, sizeof(a));
    a.w = in;
    a.out = out;
    a.lim_out = ulim_out;
    a.a_in = partial;
    a.nin = ntile;
    a.a_out = nullptr;
    a.sc = sc;
    a.flags_out = flags_out;
    a.n = n;
    a.ntile = ntile;
    a.stage = 0;
    a.bc = cfg->bc;
    a.mode = cfg->troubled_mode;
    a.system = cfg->system;
    a.fp64 = fp64;
    a.variant = cfg->variant;
    a.dx = (cfg->x1 - cfg->x0) / n;
    a.cfl = cfg->cfl;
    a.eps = cfg->eps;
    a.thr = cfg->kxrcf_threshold;
    a.gas = cfg->gas_gamma;
    for (int k = 0; k < 3; ++k) a.gam[k] = cfg->lin_w[k];
    hw::finish_stage_args(a);
    e = hw::launch_stage1d(a, s);
  }
  unsigned status = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&status, &sc->status, sizeof(status), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return HWENO_ERR_CUDA;
  if (status & hw::ST_NONPHYSICAL) return HWENO_ERR_NONPHYSICAL;
  if (status & hw::ST_NONFINITE) return HWENO_ERR_NONPHYSICAL;
  return HWENO_OK;
}

}  // extern "C"
