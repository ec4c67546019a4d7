// Host-side plumbing shared by the C-ABI layer and the kernel translation
// units (not part of the public ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "hweno.h"
#include "hweno_device.cuh"

namespace hw {

// One instance of a batch of independent 1D problems.
struct BatchInst {
  long long off;           // element offset of the instance's state in the batch buffer
  int n;                   // cells
  int first_tile;          // first tile of the instance
  double inv_dx, h, cfl_dx;
  float inv_dx_f, hthr_f, cfl_dx_f, hthr_lo_f;
};

// Time bookkeeping of one instance.
struct BatchScalars {
  double t, rem, dt;
  float dt_f, rem_f;
  unsigned last, pad;
};

// Everything one 1D stage launch needs.  Pointers are device pointers.
struct Stage1DArgs {
  const void* w;         // stage input [C][2][n]
  const void* u0;        // limited u^n (stages 2, 3)
  void* out;             // stage output (or L in rhs mode)
  void* lim_out;         // stage 1: limited u^n; rhs mode: limited input (nullable)
  // Wave-speed maxima travel between launches in the kernel's precision
  // (float or double elements): a max is exact in any precision.
  const void* a_in;      // maxima of the wave speed of w (nin entries)
  int nin;               // entries of a_in
  void* a_out;           // kAlphaSlots zeroed slots that receive, by atomic max, the
                         // wave-speed maxima of out's tiles (nullable)
  void* a_zero;          // kAlphaSlots slots this launch zeroes for a later stage (nullable)
  DevScalars* sc;        // t, dt, t_final, status, counters
  uint8_t* flags_out;    // troubled flags of the own cells (nullable)
  int n;                 // cells
  int ntile;             // tiles (= CTAs of a per-stage launch)
  int nth;               // threads per CTA of the stage kernels: 128, 256 (also 0) or 512;
                         // a tile is nth - 6 cells
  int stage;             // 1, 2, 3; 0 = rhs mode
  int bc;                // 0 periodic, 1 outflow
  int mode;              // 0 hybrid, 1 all, 2 none
  int system;            // 0 Burgers, 1 Euler
  int fp64;              // 0 FP32, 1 FP64
  int variant;           // HWENO_VARIANT_* bits
  double dx, cfl, eps, thr, gas;
  double gam[3];
  // derived on the host so that no thread spends FP64 work on them (on
  // GB300 a dependent FP64 operation or conversion costs ~80 cycles)
  double inv_dx;         // 1 / dx
  double h;              // dx / 2, the KXRCF cell size
  double cfl_dx;         // cfl * dx
  float hthr;            // (float)(thr * h)
  float hthr_lo;         // (float)(thr * h - hthr): thr * h = hthr + hthr_lo to ~2^-48
  float f32[7];          // FP32 copies: gamma_0..2, eps, gas_gamma, 1/dx, cfl*dx
  // batches of independent instances (nullable): tile -> instance, first cell
  const int* tile_inst;
  const int* tile_base;
  const BatchInst* binst;
  BatchScalars* bsc;
};

// Fills the derived fields of a from its primary ones.
inline void finish_stage_args(Stage1DArgs& a) {
  a.inv_dx = 1.0 / a.dx;
  a.h = 0.5 * a.dx;
  a.cfl_dx = a.cfl * a.dx;
  a.hthr = (float)(a.thr * a.h);
  a.hthr_lo = (float)(a.thr * a.h - (double)a.hthr);
  a.f32[0] = (float)a.gam[0];
  a.f32[1] = (float)a.gam[1];
  a.f32[2] = (float)a.gam[2];
  a.f32[3] = (float)a.eps;
  a.f32[4] = (float)a.gas;
  a.f32[5] = (float)a.inv_dx;
  a.f32[6] = (float)a.cfl_dx;
}

constexpr int kAlphaSlots = 64;  // slots that carry alpha between stages
constexpr int kTile1D = 250;     // cells per CTA of the 1D kernels
constexpr int kThreads1D = 256;  // threads per CTA (tile + 3-cell halo per side)

// KXRCF constants of the 2D reading, derived on the host
struct Kx2 {
  double dx, dy, den_h;      // den_h = h (dx + dy), h = sqrt(dx^2 + dy^2) / 2
  double thr;
  float fdx, fdy, fthr_den;  // FP32 copies: dx, dy, thr * den_h
  float fdx_lo, fdy_lo, fthr_den_lo;  // their rounding errors: dx = fdx + fdx_lo to ~2^-48
};

// Everything one 2D stage launch needs.  Pointers are device pointers.
// Wave-speed maxima: x values in [0, nin), y values in [nin, 2 nin).
struct Stage2DArgs {
  const void* w;
  const void* u0;
  void* out;
  void* lim_out;
  const void* a_in;
  int nin;
  void* a_out;           // 2 * kAlphaSlots slots (x, then y), zeroed, atomic max
  void* a_zero;          // 2 * kAlphaSlots slots to zero (nullable)
  DevScalars* sc;
  uint8_t* flags_out;
  void* rec_alpha;       // nullable: (alpha_x, alpha_y) of the stage, kernel precision
  void* rec_dt;          // nullable: dt of the step (stage 1), kernel precision
  const void* dt_in;     // nullable: stage 1 takes this dt (replay of a recorded step)
  // replay of a recorded stage (nullable): its troubled flags (one byte per
  // cell; periodic grids) and its (alpha_x, alpha_y) in the kernel precision;
  // with alpha_in the stage computes no wave-speed maxima (a_out unused)
  const uint8_t* flags_in;
  const void* alpha_in;
  int nx, ny, stage, bc, mode, system, fp64, ng;
  int variant;            // HWENO_VARIANT_* bits
  int tma;                // set by the launcher: interior tiles copied by TMA
  int comp;               // HWENO_FP32C: the averages' low parts below are read and written
  const float* w_lo;      // low parts of the stage input's averages [C][ny][nx]
  const float* u0_lo;     // low parts of u^n's averages (stages 2-3)
  float* out_lo;          // low parts of the output's averages
  double dx, dy, cfl, eps, thr, gas;
  double gam[5];
  double inv_dx, inv_dy;  // derived
  Kx2 kx;                 // derived
  float f32[10];          // FP32 copies: gamma_0..4, eps, gas, 1/dx, 1/dy, cfl
};

constexpr int kTile2DX = 32, kTile2DY = 8;  // cells per CTA of the 2D adjoint kernels
// CTAs of the 2D stage and wave-speed kernels (their own tile) for nx x ny cells
int stage2d_tiles(int nx, int ny);
constexpr int kThreads2D = 256;

void finish_stage2d_args(Stage2DArgs& a);
// The tensor map of a 2D state (planes planes of ny x nx values of esize
// bytes, x fastest) with a box_x x box_y x planes box, for TMA copies of a tile
// and its halo; false when the state cannot be copied that way (a row not a
// multiple of 16 bytes, an unaligned base, a grid smaller than the box, no
// encoder in the driver): the kernels then load every tile themselves.
bool encode_box_map(const void* w, int nx, int ny, int planes, int esize, int box_x, int box_y,
                    CUtensorMap* map);
// Allows the 2D stage kernel of this configuration its dynamic shared memory.
cudaError_t prepare_stage2d(int system, int fp64, int ng);
cudaError_t launch_stage2d(const Stage2DArgs& a, cudaStream_t s);
// dt of the step in FP64 from the stage-1 input's slots (a.a_in, a.nin), into
// a.sc; launched before every stage 1.
cudaError_t launch_dt2d(const Stage2DArgs& a, cudaStream_t s);
// Wave-speed maxima (x then y) of a 2D state, per tile (slots = 0, 2 ntile
// entries) or into 2 * kAlphaSlots zeroed slots (slots = 1).
cudaError_t launch_alpha2d(const void* w, void* a_out, int nx, int ny, int system, int fp64,
                           double gas, DevScalars* sc, int slots, cudaStream_t s);

// One backward stage of the 2D adjoint (device pointers).  For the stage
// u_out = a W0 + b (W + dt L(W)), W = Step 4 applied to the raw input w with
// the recorded troubled cells: lam_in = (dW/dw)^T [b lam + (dL/dW)^T (b dt
// lam)] (+ acc at stage 1), and acc, the adjoint of W0 = W of stage 1, gets
// a lam (stage 3 sets it, stage 2 adds).  Stage 0: lam_in = (d L(W(w))/dw)^T lam.
struct Adj2DArgs {
  const void* w;          // raw stage input [C][3][ny][nx]
  const uint8_t* flags;   // troubled cells of the stage [ny][nx]
  const void* alpha;      // (alpha_x, alpha_y) of the stage, kernel precision
  const void* dt;         // dt of the step, kernel precision (stage 0: unused)
  const void* lam;        // adjoint of the stage output
  void* G;                // scratch: per tile, C x 3 x (TY + 2) x (TX + 2) partial sums of
                          // its cells' stencil adjoints (kernel A writes, kernel B reads)
  void* acc;              // adjoint of W0
  void* lam_in;           // out: adjoint of the stage input
  int* tile_list;         // scratch, 1 + tiles ints: count, then the tiles kernel C visits
  DevScalars* sc;         // status word (a tile copy that did not land: ST_TIMEOUT)
  int tma;                // set by the launcher: kernel A's interior tiles copied by TMA
  int stage, nx, ny, system, fp64, ng;
  double dx, dy, eps, gas;
  double gam[5];
  float f32[9];           // FP32 copies: gamma_0..4, eps, gas, 1/dx, 1/dy
};
void finish_adj2d_args(Adj2DArgs& a);
cudaError_t prepare_adj2d(int system, int fp64, int ng);
// The two kernels of one backward stage (periodic boundaries).
cudaError_t launch_adj2d(const Adj2DArgs& a, cudaStream_t s);

cudaError_t launch_stage1d(const Stage1DArgs& a, cudaStream_t s);

// hweno_create's configuration checks (HWENO_OK or HWENO_ERR_ARG; the reason
// goes to hweno_last_error(NULL)).
hweno_status validate_config(const hweno_config* c);

// A run of many 1D Runge-Kutta steps in one persistent launch: every CTA
// walks its tiles of each stage, then all CTAs meet at a grid barrier.  The
// buffers rotate as in one per-stage step (stage 1: U[0] -> U[1] and W0,
// stage 2: U[1], W0 -> U[2], stage 3: U[2], W0 -> U[0]; alpha slots
// part[0] -> part[1] -> part[2] -> part[0]).
struct Run1DArgs {
  Stage1DArgs a;      // the stage-independent fields (n, ntile, nth, sc, ...)
  void* U[3];
  void* W0;
  void* part[3];
  int nsteps;
  unsigned* bar;      // grid barrier: arrivals, generation (zeroed before the launch)
};
// A whole run in one cooperative launch in which every CTA keeps its tile of
// the state in shared memory for all stages (hweno1d_resident.cu; FP32,
// single instance): only the 3-cell halos (`halo`) and the per-CTA maximum
// wave speeds (`entries`) cross CTAs, as 64-bit words tagged with their stage.
struct Resident1DArgs {
  Stage1DArgs a;      // physics and sizes; w = out = the state, sc
  int tile;           // cells per CTA (<= threads - 6)
  int nsteps;
  void* part0;        // alpha slots of the state (kAlphaSlots doubles): read
                      // at the start, rewritten for the next call at the end
  void* part1;        // zeroed at the end (the per-stage launches expect it)
  unsigned long long* halo;     // [ncta][2][6][C][2] published first and last cells
  unsigned long long* entries;  // [2][ncta] maximum wave speed of each CTA's outputs, one
                                // cache line each, then [2] alpha words (alpha_word)
  unsigned long long* alpha_word;
  unsigned polls;     // bound of every wait (2^21 polls: about a second)
  int silent_cta;     // self-test: this CTA never publishes its maximum (-1: none)
  float* lo;          // HWENO_FP32C: low parts of the averages [C][n] (read at the
                      // start, rewritten at the end); nullptr: FP32 averages
};
// Words of the entries buffer (entries and the two alpha words) for ncta CTAs.
size_t resident1d_entry_words(int ncta);
// Words of the halo buffer for ncta CTAs (room for the float-pair launch's three
// words per cell and component).
size_t resident1d_halo_words(int system, int ncta);
// Cells per CTA and CTAs of the resident launch with nth + 32 threads for n
// cells (comp: the float-pair averages of HWENO_FP32C); *tile = 0 when the
// grid does not fit on the GPU at once.
cudaError_t resident1d_geometry(int system, int nth, bool comp, int n, int* tile, int* ncta);
// HWENO_FP32C states: an FP64 state [C][M][n] into hi (FP32, the state layout)
// and the averages' low parts [C][n]; and hi + lo back into an FP64 state.
cudaError_t launch_split_pairs(const void* src, void* hi, float* lo, int C, int M, int n,
                               cudaStream_t s);
cudaError_t launch_join_pairs(const void* hi, const float* lo, double* out, int C, int M, int n,
                              cudaStream_t s);
// Zeroes the exchange words, then launches.
cudaError_t launch_resident1d(const Resident1DArgs& r, int nth, int ncta, cudaStream_t s);

// Largest co-resident grid of the persistent kernel for this configuration.
cudaError_t run1d_max_ctas(int system, int fp64, int batch, int nth, int* ctas);
// Cooperative launch of min(ntile, co-resident CTAs) CTAs.
cudaError_t launch_run1d(const Run1DArgs& r, cudaStream_t s);
// hweno_check_barrier's launch; *too_many when ctas cannot all be resident
cudaError_t launch_barrier_check(int ctas, int meetings, int missing, unsigned polls,
                                 unsigned* bar, DevScalars* sc, cudaStream_t s, bool* too_many);
// Batched variants: one launch over all instances (a.tile_inst != nullptr);
// alpha slots are one per instance.
cudaError_t launch_alpha1d_batch(const Stage1DArgs& a, cudaStream_t s);
cudaError_t launch_batch_scalars(BatchScalars* bsc, int n_inst, int reset, double t_final,
                                 cudaStream_t s);
// Wave-speed maxima of w, in the kernel's precision: one per tile (slots = 0)
// or folded into kAlphaSlots zeroed slots by atomic max (slots = 1).
cudaError_t launch_alpha1d(const void* w, void* a_out, int n, int ntile, int system, int fp64,
                           double gas, DevScalars* sc, int slots, cudaStream_t s);
cudaError_t launch_convert(const void* src, int src_fp64, void* dst, int dst_fp64, size_t count,
                           cudaStream_t s);
cudaError_t launch_set_scalars(DevScalars* sc, int reset, double t_final, cudaStream_t s);
// out[c] = sum over n cells of base[c * comp_stride + i] in FP64, c < C <= 8, with
// nblocks partials per component in partials; a fixed summation order.
cudaError_t launch_totals(const void* base, int fp64, long long comp_stride, int C, long long n,
                          double* partials, int nblocks, double* out, cudaStream_t s);

}  // namespace hw
