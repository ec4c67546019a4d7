// C ABI of the library (declared in include/hweno.h): validation, device
// buffers owned by the handle, CUDA-graph-captured Runge-Kutta steps.
//
// One third-order TVD Runge-Kutta step (Eq. (RK)) is three stage launches
// that rotate over the state buffers
//   stage 1: U[0] -> U[1], writes the limited u^n to U0
//   stage 2: U[1], U0 -> U[2]
//   stage 3: U[2], U0 -> U[0]
// and over three buffers of kAlphaSlots wave-speed maxima P0 -> P1 -> P2 -> P0
// that carry alpha from each stage to the next (each stage also zeroes the
// buffer the stage after next fills).  dt, t and the status word live in
// device memory, so a run of many steps needs no host synchronisation.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "hweno.h"
#include "hweno_internal.h"

struct hweno_ctx {
  hweno_config cfg;
  cudaStream_t stream = nullptr;     // caller's stream (may be the legacy default)
  cudaStream_t cap = nullptr;        // private stream used only to capture graphs
  int C = 0, M = 0, n = 0, ntile = 0;  // n = cells; ntile = CTAs of one stage
  int dim = 1;
  // 1D execution: threads per CTA of the stage kernels (a tile is nth1d - 6
  // cells), and how hweno_step launches: per-stage launches in CUDA graphs
  // (persist1d = 0), one persistent launch with a grid barrier per stage (1),
  // or one resident launch that keeps the tiles on chip (2, FP32 single
  // instance); hweno_autotune chooses
  int nth1d = 256, persist1d = 0;
  // the resident launch's geometry and cross-CTA buffers (allocated on first use)
  int res_tile = 0, res_ncta = 0, res_cap = 0;
  unsigned long long* res_halo = nullptr;     // tagged exchange words of the halos
  unsigned long long* res_entries = nullptr;  // and of the per-CTA maxima
  // HWENO_FP32C: the low parts of the averages ([C][n] floats beside U[0]);
  // 1D steps run as the resident launch, 2D steps carry the low parts of the
  // stage buffers U[1], U[2] too (Ulo_s)
  bool comp = false;
  float* Ulo = nullptr;
  float* Ulo_s[2] = {nullptr, nullptr};
  int ntile_alpha = 0;               // CTAs of the wave-speed kernels (1D: kTile1D cells each; 2D: the stage tiles)
  unsigned* bar = nullptr;           // grid barrier of the persistent kernel
  std::vector<int> batch_nx;         // cells of each batch instance
  std::vector<hw::BatchInst> batch_inst;
  double* tot_buf = nullptr;         // hweno_totals: partials, then the sums
  size_t elems = 0, esize = 0;
  void* U[3] = {nullptr, nullptr, nullptr};
  void* U0 = nullptr;
  void* stage_buf = nullptr;         // conversion staging (other precision)
  double* part[3] = {nullptr, nullptr, nullptr};  // kAlphaSlots slots (float or double)
  double* part_rhs = nullptr;                      // one maximum per tile
  hw::DevScalars* sc = nullptr;
  hw::DevScalars* sc_rhs = nullptr;
  cudaGraphExec_t g_many = nullptr;  // kGraphSteps steps
  cudaGraphExec_t g_one = nullptr;   // one step
  bool has_state = false;
  std::string err;
  // batches of independent 1D instances
  int n_batch = 0;
  int* d_tile_inst = nullptr;
  int* d_tile_base = nullptr;
  hw::BatchInst* d_binst = nullptr;
  hw::BatchScalars* d_bsc = nullptr;
  // adjoint: the tape of hweno_record and the scratch of hweno_backward
  struct Tape {
    int nsteps = 0, every = 0, nck = 0;
    void* ck = nullptr;         // checkpoints: u^n for n % every == 0
    uint8_t* flags = nullptr;   // troubled cells, one plane per stage
    void* alpha = nullptr;      // (alpha_x, alpha_y) per stage, kernel precision
    void* dt = nullptr;         // dt per step, kernel precision
    std::vector<double> dt_host;
    int seg_every = 0;          // capacity of seg, in steps
    void* seg = nullptr;        // 3 every + 1 recomputed stage inputs
    void* w0 = nullptr;         // limited u^n of the recomputed step
    void* G = nullptr;          // per-tile partial sums of the stencil adjoints
    int* tile_list = nullptr;   // count + the tiles near a troubled cell
    void* lam[2] = {nullptr, nullptr};
    void* acc = nullptr;
    double* slots = nullptr;    // 3 x 2 kAlphaSlots
    hw::DevScalars* sc = nullptr;
    void* aux = nullptr;        // (alpha_x, alpha_y) of hweno_rhs_vjp
    bool prepared = false;
  } tape;
};

namespace {

constexpr int kGraphSteps = 32;
std::string g_create_error;

hweno_status fail(hweno_ctx* h, hweno_status st, const std::string& msg) {
  if (h)
    h->err = msg;
  else
    g_create_error = msg;
  return st;
}

#define HW_CUDA(h, call)                                                            \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return fail((h), HWENO_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

hw::Stage1DArgs base_args(const hweno_ctx* h) {
  hw::Stage1DArgs a;
  memset(&a, 0, sizeof(a));
  const hweno_config& c = h->cfg;
  a.n = h->n;
  a.ntile = h->ntile;
  a.nth = h->nth1d;
  a.bc = c.bc;
  a.mode = c.troubled_mode;
  a.system = c.system;
  a.fp64 = c.precision == HWENO_FP64;
  a.variant = c.variant;
  a.dx = (c.x1 - c.x0) / c.nx;
  a.cfl = c.cfl;
  a.eps = c.eps;
  a.thr = c.kxrcf_threshold;
  a.gas = c.gas_gamma;
  for (int k = 0; k < 3; ++k) a.gam[k] = c.lin_w[k];
  hw::finish_stage_args(a);
  if (h->n_batch > 0) {
    a.tile_inst = h->d_tile_inst;
    a.tile_base = h->d_tile_base;
    a.binst = h->d_binst;
    a.bsc = h->d_bsc;
  }
  return a;
}

hw::Stage2DArgs base_args2d(const hweno_ctx* h) {
  hw::Stage2DArgs a;
  memset(&a, 0, sizeof(a));
  const hweno_config& c = h->cfg;
  a.nx = c.nx;
  a.ny = c.ny;
  a.bc = c.bc;
  a.mode = c.troubled_mode;
  a.system = c.system;
  a.fp64 = c.precision == HWENO_FP64;
  a.variant = c.variant;
  a.ng = c.n_gauss;
  a.dx = (c.x1 - c.x0) / c.nx;
  a.dy = (c.y1 - c.y0) / c.ny;
  a.cfl = c.cfl;
  a.eps = c.eps;
  a.thr = c.kxrcf_threshold;
  a.gas = c.gas_gamma;
  for (int k = 0; k < 5; ++k) a.gam[k] = c.lin_w[k];
  hw::finish_stage2d_args(a);
  return a;
}

// The buffers of one 2D Runge-Kutta step: in -> s1 -> s2 -> out, the limited
// u^n in w0, alpha carried through part[0..2]; optional recording of the
// switches (flags: 3 planes; rec_alpha: 3 pairs; rec_dt) or replay of a
// recorded step (dt_in; alpha_in: its 3 pairs, flags_in: its 3 planes, which
// spare the replayed stages their wave-speed maxima and KXRCF tests).
struct Step2DIO {
  const void* in;
  void* s1;
  void* s2;
  void* out;
  void* w0;
  double* part[3];
  hw::DevScalars* sc;
  uint8_t* flags;
  void* rec_alpha;
  void* rec_dt;
  const void* dt_in;
  // HWENO_FP32C: the low parts of the averages of in, s1, s2 and out (nullptr:
  // plain precision)
  const float* in_lo = nullptr;
  float* s1_lo = nullptr;
  float* s2_lo = nullptr;
  float* out_lo = nullptr;
  const uint8_t* flags_in = nullptr;
  const void* alpha_in = nullptr;
};

void* byte_off(const void* p, size_t bytes) {
  return static_cast<char*>(const_cast<void*>(p)) + bytes;
}

cudaError_t enqueue_step2d_io(hweno_ctx* h, const Step2DIO& io, cudaStream_t s) {
  hw::Stage2DArgs a = base_args2d(h);
  const size_t pair = 2 * h->esize;
  a.sc = io.sc;
  a.nin = hw::kAlphaSlots;
  a.stage = 1;
  a.w = io.in;
  a.out = io.s1;
  a.lim_out = io.w0;
  a.a_in = io.part[0];
  a.a_out = io.part[1];
  a.a_zero = io.part[2];
  a.flags_out = io.flags;
  a.rec_alpha = io.rec_alpha;
  a.rec_dt = io.rec_dt;
  a.dt_in = io.dt_in;
  a.comp = io.in_lo != nullptr;
  a.w_lo = io.in_lo;
  a.out_lo = io.s1_lo;
  const bool replay = io.alpha_in != nullptr;
  a.flags_in = io.flags_in;
  a.alpha_in = io.alpha_in;
  if (replay) a.a_out = nullptr;
  cudaError_t e = replay ? cudaSuccess : hw::launch_dt2d(a, s);
  if (e != cudaSuccess) return e;
  e = hw::launch_stage2d(a, s);
  if (e != cudaSuccess) return e;
  a.rec_dt = nullptr;
  a.dt_in = nullptr;
  a.stage = 2;
  a.w = io.s1;
  a.u0 = io.w0;
  a.out = io.s2;
  a.lim_out = nullptr;
  a.a_in = io.part[1];
  a.a_out = io.part[2];
  a.a_zero = io.part[0];
  a.w_lo = io.s1_lo;
  a.u0_lo = io.in_lo;  // the limiter leaves the averages of u^n as they are
  a.out_lo = io.s2_lo;
  if (io.flags) a.flags_out = io.flags + (size_t)h->n;
  if (io.rec_alpha) a.rec_alpha = byte_off(io.rec_alpha, pair);
  if (io.flags_in) a.flags_in = io.flags_in + (size_t)h->n;
  if (replay) {
    a.alpha_in = byte_off(io.alpha_in, pair);
    a.a_out = nullptr;
  }
  e = hw::launch_stage2d(a, s);
  if (e != cudaSuccess) return e;
  a.stage = 3;
  a.w = io.s2;
  a.out = io.out;
  a.a_in = io.part[2];
  a.a_out = io.part[0];
  a.a_zero = io.part[1];
  a.w_lo = io.s2_lo;
  a.out_lo = io.out_lo;  // may be in_lo: each cell reads its u^n low part before it writes
  if (io.flags) a.flags_out = io.flags + 2 * (size_t)h->n;
  if (io.rec_alpha) a.rec_alpha = byte_off(io.rec_alpha, 2 * pair);
  if (io.flags_in) a.flags_in = io.flags_in + 2 * (size_t)h->n;
  if (replay) {
    a.alpha_in = byte_off(io.alpha_in, 2 * pair);
    a.a_out = nullptr;
  }
  return hw::launch_stage2d(a, s);
}

cudaError_t enqueue_step2d(hweno_ctx* h, cudaStream_t s) {
  Step2DIO io = {h->U[0], h->U[1], h->U[2], h->U[0], h->U0,
                 {h->part[0], h->part[1], h->part[2]}, h->sc, nullptr, nullptr, nullptr, nullptr};
  if (h->comp) {
    io.in_lo = h->Ulo;
    io.s1_lo = h->Ulo_s[0];
    io.s2_lo = h->Ulo_s[1];
    io.out_lo = h->Ulo;
  }
  return enqueue_step2d_io(h, io, s);
}

// nsteps Runge-Kutta steps of a 1D handle in one persistent launch.
cudaError_t enqueue_run1d(hweno_ctx* h, int nsteps, cudaStream_t s) {
  hw::Run1DArgs r;
  memset(&r, 0, sizeof(r));
  r.a = base_args(h);
  r.a.sc = h->sc;
  r.a.nin = hw::kAlphaSlots;
  for (int k = 0; k < 3; ++k) {
    r.U[k] = h->U[k];
    r.part[k] = h->part[k];
  }
  r.W0 = h->U0;
  r.nsteps = nsteps;
  r.bar = h->bar;
  return hw::launch_run1d(r, s);
}

// Geometry of the resident launch for the handle's threads per CTA (res_tile =
// 0 when it cannot run: FP64, batches, or too many cells to be co-resident),
// and its buffers.
cudaError_t prepare_resident(hweno_ctx* h) {
  h->res_tile = h->res_ncta = 0;
  if (h->dim != 1 || h->n_batch > 0 || h->cfg.precision == HWENO_FP64) return cudaSuccess;
  if (h->nth1d != 256 && h->nth1d != 512) return cudaSuccess;
  int tile = 0, ncta = 0;
  cudaError_t e = hw::resident1d_geometry(h->cfg.system, h->nth1d, h->comp, h->n, &tile, &ncta);
  if (e != cudaSuccess || tile == 0) return e;
  if (ncta > h->res_cap) {
    if (h->res_halo) cudaFree(h->res_halo);
    if (h->res_entries) cudaFree(h->res_entries);
    h->res_halo = nullptr;
    h->res_entries = nullptr;
    h->res_cap = 0;
    e = cudaMalloc(&h->res_halo, hw::resident1d_halo_words(h->cfg.system, ncta) * sizeof(unsigned long long));
    if (e == cudaSuccess)
      e = cudaMalloc(&h->res_entries, sizeof(unsigned long long) * hw::resident1d_entry_words(ncta));
    if (e != cudaSuccess) return e;
    h->res_cap = ncta;
  }
  h->res_tile = tile;
  h->res_ncta = ncta;
  return cudaSuccess;
}

// nsteps Runge-Kutta steps of a 1D handle in one resident launch (silent_cta,
// polls: the failure-detection self-test; -1 and 2^21 otherwise).
cudaError_t enqueue_resident1d(hweno_ctx* h, int nsteps, cudaStream_t s, int silent_cta = -1,
                               unsigned polls = 1u << 21) {
  hw::Resident1DArgs r;
  memset(&r, 0, sizeof(r));
  r.a = base_args(h);
  r.a.sc = h->sc;
  r.a.w = h->U[0];
  r.a.out = h->U[0];
  r.tile = h->res_tile;
  r.nsteps = nsteps;
  r.part0 = h->part[0];
  r.part1 = h->part[1];
  r.halo = h->res_halo;
  r.entries = h->res_entries;
  r.alpha_word = h->res_entries + hw::resident1d_entry_words(h->res_ncta) - 2;
  r.polls = polls;
  r.silent_cta = silent_cta;
  r.lo = h->comp ? h->Ulo : nullptr;
  return hw::launch_resident1d(r, h->nth1d, h->res_ncta, s);
}

cudaError_t enqueue_step(hweno_ctx* h, cudaStream_t s) {
  if (h->dim == 2) return enqueue_step2d(h, s);
  hw::Stage1DArgs a = base_args(h);
  a.sc = h->sc;
  // stage 1
  a.stage = 1;
  a.w = h->U[0];
  a.out = h->U[1];
  a.lim_out = h->U0;
  a.a_in = h->part[0];
  a.nin = hw::kAlphaSlots;
  a.a_out = h->part[1];
  a.a_zero = h->part[2];
  cudaError_t e = hw::launch_stage1d(a, s);
  if (e != cudaSuccess) return e;
  // stage 2
  a.stage = 2;
  a.w = h->U[1];
  a.u0 = h->U0;
  a.out = h->U[2];
  a.lim_out = nullptr;
  a.a_in = h->part[1];
  a.a_out = h->part[2];
  a.a_zero = h->part[0];
  e = hw::launch_stage1d(a, s);
  if (e != cudaSuccess) return e;
  // stage 3
  a.stage = 3;
  a.w = h->U[2];
  a.out = h->U[0];
  a.a_in = h->part[2];
  a.a_out = h->part[0];
  a.a_zero = h->part[1];
  return hw::launch_stage1d(a, s);
}

hweno_status build_graph(hweno_ctx* h, int steps, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  HW_CUDA(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < steps && e == cudaSuccess; ++k) e = enqueue_step(h, h->cap);
  cudaError_t e2 = cudaStreamEndCapture(h->cap, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return fail(h, HWENO_ERR_CUDA, std::string("graph capture: ") +
                                       cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(h, HWENO_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  return HWENO_OK;
}

hweno_status validate(const hweno_config* c) {
  if (!c) return fail(nullptr, HWENO_ERR_ARG, "cfg is NULL");
  if (c->dim != 1 && c->dim != 2) return fail(nullptr, HWENO_ERR_ARG, "dim must be 1 or 2");
  if (c->dim == 2) {
    if (c->ny < 4) return fail(nullptr, HWENO_ERR_ARG, "ny must be >= 4");
    if (!(c->y1 > c->y0)) return fail(nullptr, HWENO_ERR_ARG, "y1 must exceed y0");
    if ((double)c->nx * c->ny > (double)(1u << 30)) return fail(nullptr, HWENO_ERR_ARG, "too many cells");
    const double dx = (c->x1 - c->x0) / c->nx, dy = (c->y1 - c->y0) / c->ny;
    if (fabs(dx - dy) > 1e-12 * (dx > dy ? dx : dy))
      return fail(nullptr, HWENO_ERR_ARG, "2D cells must be square (dx = dy)");
    if (c->n_gauss != 2 && c->n_gauss != 3) return fail(nullptr, HWENO_ERR_ARG, "n_gauss must be 2 or 3");
  }
  if (c->system != HWENO_BURGERS && c->system != HWENO_EULER)
    return fail(nullptr, HWENO_ERR_ARG, "unknown system");
  if (c->nx < 4) return fail(nullptr, HWENO_ERR_ARG, "nx must be >= 4");
  if (c->nx > (1 << 28)) return fail(nullptr, HWENO_ERR_ARG, "nx too large");
  if (!(c->x1 > c->x0)) return fail(nullptr, HWENO_ERR_ARG, "x1 must exceed x0");
  if (c->bc != HWENO_BC_PERIODIC && c->bc != HWENO_BC_OUTFLOW && c->bc != HWENO_BC_REFLECTIVE)
    return fail(nullptr, HWENO_ERR_ARG, "unknown boundary condition");
  if (c->bc == HWENO_BC_REFLECTIVE && (c->dim != 1 || c->system != HWENO_EULER))
    return fail(nullptr, HWENO_ERR_ARG, "reflective walls are available for 1D Euler");
  if (c->system == HWENO_EULER && !(c->gas_gamma > 1.0))
    return fail(nullptr, HWENO_ERR_ARG, "gas_gamma must exceed 1");
  const int ncand = c->dim == 1 ? 3 : 5;
  double s = 0.0;
  for (int k = 0; k < ncand; ++k) {
    if (!(c->lin_w[k] > 0.0)) return fail(nullptr, HWENO_ERR_ARG, "linear weights must be positive");
    s += c->lin_w[k];
  }
  if (fabs(s - 1.0) > 1e-12) return fail(nullptr, HWENO_ERR_ARG, "linear weights must sum to one");
  if (!(c->cfl > 0.0)) return fail(nullptr, HWENO_ERR_ARG, "cfl must be positive");
  if (!(c->eps > 0.0)) return fail(nullptr, HWENO_ERR_ARG, "eps must be positive");
  if (!(c->kxrcf_threshold >= 0.0)) return fail(nullptr, HWENO_ERR_ARG, "threshold must be >= 0");
  if (c->troubled_mode < 0 || c->troubled_mode > 2) return fail(nullptr, HWENO_ERR_ARG, "unknown troubled_mode");
  if (c->precision != HWENO_FP32 && c->precision != HWENO_FP64 && c->precision != HWENO_FP32C)
    return fail(nullptr, HWENO_ERR_ARG, "unknown precision");
  if (c->variant & ~(HWENO_VARIANT_RAW_COMBINE | HWENO_VARIANT_MEAN_EIGEN))
    return fail(nullptr, HWENO_ERR_ARG, "unknown variant bits");
  return HWENO_OK;
}

hweno_status check_scalars(hweno_ctx* h, hw::DevScalars* dev, hw::DevScalars* host) {
  HW_CUDA(h, cudaMemcpyAsync(host, dev, sizeof(*host), cudaMemcpyDeviceToHost, h->stream));
  HW_CUDA(h, cudaStreamSynchronize(h->stream));
  if (host->status & hw::ST_NONPHYSICAL)
    return fail(h, HWENO_ERR_NONPHYSICAL, "non-physical state (rho <= 0 or p <= 0)");
  if (host->status & hw::ST_NONFINITE) return fail(h, HWENO_ERR_NONPHYSICAL, "non-finite value");
  if (host->status & hw::ST_TIMEOUT) return fail(h, HWENO_ERR_TIMEOUT, "device wait timed out");
  return HWENO_OK;
}

void free_ptr(void** p) {
  if (*p) cudaFree(*p);
  *p = nullptr;
}

// Frees the recorded run (and, with scratch, the buffers of the backward pass).
void free_tape(hweno_ctx* h, bool scratch) {
  hweno_ctx::Tape& t = h->tape;
  free_ptr(&t.ck);
  free_ptr(reinterpret_cast<void**>(&t.flags));
  free_ptr(&t.alpha);
  free_ptr(&t.dt);
  t.dt_host.clear();
  t.nsteps = t.every = t.nck = 0;
  if (!scratch) return;
  free_ptr(&t.seg);
  free_ptr(&t.w0);
  free_ptr(&t.G);
  free_ptr(&t.lam[0]);
  free_ptr(&t.lam[1]);
  free_ptr(&t.acc);
  free_ptr(reinterpret_cast<void**>(&t.slots));
  free_ptr(reinterpret_cast<void**>(&t.sc));
  free_ptr(&t.aux);
  free_ptr(reinterpret_cast<void**>(&t.tile_list));
  t.seg_every = 0;
}

hweno_status check_adjoint_config(hweno_ctx* h) {
  if (h->dim != 2) return fail(h, HWENO_ERR_ARG, "the adjoint is for 2D handles");
  if (h->n_batch > 0) return fail(h, HWENO_ERR_ARG, "the adjoint takes a single-instance handle");
  if (h->cfg.bc != HWENO_BC_PERIODIC) return fail(h, HWENO_ERR_ARG, "the adjoint needs periodic boundaries");
  if (h->cfg.variant != 0) return fail(h, HWENO_ERR_ARG, "the adjoint is of the default variant");
  if (h->comp) return fail(h, HWENO_ERR_ARG, "the adjoint takes HWENO_FP32 or HWENO_FP64 handles");
  return HWENO_OK;
}

// Scratch of the adjoint kernels (G, the alpha pair, the device scalars),
// allocated on first use.
hweno_status adjoint_scratch(hweno_ctx* h) {
  hweno_ctx::Tape& t = h->tape;
  if (!t.prepared) {
    HW_CUDA(h, hw::prepare_adj2d(h->cfg.system, h->cfg.precision == HWENO_FP64, h->cfg.n_gauss));
    t.prepared = true;
  }
  if (!t.G)
    HW_CUDA(h, cudaMalloc(&t.G, (size_t)h->ntile * h->C * 3 * (hw::kTile2DX + 2) *
                                    (hw::kTile2DY + 2) * h->esize));
  if (!t.aux) HW_CUDA(h, cudaMalloc(&t.aux, 2 * sizeof(double)));
  if (!t.tile_list) HW_CUDA(h, cudaMalloc(reinterpret_cast<void**>(&t.tile_list), sizeof(int) * (1 + (size_t)h->ntile)));
  if (!t.sc) HW_CUDA(h, cudaMalloc(&t.sc, sizeof(hw::DevScalars)));
  return HWENO_OK;
}

hw::Adj2DArgs base_adj_args(const hweno_ctx* h) {
  hw::Adj2DArgs a;
  memset(&a, 0, sizeof(a));
  const hweno_config& c = h->cfg;
  a.nx = c.nx;
  a.ny = c.ny;
  a.system = c.system;
  a.fp64 = c.precision == HWENO_FP64;
  a.ng = c.n_gauss;
  a.dx = (c.x1 - c.x0) / c.nx;
  a.dy = (c.y1 - c.y0) / c.ny;
  a.eps = c.eps;
  a.gas = c.gas_gamma;
  for (int k = 0; k < 5; ++k) a.gam[k] = c.lin_w[k];
  a.G = h->tape.G;
  a.tile_list = h->tape.tile_list;
  a.sc = h->tape.sc;
  hw::finish_adj2d_args(a);
  return a;
}

// The tiles of every batch instance for stage CTAs of nth threads (nth - 6
// cells per tile): tile -> instance and first cell, each instance's first
// tile; replaces the previous tiling.
cudaError_t batch_tiles(hweno_ctx* h, int nth) {
  const int T = nth - 6;
  std::vector<int> tinst, tbase;
  for (int b = 0; b < h->n_batch; ++b) {
    h->batch_inst[b].first_tile = (int)tinst.size();
    for (int base = 0; base < h->batch_nx[b]; base += T) {
      tinst.push_back(b);
      tbase.push_back(base);
    }
  }
  if (h->d_tile_inst) cudaFree(h->d_tile_inst);
  if (h->d_tile_base) cudaFree(h->d_tile_base);
  h->d_tile_inst = h->d_tile_base = nullptr;
  const size_t nt = tinst.size();
  cudaError_t e = cudaMalloc(&h->d_tile_inst, sizeof(int) * nt);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_tile_base, sizeof(int) * nt);
  if (e == cudaSuccess) e = cudaMemcpy(h->d_tile_inst, tinst.data(), sizeof(int) * nt, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->d_tile_base, tbase.data(), sizeof(int) * nt, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(h->d_binst, h->batch_inst.data(), sizeof(hw::BatchInst) * h->n_batch,
                   cudaMemcpyHostToDevice);
  h->ntile = (int)nt;
  return e;
}

}  // namespace

namespace hw {
// The configuration checks of hweno_create, for entry points without a handle.
hweno_status validate_config(const hweno_config* c) { return validate(c); }
}  // namespace hw

extern "C" {

void hweno_default_config(hweno_config* cfg, int dim, int system) {
  if (!cfg) return;
  memset(cfg, 0, sizeof(*cfg));
  cfg->dim = dim;
  cfg->system = system;
  cfg->x0 = 0.0;
  cfg->x1 = 1.0;
  cfg->y0 = 0.0;
  cfg->y1 = 1.0;
  cfg->bc = HWENO_BC_PERIODIC;
  cfg->gas_gamma = 1.4;
  if (dim == 2) {
    cfg->lin_w[0] = 0.96;
    for (int k = 1; k < 5; ++k) cfg->lin_w[k] = 0.01;
  } else {
    cfg->lin_w[0] = 0.98;
    cfg->lin_w[1] = 0.01;
    cfg->lin_w[2] = 0.01;
  }
  cfg->cfl = 0.6;
  cfg->eps = 1e-6;
  cfg->kxrcf_threshold = 1.0;
  cfg->troubled_mode = HWENO_TROUBLED_HYBRID;
  cfg->n_gauss = 3;
  cfg->precision = HWENO_FP32;
}

hweno_status hweno_create(const hweno_config* cfg, void* cuda_stream, hweno_handle* out) {
  if (!out) return fail(nullptr, HWENO_ERR_ARG, "out is NULL");
  hweno_status st = validate(cfg);
  if (st != HWENO_OK) return st;
  hweno_ctx* h = new hweno_ctx();
  h->cfg = *cfg;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  h->dim = cfg->dim;
  if (cfg->dim == 2) {
    h->C = cfg->system == HWENO_EULER ? 4 : 1;
    h->M = 3;
    h->n = cfg->nx * cfg->ny;
    // ntile: the adjoint kernels' tiles; ntile_alpha: the stage and wave-speed
    // kernels' (the per-tile maxima of hweno_rhs)
    h->ntile = ((cfg->nx + hw::kTile2DX - 1) / hw::kTile2DX) * ((cfg->ny + hw::kTile2DY - 1) / hw::kTile2DY);
    h->ntile_alpha = hw::stage2d_tiles(cfg->nx, cfg->ny);
  } else {
    h->C = cfg->system == HWENO_EULER ? 3 : 1;
    h->M = 2;
    h->n = cfg->nx;
    h->ntile = (h->n + h->nth1d - 7) / (h->nth1d - 6);
    h->ntile_alpha = (h->n + hw::kTile1D - 1) / hw::kTile1D;
  }
  h->elems = (size_t)h->C * h->M * h->n;
  h->esize = cfg->precision == HWENO_FP64 ? 8 : 4;
  h->comp = cfg->precision == HWENO_FP32C;
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaMalloc(&h->U[k], h->elems * h->esize);
  if (e == cudaSuccess && h->comp) e = cudaMalloc(&h->Ulo, sizeof(float) * h->C * h->n);
  for (int k = 0; k < 2 && e == cudaSuccess && h->comp && cfg->dim == 2; ++k)
    e = cudaMalloc(&h->Ulo_s[k], sizeof(float) * h->C * h->n);
  if (e == cudaSuccess) e = cudaMalloc(&h->U0, h->elems * h->esize);
  if (e == cudaSuccess) e = cudaMalloc(&h->stage_buf, h->elems * 8);
  for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaMalloc(&h->part[k], sizeof(double) * 2 * hw::kAlphaSlots);
  if (e == cudaSuccess)
    e = cudaMalloc(&h->part_rhs, sizeof(double) * 2 * (h->ntile > h->ntile_alpha ? h->ntile : h->ntile_alpha));
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&h->bar), 2 * sizeof(unsigned));
  if (e == cudaSuccess && cfg->dim == 2)
    e = hw::prepare_stage2d(cfg->system, cfg->precision == HWENO_FP64, cfg->n_gauss);
  if (e == cudaSuccess) e = cudaMalloc(&h->sc, sizeof(hw::DevScalars));
  if (e == cudaSuccess) e = cudaMalloc(&h->sc_rhs, sizeof(hw::DevScalars));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = hw::launch_set_scalars(h->sc, 1, -1.0, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    std::string msg = std::string("allocation: ") + cudaGetErrorString(e);
    hweno_destroy(h);
    return fail(nullptr, HWENO_ERR_CUDA, msg);
  }
  if (h->comp && h->dim == 1) {  // the resident launch only
    h->persist1d = 2;
    e = prepare_resident(h);
    if (e != cudaSuccess || h->res_tile == 0) {
      std::string msg = e != cudaSuccess ? std::string("resident launch: ") + cudaGetErrorString(e)
                                         : std::string("HWENO_FP32C runs as the resident launch, "
                                                       "and this grid does not fit on the GPU at once");
      hweno_destroy(h);
      return fail(nullptr, e != cudaSuccess ? HWENO_ERR_CUDA : HWENO_ERR_ARG, msg);
    }
  }
  *out = h;
  return HWENO_OK;
}

hweno_status hweno_set_state(hweno_handle h, const void* moments, int dtype, int on_device) {
  if (!h) return fail(nullptr, HWENO_ERR_ARG, "handle is NULL");
  if (!moments) return fail(h, HWENO_ERR_ARG, "moments is NULL");
  if (dtype != HWENO_FP32 && dtype != HWENO_FP64) return fail(h, HWENO_ERR_ARG, "unknown dtype");
  const int src64 = dtype == HWENO_FP64, dst64 = h->cfg.precision == HWENO_FP64;
  const size_t sbytes = h->elems * (src64 ? 8 : 4);
  const void* src = moments;
  if (!on_device) {
    if (src64 == dst64) {
      HW_CUDA(h, cudaMemcpyAsync(h->U[0], moments, sbytes, cudaMemcpyHostToDevice, h->stream));
      src = nullptr;
    } else {
      HW_CUDA(h, cudaMemcpyAsync(h->stage_buf, moments, sbytes, cudaMemcpyHostToDevice, h->stream));
      src = h->stage_buf;
    }
  }
  if (h->comp) {
    // hi into the state, the low parts of the averages beside it
    if (src64) HW_CUDA(h, hw::launch_split_pairs(src ? src : h->U[0], h->U[0], h->Ulo, h->C, h->M, h->n, h->stream));
    else {
      if (src) HW_CUDA(h, hw::launch_convert(src, 0, h->U[0], 0, h->elems, h->stream));
      HW_CUDA(h, cudaMemsetAsync(h->Ulo, 0, sizeof(float) * h->C * h->n, h->stream));
    }
  } else if (src) {
    HW_CUDA(h, hw::launch_convert(src, src64, h->U[0], dst64, h->elems, h->stream));
  }
  HW_CUDA(h, hw::launch_set_scalars(h->sc, 1, -1.0, h->stream));
  const size_t nslot = h->n_batch > 2 * hw::kAlphaSlots ? (size_t)h->n_batch : 2 * hw::kAlphaSlots;
  for (int k = 0; k < 3; ++k)
    HW_CUDA(h, cudaMemsetAsync(h->part[k], 0, sizeof(double) * nslot, h->stream));
  if (h->n_batch > 0) {
    HW_CUDA(h, hw::launch_batch_scalars(h->d_bsc, h->n_batch, 1, -1.0, h->stream));
    hw::Stage1DArgs a = base_args(h);
    a.w = h->U[0];
    a.a_out = h->part[0];
    a.sc = h->sc;
    HW_CUDA(h, hw::launch_alpha1d_batch(a, h->stream));
  } else if (h->dim == 2)
    HW_CUDA(h, hw::launch_alpha2d(h->U[0], h->part[0], h->cfg.nx, h->cfg.ny, h->cfg.system, dst64,
                                  h->cfg.gas_gamma, h->sc, 1, h->stream));
  else
    HW_CUDA(h, hw::launch_alpha1d(h->U[0], h->part[0], h->n, h->ntile_alpha, h->cfg.system, dst64,
                                  h->cfg.gas_gamma, h->sc, 1, h->stream));
  h->has_state = true;
  return HWENO_OK;
}

hweno_status hweno_step(hweno_handle h, int nsteps, double t_final, double* t_out) {
  if (!h) return fail(nullptr, HWENO_ERR_ARG, "handle is NULL");
  if (!h->has_state) return fail(h, HWENO_ERR_STATE, "hweno_step before hweno_set_state");
  if (nsteps < 0) return fail(h, HWENO_ERR_ARG, "nsteps must be >= 0");
  HW_CUDA(h, hw::launch_set_scalars(h->sc, 0, t_final, h->stream));
  if (h->n_batch > 0)
    HW_CUDA(h, hw::launch_batch_scalars(h->d_bsc, h->n_batch, 0, t_final, h->stream));
  int left = nsteps;
  if (h->dim == 1 && h->persist1d == 2) {
    if (left > 0) HW_CUDA(h, enqueue_resident1d(h, left, h->stream));
    left = 0;
  } else if (h->dim == 1 && h->persist1d) {
    if (left > 0) HW_CUDA(h, enqueue_run1d(h, left, h->stream));
    left = 0;
  }
  if (left >= kGraphSteps) {
    if (!h->g_many) {
      hweno_status st = build_graph(h, kGraphSteps, &h->g_many);
      if (st != HWENO_OK) return st;
    }
    for (; left >= kGraphSteps; left -= kGraphSteps) HW_CUDA(h, cudaGraphLaunch(h->g_many, h->stream));
  }
  if (left > 0) {
    if (!h->g_one) {
      hweno_status st = build_graph(h, 1, &h->g_one);
      if (st != HWENO_OK) return st;
    }
    for (; left > 0; --left) HW_CUDA(h, cudaGraphLaunch(h->g_one, h->stream));
  }
  if (t_out) {
    hw::DevScalars s;
    hweno_status st = check_scalars(h, h->sc, &s);
    *t_out = s.t;
    return st;
  }
  return HWENO_OK;
}

hweno_status hweno_rhs(hweno_handle h, const void* in, void* out, uint8_t* flags_out, void* ulim_out) {
  if (!h) return fail(nullptr, HWENO_ERR_ARG, "handle is NULL");
  if (h->n_batch > 0) return fail(h, HWENO_ERR_ARG, "hweno_rhs takes a single-instance handle");
  if (!in || !out) return fail(h, HWENO_ERR_ARG, "in and out must be device pointers");
  if (in == out || (ulim_out && (ulim_out == in || ulim_out == out)))
    return fail(h, HWENO_ERR_ARG, "in, out and ulim_out must not overlap");
  HW_CUDA(h, hw::launch_set_scalars(h->sc_rhs, 1, -1.0, h->stream));
  if (h->dim == 2) {
    HW_CUDA(h, hw::launch_alpha2d(in, h->part_rhs, h->cfg.nx, h->cfg.ny, h->cfg.system,
                                  h->cfg.precision == HWENO_FP64, h->cfg.gas_gamma, h->sc_rhs, 0,
                                  h->stream));
    hw::Stage2DArgs a = base_args2d(h);
    a.stage = 0;
    a.w = in;
    a.out = out;
    a.lim_out = ulim_out;
    a.a_in = h->part_rhs;
    a.nin = h->ntile_alpha;
    a.sc = h->sc_rhs;
    a.flags_out = flags_out;
    HW_CUDA(h, hw::launch_stage2d(a, h->stream));
    hw::DevScalars s2;
    return check_scalars(h, h->sc_rhs, &s2);
  }
  HW_CUDA(h, hw::launch_alpha1d(in, h->part_rhs, h->n, h->ntile_alpha, h->cfg.system,
                                h->cfg.precision == HWENO_FP64, h->cfg.gas_gamma, h->sc_rhs, 0,
                                h->stream));
  hw::Stage1DArgs a = base_args(h);
  a.stage = 0;
  a.w = in;
  a.out = out;
  a.lim_out = ulim_out;
  a.a_in = h->part_rhs;
  a.nin = h->ntile_alpha;
  a.a_out = nullptr;
  a.sc = h->sc_rhs;
  a.flags_out = flags_out;
  HW_CUDA(h, hw::launch_stage1d(a, h->stream));
  hw::DevScalars s;
  return check_scalars(h, h->sc_rhs, &s);
}

hweno_status hweno_get_state(hweno_handle h, void* out, int dtype, int on_device) {
  if (!h) return fail(nullptr, HWENO_ERR_ARG, "handle is NULL");
  if (!out) return fail(h, HWENO_ERR_ARG, "out is NULL");
  if (!h->has_state) return fail(h, HWENO_ERR_STATE, "hweno_get_state before hweno_set_state");
  if (dtype != HWENO_FP32 && dtype != HWENO_FP64) return fail(h, HWENO_ERR_ARG, "unknown dtype");
  const int dst64 = dtype == HWENO_FP64, src64 = h->cfg.precision == HWENO_FP64;
  const size_t dbytes = h->elems * (dst64 ? 8 : 4);
  if (h->comp && dst64) {  // hi + lo of the averages
    void* dst = on_device ? out : h->stage_buf;
    HW_CUDA(h, hw::launch_join_pairs(h->U[0], h->Ulo, static_cast<double*>(dst), h->C, h->M, h->n, h->stream));
    if (on_device) return HWENO_OK;
    HW_CUDA(h, cudaMemcpyAsync(out, h->stage_buf, dbytes, cudaMemcpyDeviceToHost, h->stream));
    HW_CUDA(h, cudaStreamSynchronize(h->stream));
    return HWENO_OK;
  }
  if (on_device) {
    HW_CUDA(h, hw::launch_convert(h->U[0], src64, out, dst64, h->elems, h->stream));
    return HWENO_OK;
  }
  const void* src = h->U[0];
  if (src64 != dst64) {
    HW_CUDA(h, hw::launch_convert(h->U[0], src64, h->stage_buf, dst64, h->elems, h->stream));
    src = h->stage_buf;
  }
  HW_CUDA(h, cudaMemcpyAsync(out, src, dbytes, cudaMemcpyDeviceToHost, h->stream));
  HW_CUDA(h, cudaStreamSynchronize(h->stream));
  return HWENO_OK;
}

hweno_status hweno_stats(hweno_handle h, double* t, double* last_dt, int64_t* steps,
                         int64_t* troubled_cell_stages) {
  if (!h) return fail(nullptr, HWENO_ERR_ARG, "handle is NULL");
  hw::DevScalars s;
  HW_CUDA(h, cudaMemcpyAsync(&s, h->sc, sizeof(s), cudaMemcpyDeviceToHost, h->stream));
  HW_CUDA(h, cudaStreamSynchronize(h->stream));
  if (h->n_batch > 0) {  // the time of instance 0
    hw::BatchScalars b0;
    HW_CUDA(h, cudaMemcpy(&b0, h->d_bsc, sizeof(b0), cudaMemcpyDeviceToHost));
    s.t = b0.t;
    s.dt = b0.dt;
  }
  if (t) *t = s.t;
  if (last_dt) *last_dt = s.dt;
  if (steps) *steps = (int64_t)s.steps;
  if (troubled_cell_stages) *troubled_cell_stages = (int64_t)s.troubled;
  return HWENO_OK;
}

void hweno_destroy(hweno_handle h) {
  if (!h) return;
  if (h->g_many) cudaGraphExecDestroy(h->g_many);
  if (h->g_one) cudaGraphExecDestroy(h->g_one);
  for (int k = 0; k < 3; ++k) {
    if (h->U[k]) cudaFree(h->U[k]);
    if (h->part[k]) cudaFree(h->part[k]);
  }
  if (h->U0) cudaFree(h->U0);
  if (h->stage_buf) cudaFree(h->stage_buf);
  if (h->part_rhs) cudaFree(h->part_rhs);
  if (h->sc) cudaFree(h->sc);
  if (h->sc_rhs) cudaFree(h->sc_rhs);
  if (h->bar) cudaFree(h->bar);
  if (h->res_halo) cudaFree(h->res_halo);
  if (h->res_entries) cudaFree(h->res_entries);
  if (h->Ulo) cudaFree(h->Ulo);
  for (int k = 0; k < 2; ++k)
    if (h->Ulo_s[k]) cudaFree(h->Ulo_s[k]);
  if (h->tot_buf) cudaFree(h->tot_buf);
  if (h->d_tile_inst) cudaFree(h->d_tile_inst);
  if (h->d_tile_base) cudaFree(h->d_tile_base);
  if (h->d_binst) cudaFree(h->d_binst);
  if (h->d_bsc) cudaFree(h->d_bsc);
  free_tape(h, true);
  if (h->cap) cudaStreamDestroy(h->cap);
  delete h;
}

hweno_status hweno_create_batch(const hweno_config* cfg, int n_batch, const int* nx,
                                void* cuda_stream, hweno_handle* out) {
  if (!out) return fail(nullptr, HWENO_ERR_ARG, "out is NULL");
  if (!cfg || cfg->dim != 1) return fail(nullptr, HWENO_ERR_ARG, "batches are of 1D instances");
  if (cfg->precision == HWENO_FP32C)
    return fail(nullptr, HWENO_ERR_ARG, "batches take HWENO_FP32 or HWENO_FP64");
  if (n_batch < 1 || !nx) return fail(nullptr, HWENO_ERR_ARG, "n_batch must be >= 1 with sizes");
  hweno_config c = *cfg;
  long long total = 0;
  for (int b = 0; b < n_batch; ++b) {
    if (nx[b] < 4) return fail(nullptr, HWENO_ERR_ARG, "every instance needs nx >= 4");
    total += nx[b];
  }
  if (total > (1ll << 28)) return fail(nullptr, HWENO_ERR_ARG, "batch too large");
  c.nx = nx[0];
  hweno_status st = validate(&c);
  if (st != HWENO_OK) return st;
  c.nx = (int)total;
  hweno_handle h = nullptr;
  st = hweno_create(&c, cuda_stream, &h);
  if (st != HWENO_OK) return st;
  h->cfg.nx = (int)total;
  h->n_batch = n_batch;
  // each instance's geometry, and the tiles
  std::string msg;
  const int C = h->C;
  long long cells = 0;
  h->batch_nx.assign(nx, nx + n_batch);
  h->batch_inst.resize(n_batch);
  for (int b = 0; b < n_batch; ++b) {
    hw::BatchInst& bi = h->batch_inst[b];
    const double dx = (c.x1 - c.x0) / nx[b];
    bi.off = (long long)C * 2 * cells;
    bi.n = nx[b];
    bi.first_tile = 0;
    bi.inv_dx = 1.0 / dx;
    bi.h = 0.5 * dx;
    bi.cfl_dx = c.cfl * dx;
    bi.inv_dx_f = (float)bi.inv_dx;
    bi.hthr_f = (float)(c.kxrcf_threshold * bi.h);
    bi.cfl_dx_f = (float)bi.cfl_dx;
    bi.hthr_lo_f = (float)(c.kxrcf_threshold * bi.h - (double)bi.hthr_f);
    cells += nx[b];
  }
  cudaError_t e = cudaMalloc(&h->d_binst, sizeof(hw::BatchInst) * n_batch);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_bsc, sizeof(hw::BatchScalars) * n_batch);
  if (e == cudaSuccess) e = batch_tiles(h, h->nth1d);
  // one alpha slot per instance in each of the three rotating buffers
  for (int r = 0; r < 3 && e == cudaSuccess && n_batch > 2 * hw::kAlphaSlots; ++r) {
    cudaFree(h->part[r]);
    h->part[r] = nullptr;
    e = cudaMalloc(&h->part[r], sizeof(double) * n_batch);
  }
  if (e != cudaSuccess) {
    msg = std::string("batch allocation: ") + cudaGetErrorString(e);
    hweno_destroy(h);
    return fail(nullptr, HWENO_ERR_CUDA, msg);
  }
  *out = h;
  return HWENO_OK;
}

hweno_status hweno_batch_times(hweno_handle h, double* t) {
  if (!h) return fail(nullptr, HWENO_ERR_ARG, "handle is NULL");
  if (h->n_batch < 1 || !t) return fail(h, HWENO_ERR_ARG, "not a batch handle, or t is NULL");
  HW_CUDA(h, cudaStreamSynchronize(h->stream));
  hw::BatchScalars* b = new hw::BatchScalars[h->n_batch];
  cudaError_t e = cudaMemcpy(b, h->d_bsc, sizeof(hw::BatchScalars) * h->n_batch, cudaMemcpyDeviceToHost);
  for (int k = 0; k < h->n_batch && e == cudaSuccess; ++k) t[k] = b[k].t;
  delete[] b;
  if (e != cudaSuccess) return fail(h, HWENO_ERR_CUDA, cudaGetErrorString(e));
  return HWENO_OK;
}

hweno_status hweno_record(hweno_handle h, int nsteps, int checkpoint_every, double t_final,
                          double* t_out) {
  if (!h) return fail(nullptr, HWENO_ERR_ARG, "handle is NULL");
  hweno_status st = check_adjoint_config(h);
  if (st != HWENO_OK) return st;
  if (!h->has_state) return fail(h, HWENO_ERR_STATE, "hweno_record before hweno_set_state");
  if (nsteps < 1 || checkpoint_every < 1)
    return fail(h, HWENO_ERR_ARG, "nsteps and checkpoint_every must be >= 1");
  free_tape(h, false);
  hweno_ctx::Tape& t = h->tape;
  const size_t sbytes = h->elems * h->esize;
  const int nck = (nsteps + checkpoint_every - 1) / checkpoint_every;
  HW_CUDA(h, cudaMalloc(&t.ck, sbytes * nck));
  HW_CUDA(h, cudaMalloc(reinterpret_cast<void**>(&t.flags), (size_t)3 * nsteps * h->n));
  HW_CUDA(h, cudaMalloc(&t.alpha, (size_t)6 * nsteps * h->esize));
  HW_CUDA(h, cudaMalloc(&t.dt, (size_t)nsteps * h->esize));
  HW_CUDA(h, cudaMemsetAsync(t.dt, 0, (size_t)nsteps * h->esize, h->stream));
  HW_CUDA(h, hw::launch_set_scalars(h->sc, 0, t_final, h->stream));
  for (int n = 0; n < nsteps; ++n) {
    if (n % checkpoint_every == 0)
      HW_CUDA(h, cudaMemcpyAsync(byte_off(t.ck, sbytes * (n / checkpoint_every)), h->U[0], sbytes,
                                 cudaMemcpyDeviceToDevice, h->stream));
    Step2DIO io = {h->U[0], h->U[1], h->U[2], h->U[0], h->U0,
                   {h->part[0], h->part[1], h->part[2]}, h->sc,
                   t.flags + (size_t)3 * n * h->n, byte_off(t.alpha, (size_t)6 * n * h->esize),
                   byte_off(t.dt, (size_t)n * h->esize), nullptr};
    HW_CUDA(h, enqueue_step2d_io(h, io, h->stream));
  }
  hw::DevScalars sc;
  st = check_scalars(h, h->sc, &sc);
  if (t_out) *t_out = sc.t;
  if (st != HWENO_OK) return st;
  t.dt_host.assign(nsteps, 0.0);
  if (h->esize == 8) {
    HW_CUDA(h, cudaMemcpy(t.dt_host.data(), t.dt, sizeof(double) * nsteps, cudaMemcpyDeviceToHost));
  } else {
    std::vector<float> f(nsteps);
    HW_CUDA(h, cudaMemcpy(f.data(), t.dt, sizeof(float) * nsteps, cudaMemcpyDeviceToHost));
    for (int n = 0; n < nsteps; ++n) t.dt_host[n] = f[n];
  }
  t.nsteps = nsteps;
  t.every = checkpoint_every;
  t.nck = nck;
  return HWENO_OK;
}

hweno_status hweno_backward(hweno_handle h, const void* grad_out, void* grad_in, int dtype,
                            int on_device) {
  if (!h) return fail(nullptr, HWENO_ERR_ARG, "handle is NULL");
  hweno_ctx::Tape& t = h->tape;
  if (t.nsteps < 1) return fail(h, HWENO_ERR_STATE, "hweno_backward without a recorded run");
  if (!grad_out || !grad_in) return fail(h, HWENO_ERR_ARG, "grad_out and grad_in are required");
  if (dtype != HWENO_FP32 && dtype != HWENO_FP64) return fail(h, HWENO_ERR_ARG, "unknown dtype");
  hweno_status st = adjoint_scratch(h);
  if (st != HWENO_OK) return st;
  const size_t sbytes = h->elems * h->esize;
  if (t.seg_every < t.every) {
    free_ptr(&t.seg);
    HW_CUDA(h, cudaMalloc(&t.seg, sbytes * (3 * (size_t)t.every + 1)));
    t.seg_every = t.every;
  }
  if (!t.w0) HW_CUDA(h, cudaMalloc(&t.w0, sbytes));
  for (int k = 0; k < 2; ++k)
    if (!t.lam[k]) HW_CUDA(h, cudaMalloc(&t.lam[k], sbytes));
  if (!t.acc) HW_CUDA(h, cudaMalloc(&t.acc, sbytes));
  if (!t.slots) HW_CUDA(h, cudaMalloc(reinterpret_cast<void**>(&t.slots), sizeof(double) * 6 * hw::kAlphaSlots));
  const int src64 = dtype == HWENO_FP64, k64 = h->cfg.precision == HWENO_FP64;
  // the adjoint of the final state, in the kernel precision
  const void* src = grad_out;
  if (!on_device) {
    void* dst = src64 == k64 ? t.lam[0] : h->stage_buf;
    HW_CUDA(h, cudaMemcpyAsync(dst, grad_out, h->elems * (src64 ? 8 : 4), cudaMemcpyHostToDevice,
                               h->stream));
    src = src64 == k64 ? nullptr : h->stage_buf;
  }
  if (src) HW_CUDA(h, hw::launch_convert(src, src64, t.lam[0], k64, h->elems, h->stream));
  HW_CUDA(h, hw::launch_set_scalars(t.sc, 1, -1.0, h->stream));
  void* cur = t.lam[0];
  void* oth = t.lam[1];
  const size_t pair = 2 * h->esize;
  for (int seg = t.nck - 1; seg >= 0; --seg) {
    const int n0 = seg * t.every, n1 = n0 + t.every < t.nsteps ? n0 + t.every : t.nsteps;
    // recompute the segment's stage inputs from its checkpoint
    HW_CUDA(h, cudaMemcpyAsync(t.seg, byte_off(t.ck, sbytes * seg), sbytes, cudaMemcpyDeviceToDevice,
                               h->stream));
    // (each stage takes its recorded alpha and flags: the stage inputs are
    // bitwise those of the recorded run, and no alpha slots are needed)
    double* sl[3] = {t.slots, t.slots + 2 * hw::kAlphaSlots, t.slots + 4 * hw::kAlphaSlots};
    for (int n = n0; n < n1; ++n) {
      if (!(t.dt_host[n] > 0.0)) break;  // past t_final: the remaining steps did nothing
      const size_t m = (size_t)(n - n0);
      Step2DIO io = {byte_off(t.seg, sbytes * 3 * m), byte_off(t.seg, sbytes * (3 * m + 1)),
                     byte_off(t.seg, sbytes * (3 * m + 2)), byte_off(t.seg, sbytes * (3 * m + 3)),
                     t.w0, {sl[0], sl[1], sl[2]}, t.sc, nullptr, nullptr, nullptr,
                     byte_off(t.dt, (size_t)n * h->esize)};
      io.flags_in = t.flags + (size_t)3 * n * h->n;
      io.alpha_in = byte_off(t.alpha, (size_t)6 * n * h->esize);
      HW_CUDA(h, enqueue_step2d_io(h, io, h->stream));
    }
    // the adjoint stages, last step first
    for (int n = n1 - 1; n >= n0; --n) {
      if (!(t.dt_host[n] > 0.0)) continue;
      const size_t m = (size_t)(n - n0);
      hw::Adj2DArgs a = base_adj_args(h);
      a.dt = byte_off(t.dt, (size_t)n * h->esize);
      a.acc = t.acc;
      for (int stage = 3; stage >= 1; --stage) {
        const size_t ks = (size_t)3 * n + (stage - 1);
        a.stage = stage;
        a.w = byte_off(t.seg, sbytes * (3 * m + stage - 1));
        a.flags = t.flags + ks * h->n;
        a.alpha = byte_off(t.alpha, ks * pair);
        a.lam = cur;
        a.lam_in = oth;
        HW_CUDA(h, hw::launch_adj2d(a, h->stream));
        void* x = cur;
        cur = oth;
        oth = x;
      }
    }
  }
  hw::DevScalars sc;
  st = check_scalars(h, t.sc, &sc);
  if (st != HWENO_OK) return st;
  const int d64 = dtype == HWENO_FP64;
  if (on_device) {
    HW_CUDA(h, hw::launch_convert(cur, k64, grad_in, d64, h->elems, h->stream));
  } else {
    const void* from = cur;
    if (d64 != k64) {
      HW_CUDA(h, hw::launch_convert(cur, k64, h->stage_buf, d64, h->elems, h->stream));
      from = h->stage_buf;
    }
    HW_CUDA(h, cudaMemcpyAsync(grad_in, from, h->elems * (d64 ? 8 : 4), cudaMemcpyDeviceToHost,
                               h->stream));
  }
  HW_CUDA(h, cudaStreamSynchronize(h->stream));
  return HWENO_OK;
}

hweno_status hweno_rhs_vjp(hweno_handle h, const void* in, const uint8_t* flags, double alpha_x,
                           double alpha_y, const void* lam, void* grad) {
  if (!h) return fail(nullptr, HWENO_ERR_ARG, "handle is NULL");
  hweno_status st = check_adjoint_config(h);
  if (st != HWENO_OK) return st;
  if (!in || !flags || !lam || !grad) return fail(h, HWENO_ERR_ARG, "in, flags, lam and grad are required");
  if (grad == in || grad == lam) return fail(h, HWENO_ERR_ARG, "grad must not overlap in or lam");
  st = adjoint_scratch(h);
  if (st != HWENO_OK) return st;
  if (h->esize == 8) {
    const double al[2] = {alpha_x, alpha_y};
    HW_CUDA(h, cudaMemcpy(h->tape.aux, al, sizeof(al), cudaMemcpyHostToDevice));
  } else {
    const float al[2] = {(float)alpha_x, (float)alpha_y};
    HW_CUDA(h, cudaMemcpy(h->tape.aux, al, sizeof(al), cudaMemcpyHostToDevice));
  }
  hw::Adj2DArgs a = base_adj_args(h);
  a.stage = 0;
  a.w = in;
  a.flags = flags;
  a.alpha = h->tape.aux;
  a.dt = h->tape.aux;
  a.lam = lam;
  a.lam_in = grad;
  HW_CUDA(h, hw::launch_set_scalars(h->tape.sc, 1, -1.0, h->stream));
  HW_CUDA(h, hw::launch_adj2d(a, h->stream));
  hw::DevScalars sc;
  return check_scalars(h, h->tape.sc, &sc);
}

hweno_status hweno_totals(hweno_handle h, double* totals) {
  if (!h) return fail(nullptr, HWENO_ERR_ARG, "handle is NULL");
  if (!totals) return fail(h, HWENO_ERR_ARG, "totals is NULL");
  if (!h->has_state) return fail(h, HWENO_ERR_STATE, "hweno_totals before hweno_set_state");
  constexpr int kBlocks = 304;  // 2 per SM
  const int C = h->C;
  if (!h->tot_buf)
    HW_CUDA(h, cudaMalloc(reinterpret_cast<void**>(&h->tot_buf), sizeof(double) * (kBlocks + 1) * 8));
  double* part = h->tot_buf;
  double* out = h->tot_buf + kBlocks * 8;
  const int fp64 = h->cfg.precision == HWENO_FP64;
  const int ninst = h->n_batch > 0 ? h->n_batch : 1;
  for (int b = 0; b < ninst; ++b) {
    long long n, off = 0;
    double cell;
    if (h->n_batch > 0) {
      n = h->batch_nx[b];
      off = h->batch_inst[b].off;
      cell = (h->cfg.x1 - h->cfg.x0) / n;
    } else if (h->dim == 2) {
      n = h->n;
      cell = (h->cfg.x1 - h->cfg.x0) / h->cfg.nx * ((h->cfg.y1 - h->cfg.y0) / h->cfg.ny);
    } else {
      n = h->n;
      cell = (h->cfg.x1 - h->cfg.x0) / h->cfg.nx;
    }
    const long long stride = (long long)h->M * n;  // [c][m][cells]: component c's averages
    HW_CUDA(h, hw::launch_totals(byte_off(h->U[0], (size_t)off * h->esize), fp64, stride, C, n, part,
                                 kBlocks, out, h->stream));
    double sums[8], lows[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    HW_CUDA(h, cudaMemcpyAsync(sums, out, sizeof(double) * C, cudaMemcpyDeviceToHost, h->stream));
    if (h->comp) {  // the averages' low parts, [c][cells]
      HW_CUDA(h, cudaStreamSynchronize(h->stream));
      HW_CUDA(h, hw::launch_totals(h->Ulo, 0, n, C, n, part, kBlocks, out, h->stream));
      HW_CUDA(h, cudaMemcpyAsync(lows, out, sizeof(double) * C, cudaMemcpyDeviceToHost, h->stream));
    }
    HW_CUDA(h, cudaStreamSynchronize(h->stream));
    for (int c = 0; c < C; ++c) totals[(size_t)b * C + c] = (sums[c] + lows[c]) * cell;
  }
  return HWENO_OK;
}

hweno_status hweno_set_execution(hweno_handle h, int threads, int persistent) {
  if (!h) return fail(nullptr, HWENO_ERR_ARG, "handle is NULL");
  if (h->dim != 1) return fail(h, HWENO_ERR_ARG, "the execution choice is for 1D handles");
  if (threads != 128 && threads != 256 && threads != 512)
    return fail(h, HWENO_ERR_ARG, "threads must be 128, 256 or 512");
  if (persistent < 0 || persistent > 2) return fail(h, HWENO_ERR_ARG, "persistent must be 0, 1 or 2");
  if (h->comp && (persistent != 2 || threads == 128))
    return fail(h, HWENO_ERR_ARG, "HWENO_FP32C runs as the resident launch (2) with 256 or 512 threads");
  HW_CUDA(h, cudaStreamSynchronize(h->stream));
  if (h->g_many) cudaGraphExecDestroy(h->g_many);
  if (h->g_one) cudaGraphExecDestroy(h->g_one);
  h->g_many = h->g_one = nullptr;
  h->nth1d = threads;
  h->persist1d = persistent;
  if (h->n_batch > 0) {
    HW_CUDA(h, batch_tiles(h, threads));
  } else {
    h->ntile = (h->n + threads - 7) / (threads - 6);
  }
  if (persistent == 2) {
    HW_CUDA(h, prepare_resident(h));
    if (h->res_tile == 0) {
      h->persist1d = 0;
      return fail(h, HWENO_ERR_ARG,
                  "the resident launch takes FP32 single-instance handles, 256 or 512 threads, "
                  "and a grid whose tiles fit on the GPU at once");
    }
  }
  return HWENO_OK;
}

hweno_status hweno_autotune(hweno_handle h, int nsteps_trial, int* choice_out) {
  if (!h) return fail(nullptr, HWENO_ERR_ARG, "handle is NULL");
  if (h->dim != 1) return fail(h, HWENO_ERR_ARG, "hweno_autotune tunes 1D handles");
  if (!h->has_state) return fail(h, HWENO_ERR_STATE, "hweno_autotune before hweno_set_state");
  if (nsteps_trial < 1) return fail(h, HWENO_ERR_ARG, "nsteps_trial must be >= 1");
  const size_t sbytes = h->elems * h->esize;
  const size_t nslot = h->n_batch > 2 * hw::kAlphaSlots ? (size_t)h->n_batch : 2 * hw::kAlphaSlots;
  const size_t pbytes = sizeof(double) * nslot;
  const size_t bbytes = sizeof(hw::BatchScalars) * (size_t)h->n_batch;
  const size_t lbytes = h->comp ? sizeof(float) * h->C * h->n : 0;
  // everything a run changes, saved on the device and put back before each trial
  char* save = nullptr;
  HW_CUDA(h, cudaMalloc(&save, sbytes + 3 * pbytes + sizeof(hw::DevScalars) + bbytes + lbytes));
  char* sv_u = save;
  char* sv_p = save + sbytes;
  char* sv_sc = sv_p + 3 * pbytes;
  char* sv_b = sv_sc + sizeof(hw::DevScalars);
  char* sv_l = sv_b + bbytes;
  cudaStream_t s = h->stream;
  auto copy_all = [&](bool to_save) -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(to_save ? sv_u : h->U[0], to_save ? h->U[0] : sv_u, sbytes,
                                    cudaMemcpyDeviceToDevice, s);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k)
      e = cudaMemcpyAsync(to_save ? sv_p + k * pbytes : (char*)h->part[k],
                          to_save ? (char*)h->part[k] : sv_p + k * pbytes, pbytes,
                          cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(to_save ? sv_sc : (char*)h->sc, to_save ? (char*)h->sc : sv_sc,
                          sizeof(hw::DevScalars), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && bbytes)
      e = cudaMemcpyAsync(to_save ? sv_b : (char*)h->d_bsc, to_save ? (char*)h->d_bsc : sv_b,
                          bbytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && lbytes)
      e = cudaMemcpyAsync(to_save ? sv_l : (char*)h->Ulo, to_save ? (char*)h->Ulo : sv_l, lbytes,
                          cudaMemcpyDeviceToDevice, s);
    return e;
  };
  auto configure = [&](int nth, int persist) -> cudaError_t {
    if (h->g_many) cudaGraphExecDestroy(h->g_many);
    if (h->g_one) cudaGraphExecDestroy(h->g_one);
    h->g_many = h->g_one = nullptr;
    h->nth1d = nth;
    h->persist1d = persist;
    if (h->n_batch > 0) return batch_tiles(h, nth);
    h->ntile = (h->n + nth - 7) / (nth - 6);
    if (persist == 2) return prepare_resident(h);
    return cudaSuccess;
  };
  cudaError_t e = copy_all(true);
  const int cand_nth[3] = {128, 256, 512};
  float best = -1.0f;
  int best_nth = h->nth1d, best_persist = h->persist1d;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  for (int persist = h->comp ? 2 : 0; persist < 3 && e == cudaSuccess; ++persist)
    for (int ci = h->comp ? 1 : 0; ci < 3 && e == cudaSuccess; ++ci) {
      e = configure(cand_nth[ci], persist);
      if (e != cudaSuccess) break;
      if (persist == 2 && h->res_tile == 0) continue;  // not available here
      // one untimed run of the trial length (it builds every graph the trial
      // launches, so that no graph instantiation is timed), then the best of
      // two timed trials
      hweno_status st = HWENO_OK;
      float ms = -1.0f;
      for (int rep = 0; rep < 3 && st == HWENO_OK && e == cudaSuccess; ++rep) {
        e = copy_all(false);
        if (e == cudaSuccess && rep > 0) e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) st = hweno_step(h, nsteps_trial, -1.0, nullptr);
        if (e == cudaSuccess && rep > 0) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess && st == HWENO_OK && rep > 0) {
          float t = 0.0f;
          e = cudaEventSynchronize(e1);
          if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
          if (e == cudaSuccess && (ms < 0.0f || t < ms)) ms = t;
        }
      }
      if (e != cudaSuccess) break;
      if (st != HWENO_OK) {
        cudaFree(save);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return st;
      }
      if (best < 0.0f || ms < best) {
        best = ms;
        best_nth = cand_nth[ci];
        best_persist = persist;
      }
    }
  if (e == cudaSuccess) e = configure(best_nth, best_persist);
  if (e == cudaSuccess) e = copy_all(false);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(save);
  if (e != cudaSuccess) return fail(h, HWENO_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
  hw::DevScalars sc;
  hweno_status st = check_scalars(h, h->sc, &sc);
  if (choice_out) {
    choice_out[0] = best_nth;
    choice_out[1] = best_persist;
  }
  return st;
}

hweno_status hweno_check_barrier(int ctas, int meetings, int missing, unsigned polls) {
  if (ctas < 1 || ctas > 1024 || meetings < 1 || meetings > 1000000 || missing < 0 ||
      missing > 1024 || polls < 1u)
    return fail(nullptr, HWENO_ERR_ARG,
                "hweno_check_barrier: need 1 <= ctas <= 1024, 1 <= meetings <= 1e6, "
                "0 <= missing <= 1024, polls >= 1");
  unsigned* bar = nullptr;
  hw::DevScalars* sc = nullptr;
  cudaStream_t s = nullptr;
  bool too_many = false;
  hw::DevScalars host;
  memset(&host, 0, sizeof(host));
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&bar), 2 * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&sc), sizeof(hw::DevScalars));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMemsetAsync(sc, 0, sizeof(hw::DevScalars), s);
  if (e == cudaSuccess)
    e = hw::launch_barrier_check(ctas, meetings, missing, polls, bar, sc, s, &too_many);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&host, sc, sizeof(host), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (s) cudaStreamDestroy(s);
  if (sc) cudaFree(sc);
  if (bar) cudaFree(bar);
  if (e != cudaSuccess)
    return fail(nullptr, HWENO_ERR_CUDA, std::string("hweno_check_barrier: ") + cudaGetErrorString(e));
  if (too_many)
    return fail(nullptr, HWENO_ERR_ARG, "hweno_check_barrier: more CTAs than can be resident");
  if (host.status & hw::ST_TIMEOUT)
    return fail(nullptr, HWENO_ERR_TIMEOUT, "hweno_check_barrier: a bounded barrier wait ran out");
  return HWENO_OK;
}

hweno_status hweno_check_resident(hweno_handle h, int nsteps, int silent_cta, unsigned polls) {
  if (!h) return fail(nullptr, HWENO_ERR_ARG, "handle is NULL");
  if (h->dim != 1 || h->persist1d != 2 || h->res_tile == 0)
    return fail(h, HWENO_ERR_ARG, "hweno_check_resident: set the resident launch first");
  if (!h->has_state) return fail(h, HWENO_ERR_STATE, "hweno_check_resident before hweno_set_state");
  if (nsteps < 1 || silent_cta < -1 || silent_cta >= h->res_ncta || polls < 1u)
    return fail(h, HWENO_ERR_ARG,
                "hweno_check_resident: need nsteps >= 1, -1 <= silent_cta < CTAs, polls >= 1");
  HW_CUDA(h, hw::launch_set_scalars(h->sc, 0, -1.0, h->stream));
  HW_CUDA(h, enqueue_resident1d(h, nsteps, h->stream, silent_cta, polls));
  hw::DevScalars host;
  return check_scalars(h, h->sc, &host);  // HWENO_ERR_TIMEOUT when a wait ran out
}

const char* hweno_last_error(hweno_handle h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

}  // extern "C"
