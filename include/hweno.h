/*
 * hweno.h -- C ABI of the GB300 (sm_103a) hybrid Hermite WENO library.
 *
 * The library evolves the zeroth and first moments of 1D and 2D conservation
 * laws (scalar Burgers, compressible Euler) with the fifth-order hybrid HWENO
 * scheme with artificial linear weights of Zhao & Qiu, "A Hermite WENO scheme
 * with artificial linear weights for hyperbolic conservation laws"
 * (arXiv:2002.08816):
 *   - semi-discrete moment scheme, Eq. (odeH) (1D) and Eq. (ode2) (2D);
 *   - KXRCF troubled-cell detection and first-moment modification, Steps 1, 4;
 *   - hybrid reconstruction: linear p0 on smooth stencils (Steps 2.2, 5.2),
 *     HWENO nonlinear combination with any positive linear weights summing to
 *     one on stencils holding a troubled cell (Steps 2.1, 5.1), linear values
 *     at interior quadrature points (Steps 2.3, 5.3);
 *   - global Lax-Friedrichs flux, Gauss(-Lobatto) quadratures, Sec. 2.1/2.2;
 *   - third-order TVD Runge-Kutta, Eq. (RK), with a device-side CFL step.
 *
 * Every call takes plain pointers and sizes; no C++ or torch type crosses it.
 * Errors are returned as hweno_status; no exception leaves the library.  A
 * handle may be used from one host thread at a time.
 *
 * Layout of a state ("moments") buffer, structure of arrays, no padding:
 *   1D: element (c, m, i)    at ((c*2 + m)*nx + i)
 *   2D: element (c, m, j, i) at (((c*3 + m)*ny + j)*nx + i)
 * with c the conserved component (Burgers: u; 1D Euler: rho, rho*mu, E;
 * 2D Euler: rho, rho*mu, rho*nu, E) and m the moment: 0 the cell average
 * (1/|I|) int u, 1 the x-moment (1/|I|) int u (x-x_i)/dx, 2 (2D) the
 * y-moment (1/|I|) int u (y-y_j)/dy (Sec. 2.1 after Eq. (odeH); Sec. 2.2
 * after Eq. (ode2)).
 */
#ifndef HWENO_H
#define HWENO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HWENO_OK = 0,
  HWENO_ERR_ARG = 1,           /* invalid argument or configuration */
  HWENO_ERR_CUDA = 2,          /* a CUDA runtime call failed */
  HWENO_ERR_NONPHYSICAL = 3,   /* non-finite value, rho <= 0 or p <= 0 seen */
  HWENO_ERR_TIMEOUT = 4,       /* a bounded device wait gave up */
  HWENO_ERR_STATE = 5,         /* call out of order (e.g. step before set_state) */
  HWENO_ERR_TOO_LARGE = 6      /* more cells than hweno_rhs1d_noalloc's fixed scratch holds */
} hweno_status;

enum { HWENO_BURGERS = 0, HWENO_EULER = 1 };
enum { HWENO_BC_PERIODIC = 0, HWENO_BC_OUTFLOW = 1, HWENO_BC_REFLECTIVE = 2 };
enum { HWENO_TROUBLED_HYBRID = 0, HWENO_TROUBLED_ALL = 1, HWENO_TROUBLED_NONE = 2 };
/* Precision of the bulk arithmetic.  HWENO_FP32C (single-instance handles,
 * 1D and 2D): FP32 arithmetic with the cell averages carried as float pairs
 * (hi + lo) between stages and the operator formed on increments over each
 * cell's hi, so that no FP32 rounding of an average reaches the first moments'
 * right-hand side (whose response to the averages has a factor 1/dx).  1D
 * steps run as the resident launch (a grid that does not fit on the GPU at
 * once is refused); 2D steps run the stage kernels with the low parts beside
 * each stage buffer.  Its state buffers are FP32 (hi); get_state with
 * HWENO_FP64 returns hi + lo, set_state from HWENO_FP64 keeps the low parts.
 * hweno_rhs and hweno_rhs1d_noalloc evaluate the FP32 operator on the caller's
 * FP32 buffers; batches and the adjoint take HWENO_FP32 or HWENO_FP64.  As a
 * dtype (set_state, get_state, backward) only HWENO_FP32 and HWENO_FP64
 * exist. */
enum { HWENO_FP32 = 0, HWENO_FP64 = 1, HWENO_FP32C = 2 };

typedef struct {
  int dim;                /* 1 or 2 */
  int system;             /* HWENO_BURGERS or HWENO_EULER */
  int nx, ny;             /* cells per direction (ny ignored for dim 1); nx, ny >= 4;
                             2D cells must be square: (x1-x0)/nx = (y1-y0)/ny */
  double x0, x1, y0, y1;  /* domain [x0,x1] x [y0,y1] */
  int bc;                 /* HWENO_BC_PERIODIC or HWENO_BC_OUTFLOW on all sides, or
                             HWENO_BC_REFLECTIVE (solid walls; 1D Euler only): a ghost
                             is the mirror image of an interior cell, density and
                             energy even, momentum odd */
  double gas_gamma;       /* ratio of specific heats (Euler), > 1 */
  double lin_w[5];        /* linear weights gamma_0..gamma_2 (1D) or ..gamma_4 (2D):
                             all > 0, |sum - 1| <= 1e-12 (Sec. 2.1 Step 1) */
  double cfl;             /* CFL number of the time step, > 0 */
  double eps;             /* epsilon of the nonlinear weights (paper: 1e-6), > 0 */
  double kxrcf_threshold; /* troubled iff KXRCF indicator > threshold (1) */
  int troubled_mode;      /* HWENO_TROUBLED_HYBRID (the paper's scheme), _ALL, _NONE */
  int n_gauss;            /* 2D quadrature points per direction: 3 (paper) or 2 */
  int precision;          /* HWENO_FP32, HWENO_FP64 or HWENO_FP32C bulk arithmetic */
  int variant;            /* 0, or HWENO_VARIANT_* bits (readings the paper leaves open) */
} hweno_config;

/* Variants of two points the paper leaves open (0 = the readings used
 * throughout: the modified first moments are stored in the state, and the
 * characteristic fields are those of the cell average). */
#define HWENO_VARIANT_RAW_COMBINE 1  /* the RK combination uses the unmodified first moments */
#define HWENO_VARIANT_MEAN_EIGEN 2   /* Euler HWENO interface values in the characteristic
                                        fields of the mean of the two averages at that
                                        interface (one eigen-system per interface) */

typedef struct hweno_ctx* hweno_handle;

/* Fills cfg with the paper's defaults for the given dimension and system:
 * gamma = 1.4, linear weights (0.98, 0.01, 0.01) in 1D and (0.96, 0.01 x 4)
 * in 2D (Sec. 3.2), CFL 0.6 (Sec. 3), eps = 1e-6, threshold 1, hybrid mode,
 * three Gauss points, FP32, periodic, unit domain.  Sizes are left at 0. */
void hweno_default_config(hweno_config* cfg, int dim, int system);

/* Validates cfg, allocates every device buffer the scheme needs (the library
 * owns them) and binds the handle to cuda_stream (a cudaStream_t; NULL = the
 * legacy default stream).  *out is set only on HWENO_OK.  Returns
 * HWENO_ERR_ARG for an invalid configuration (see hweno_config). */
hweno_status hweno_create(const hweno_config* cfg, void* cuda_stream, hweno_handle* out);

/* Copies a state in the layout above into the handle and sets t = 0.
 * moments: host (on_device = 0) or device (on_device = 1) pointer, caller
 * owned, element type dtype (HWENO_FP32 / HWENO_FP64; converted when it
 * differs from the configured precision).  Asynchronous with respect to the
 * host for device sources; a host source is staged through a synchronous
 * copy.  The state must hold the moments defined in Sec. 2 (the helper
 * module workloads.py projects point data by Gauss quadrature). */
hweno_status hweno_set_state(hweno_handle h, const void* moments, int dtype, int on_device);

/* Enqueues nsteps third-order TVD Runge-Kutta steps (Eq. (RK)) on the bound
 * stream.  dt = cfl * dx / alpha (1D) or cfl / (alpha_x/dx + alpha_y/dy) (2D)
 * from the state at the start of each step, computed and kept on the device;
 * with t_final > 0 the step is clipped so that t does not pass t_final and
 * steps after t_final do nothing.  t_out NULL: returns without waiting.
 * t_out non-NULL: waits for the stream, stores the time reached, and returns
 * HWENO_ERR_NONPHYSICAL if any stage saw a non-finite or non-physical value. */
hweno_status hweno_step(hweno_handle h, int nsteps, double t_final, double* t_out);

/* One evaluation of the right-hand side L of Eq. (odeH)/(ode2) on caller
 * device buffers in the configured precision (FP32 for HWENO_FP32C) and the
 * state layout: out =
 * L(in) with alpha from in.  flags_out (nullable, nx*ny bytes) receives the
 * troubled-cell flags (1 = troubled); ulim_out (nullable, state layout)
 * receives in with the first moments of troubled cells modified (Step 1/4).
 * in, out and ulim_out must not overlap.  Waits for the stream and returns
 * HWENO_ERR_NONPHYSICAL on a non-finite result. */
hweno_status hweno_rhs(hweno_handle h, const void* in, void* out, uint8_t* flags_out,
                       void* ulim_out);

/* Copies the current state out (host or device pointer, caller owned, dtype
 * as in set_state).  A host destination makes the call wait for the stream. */
hweno_status hweno_get_state(hweno_handle h, void* out, int dtype, int on_device);

/* Statistics since set_state: the time reached, the last dt, the number of
 * completed steps and of troubled cell-stages.  Waits for the stream. */
hweno_status hweno_stats(hweno_handle h, double* t, double* last_dt, int64_t* steps,
                         int64_t* troubled_cell_stages);

/* Largest nx that hweno_rhs1d_noalloc accepts: its scratch is a fixed array
 * of one double per 250-cell tile (about 131 KiB) plus a 64-byte status block. */
#define HWENO_NOALLOC_MAX_CELLS 4194304

/* hweno_rhs for 1D without any device allocation.  The paper has no
 * counterpart; this exists for callers that cannot let a library call
 * cudaMalloc: a framework whose device memory is owned by its own pool
 * allocator (an allocation behind the pool's back is not accounted and can
 * fail when the pool has reserved the memory), a process whose device memory
 * is budgeted allocation by allocation, or a latency-bound loop that cannot
 * afford the device synchronisation an allocation or a free may cause.
 * It needs no handle: cfg (dim must be 1) passes the checks of hweno_create
 * (every boundary condition, variant and precision hweno_create accepts for
 * 1D) and cuda_stream is the stream to run on (NULL: legacy default stream).
 * in, out, flags_out and ulim_out mean exactly what they mean for hweno_rhs
 * (caller-owned device buffers in cfg->precision, FP32 for HWENO_FP32C;
 * flags_out and ulim_out
 * nullable; no overlap), and the result is the same L(in).
 * Scratch: a file-scope __device__ array inside the library, which every GPU
 * that loads the library holds until the process exits; every call looks up
 * its device address on the current device (cudaGetSymbolAddress), so a
 * device reset leaves nothing stale behind.  Every call shares the one array and each call resets the part that must start at zero, so calls
 * that overlap on the GPU (other streams, other host threads) race and must
 * be serialised by the caller.
 * Returns HWENO_ERR_TOO_LARGE when cfg->nx > HWENO_NOALLOC_MAX_CELLS,
 * HWENO_ERR_ARG for any other invalid argument, HWENO_ERR_NONPHYSICAL for a
 * non-finite or non-physical result; copies the status word to the host and
 * waits for the stream before returning. */
hweno_status hweno_rhs1d_noalloc(const hweno_config* cfg, void* cuda_stream, const void* in,
                                 void* out, uint8_t* flags_out, void* ulim_out);

/* A batch of n_batch independent 1D problems of nx[b] cells each (nx[b] >= 4),
 * sharing every other field of cfg (dim must be 1; cfg->nx is ignored); each
 * instance covers [x0, x1] with its own dx, alpha, dt and time (the scheme of
 * Sec. 2.1 applied to each instance separately).  All instances advance in
 * the same launches.  The state layout is the instances' 1D states one after
 * the other (instance b at offset 2 C sum_{b'<b} nx[b']).  set_state,
 * get_state, step and stats work as for one instance (stats report instance
 * 0's time); hweno_rhs is not available on a batch. */
hweno_status hweno_create_batch(const hweno_config* cfg, int n_batch, const int* nx,
                                void* cuda_stream, hweno_handle* out);

/* The time reached by every instance of a batch (t: n_batch doubles).  Waits
 * for the stream. */
hweno_status hweno_batch_times(hweno_handle h, double* t);

/* ---- Adjoint (2D, periodic boundaries) --------------------------------
 * The derivative of the Runge-Kutta map with the scheme's switches held
 * fixed: the troubled cells of every stage, the Lax-Friedrichs speeds
 * (alpha_x, alpha_y) of every stage and the dt of every step are those of the
 * recorded forward run (Sec. 2.2 Steps 4-6 with Eq. (ode2) and Eq. (RK)).  The
 * paper defines no adjoint; the derivative is of the discrete scheme as it
 * runs.  Where an absolute value in tau (Eq. (tao4), Eq. (tao5)) has a kink,
 * the derivative with sign(0) = 0 is taken. */

/* Like hweno_step (from the current state, t_final as there), and records
 * the switches and every checkpoint_every-th state for hweno_backward.  The
 * tape (3 nsteps nx ny bytes of flags, ceil(nsteps / checkpoint_every)
 * states, a few scalars per step) belongs to the handle and is replaced by
 * the next hweno_record.  Waits for the stream; returns HWENO_ERR_ARG unless
 * dim == 2, bc == HWENO_BC_PERIODIC, nsteps >= 1 and checkpoint_every >= 1,
 * HWENO_ERR_STATE before set_state, HWENO_ERR_NONPHYSICAL as hweno_step. */
hweno_status hweno_record(hweno_handle h, int nsteps, int checkpoint_every, double t_final,
                          double* t_out);

/* Vector-Jacobian product of the recorded run: grad_in = (d u_N / d u_0)^T
 * grad_out, with u_0 the state hweno_record started from and u_N the state
 * it ended at (state layout, element type dtype, host or device pointers as
 * in set_state; caller owned).  Recomputes each checkpoint segment forward
 * (3 checkpoint_every + 1 states of scratch) and runs the adjoint stages
 * backwards through it.  The current state is not changed.  Waits for the
 * stream; HWENO_ERR_STATE without a recorded run. */
hweno_status hweno_backward(hweno_handle h, const void* grad_out, void* grad_in, int dtype,
                            int on_device);

/* Vector-Jacobian product of one operator evaluation: grad = (d L(in)/d in)^T
 * lam, L as in hweno_rhs (Step 4 included) but with the troubled cells given
 * (flags, nx*ny bytes, 1 = troubled) and alpha_x, alpha_y given.  Device
 * pointers in the configured precision; grad must not overlap in or lam.
 * Waits for the stream. */
hweno_status hweno_rhs_vjp(hweno_handle h, const void* in, const uint8_t* flags, double alpha_x,
                           double alpha_y, const void* lam, void* grad);

/* Chooses how a 1D handle (single instance or batch) runs its steps: per-
 * stage launches captured in CUDA graphs, or one persistent cooperative
 * launch per hweno_step call (every CTA walks its tiles of a stage, then the
 * grid meets at a barrier whose wait is bounded), each with 128, 256 or 512
 * threads per CTA (a tile is that number minus 6 cells), and, for FP32
 * single-instance handles whose tiles fit on the GPU at once, one resident
 * launch per hweno_step call with 256 or 512 threads per CTA (every CTA keeps
 * its tile in shared memory for the whole run and exchanges only 3-cell halos
 * and its maximum wave speed with the others, all waits bounded).  Each
 * candidate advances the current state nsteps_trial steps once untimed (which
 * builds its graphs) and then twice timed with CUDA events on the handle's
 * stream; the one with the fastest trial is kept for later calls; the
 * state, time, counters and wave-speed slots are restored afterwards.  The
 * per-stage candidates give bitwise the same results; the persistent and
 * resident ones agree with them to rounding (their copy of the stage body may
 * contract a few multiply-adds differently).  The paper has no counterpart (it
 * fixes no hardware mapping).  choice_out (nullable, 2 ints) receives the
 * threads per CTA and the launch kind (0 graphs, 1 persistent, 2 resident).
 * New handles start with 256 threads and per-stage graphs (HWENO_FP32C: the
 * resident launch, the only one it has; its autotuner times 256 and 512
 * threads).  Waits for the stream; HWENO_ERR_ARG for 2D handles,
 * HWENO_ERR_STATE before set_state. */
hweno_status hweno_autotune(hweno_handle h, int nsteps_trial, int* choice_out);

/* Failure-detection self-test of the grid barrier the persistent launch uses
 * between stages (no counterpart in the paper).  ctas co-resident CTAs of 128
 * threads (a cooperative launch) meet `meetings` times; each meeting waits for
 * ctas + missing arrivals, polling a counter in device memory at most `polls`
 * times.  With missing = 0 every meeting completes and the result is HWENO_OK;
 * with missing > 0 nothing ever supplies the extra arrivals, so every wait runs
 * out, each CTA records the timeout in a status word and returns, and the result
 * is HWENO_ERR_TIMEOUT: the context stays usable (the persistent launch ends
 * the same way, within about a second, when an arrival is lost).  The library
 * allocates and frees its own device memory and stream; waits for completion.
 * HWENO_ERR_ARG unless 1 <= ctas <= 1024, 1 <= meetings <= 1e6,
 * 0 <= missing <= 1024 and polls >= 1 (checked before any CUDA call), or when
 * ctas CTAs cannot all be resident.  The error text is hweno_last_error(NULL). */
hweno_status hweno_check_barrier(int ctas, int meetings, int missing, unsigned polls);

/* Failure-detection self-test of the resident launch (no counterpart in the
 * paper).  On a handle set to the resident launch (hweno_set_execution(h, 256
 * or 512, 2)) with a state, runs nsteps Runge-Kutta steps in one resident
 * launch in which CTA silent_cta (0 <= silent_cta < the launch's CTAs; -1:
 * none) never publishes the maximum wave speed of its outputs, and every wait
 * of the launch gives up after `polls` polls.  With a silent CTA no CTA can
 * form alpha: the waits run out, each CTA records the timeout in the status
 * word and leaves, the state is not written, and the result is
 * HWENO_ERR_TIMEOUT; the context stays usable (hweno_set_state resets the
 * status).  With silent_cta = -1 it is an ordinary run (HWENO_OK).  Waits for
 * the stream.  HWENO_ERR_ARG for another launch kind or invalid arguments,
 * HWENO_ERR_STATE before hweno_set_state. */
hweno_status hweno_check_resident(hweno_handle h, int nsteps, int silent_cta, unsigned polls);

/* Sets the choice hweno_autotune makes by hand: threads per CTA (128, 256 or
 * 512) and the launch kind: 0 per-stage launches in CUDA graphs, 1 one
 * persistent launch per hweno_step with a grid barrier between stages, 2 one
 * resident launch per hweno_step in which every CTA keeps its tile of the
 * state in shared memory for the whole run (FP32 single-instance handles, 256
 * or 512 threads, grids small enough for every tile to be on the GPU at once;
 * HWENO_ERR_ARG otherwise; HWENO_FP32C handles take only this kind).  1D
 * handles only; waits for the stream.  All choices compute the same scheme;
 * results agree to rounding (the per-stage choices bit for bit). */
hweno_status hweno_set_execution(hweno_handle h, int threads, int persistent);

/* The conserved totals of the current state: totals[c] = the sum over cells
 * of the average of component c times the cell size (dx, or dx dy in 2D),
 * accumulated in FP64 on the device in a fixed order (so repeatable to the
 * bit).  C values (Burgers 1, 1D Euler 3, 2D Euler 4); for a batch, n_batch
 * x C values, instance after instance.  With periodic boundaries the scheme
 * conserves them (Eq. (odeH), Eq. (ode2) are in flux form).  Waits for the
 * stream. */
hweno_status hweno_totals(hweno_handle h, double* totals);

/* Measures the fused multiply-add throughput of the current device for the
 * arithmetic roofline of the stage kernels (no counterpart in the paper, which
 * names no hardware): kind 0 FP32, 1 FP64, 2 packed FP32 (fma.rn.f32x2, two
 * FMAs per instruction; it shows whether the packed form used by the 2D
 * kernels raises the FP32 flop rate).  A kernel of eight independent FMA
 * chains per thread (kind 2: eight chains of pairs) on a grid that fills every
 * SM, each thread doing iters x 128 FMAs (kind 2: iters x 256), timed with
 * CUDA events after one untimed launch on a private stream; *flops_per_s =
 * 2 x FMAs / time, at whatever SM clock the GPU runs.  Allocates and frees a
 * small buffer; waits for completion.  HWENO_ERR_ARG unless 0 <= kind <= 2,
 * 1 <= iters <= 2^24 and flops_per_s is non-NULL. */
hweno_status hweno_fma_peak(int kind, int iters, double* flops_per_s);

/* Frees every device buffer of the handle; NULL is ignored. */
void hweno_destroy(hweno_handle h);

/* Text of the last error on this handle (or of the last failed create when
 * h is NULL); valid until the next call on the handle. */
const char* hweno_last_error(hweno_handle h);

#ifdef __cplusplus
}
#endif
#endif
