/*
 * ORACLE -- test infrastructure only.
 *
 * Plain, slow FP64 CPU restatement of the fifth-order hybrid Hermite WENO
 * scheme with artificial linear weights (Zhao & Qiu, arXiv:2002.08816).
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
 * load this library.  It shares no code, header or table with the CUDA path
 * in paper_2002_08816_gb300/: every reconstruction coefficient here is derived
 * at start-up from the moment conditions the paper states, by a dense linear
 * solve, never typed in.
 *
 * State layout (both dimensions): structure of arrays
 *   1D: u[(c*2 + m)*nx + i],           m = 0 cell average, 1 first moment
 *   2D: u[((c*3 + m)*ny + j)*nx + i],  m = 0 average, 1 x-moment, 2 y-moment
 * c runs over the conserved components: Burgers 1; 1D Euler (rho, rho*mu, E);
 * 2D Euler (rho, rho*mu, rho*nu, E).
 */
#ifndef HWENO_ORACLE_H
#define HWENO_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define HWO_BURGERS 0
#define HWO_EULER 1

#define HWO_BC_PERIODIC 0
#define HWO_BC_OUTFLOW 1
#define HWO_BC_REFLECTIVE 2 /* 1D Euler: a solid wall at each end */

#define HWO_TROUBLED_HYBRID 0 /* KXRCF decides (the "new hybrid HWENO" scheme) */
#define HWO_TROUBLED_ALL 1    /* every cell troubled (the "new HWENO" scheme, Sec. 3) */
#define HWO_TROUBLED_NONE 2   /* no cell troubled: purely linear scheme */

typedef struct {
  int system;             /* HWO_BURGERS or HWO_EULER */
  int nx;                 /* number of uniform cells */
  double x0, x1;          /* domain [x0, x1] */
  int bc;                 /* HWO_BC_* */
  double gas_gamma;       /* ratio of specific heats (Euler) */
  double lin_w[3];        /* artificial linear weights gamma_0..gamma_2 */
  double eps;             /* epsilon of the nonlinear weights (1e-6) */
  double kxrcf_threshold; /* troubled iff indicator > threshold (1) */
  int troubled_mode;      /* HWO_TROUBLED_* */
  int limit_in_place;     /* 1: the RK combination uses the limited first moments */
  int char_state;         /* 0: characteristic fields of the cell average (both
                             interfaces); 1: of the mean of the two averages at
                             each interface (the variant) */
} hwo1d_cfg;

typedef struct {
  int system;             /* HWO_BURGERS (f = g = u^2/2) or HWO_EULER */
  int nx, ny;
  double x0, x1, y0, y1;
  int bc;                 /* same condition on all four sides */
  double gas_gamma;
  double lin_w[5];        /* gamma_0..gamma_4 */
  double eps;
  double kxrcf_threshold;
  int troubled_mode;
  int limit_in_place;
  int n_gauss;            /* 3 (the paper) or 2 Gauss points per direction */
  int char_state;         /* as in 1D: 1 = fields of each interface's mean state */
} hwo2d_cfg;

/* ---------------- 1D ---------------- */
int hwo1d_ncomp(int system);
double hwo1d_alpha(const hwo1d_cfg* cfg, const double* u);
int hwo1d_rhs(const hwo1d_cfg* cfg, const double* u, double alpha, double* rhs,
              double* ulim, unsigned char* flags, double* indicator);
int hwo1d_rhs_ex(const hwo1d_cfg* cfg, const double* u, double alpha, double* rhs,
                 double* ulim, unsigned char* flags, double* indicator,
                 double* faces);
int hwo1d_step(const hwo1d_cfg* cfg, double* u, double dt, long* n_troubled);
double hwo1d_dt(const hwo1d_cfg* cfg, const double* u, double cfl, double t,
                double t_final);
int hwo1d_run(const hwo1d_cfg* cfg, double* u, int nsteps, double cfl,
              double t0, double t_final, double dt_fixed,
              const double* lin_w_per_step, double* t_out, long* n_troubled);

/* pieces exposed for the pin tests */
void hwo1d_limiter_candidates(const double ub[3], double v_m1, double v_p1,
                              double q[3], double beta[3]);
double hwo1d_limit_scalar(const double gam[3], double eps, const double ub[3],
                          double v_m1, double v_p1);
void hwo1d_recon_candidates(const double ub[3], const double vb[3],
                            double val[12], double beta[3]);
void hwo1d_recon_scalar(const double gam[3], double eps, const double ub[3],
                        const double vb[3], int hweno, double out[4]);
void hwo_euler1d_eigen(double g, const double U[3], double R[9], double L[9]);
void hwo_euler1d_flux(double g, const double U[3], double F[3]);

/* ---------------- 2D ---------------- */
int hwo2d_ncomp(int system);
int hwo2d_rhs(const hwo2d_cfg* cfg, const double* u, double alpha_x,
              double alpha_y, double* rhs, double* ulim, unsigned char* flags,
              double* indicator);
int hwo2d_rhs_ex(const hwo2d_cfg* cfg, const double* u, double alpha_x, double alpha_y,
                 double* rhs, double* ulim, unsigned char* flags, double* indicator,
                 double* points);
int hwo2d_rhs_fx(const hwo2d_cfg* cfg, const double* u, double alpha_x, double alpha_y,
                 const unsigned char* flags_in, double* rhs, double* ulim,
                 unsigned char* flags, double* indicator, double* points);
void hwo2d_alpha(const hwo2d_cfg* cfg, const double* u, double* ax, double* ay);
double hwo2d_dt(const hwo2d_cfg* cfg, const double* u, double cfl, double t,
                double t_final);
int hwo2d_step(const hwo2d_cfg* cfg, double* u, double dt, long* n_troubled);
int hwo2d_run(const hwo2d_cfg* cfg, double* u, int nsteps, double cfl,
              double t0, double t_final, double dt_fixed,
              const double* lin_w_per_step, double* t_out, long* n_troubled);
int hwo2d_recon_candidates(const double ub[9], const double vb[9],
                           const double wb[9], int n_gauss, double* val,
                           double beta[5]);
int hwo2d_linear_weights(int n_gauss, double* W);
void hwo2d_p0_coeffs(const double* d19, double* c15);
void hwo2d_quad_coeffs(int n, const double* d19, double* c6);
double hwo2d_beta_of_coeffs(int degree, const double* c, double ratio);
void hwo_euler2d_flux(double g, const double* U, int dir, double* F);
void hwo_euler2d_eigen(double g, const double* U, int dir, double R[16], double L[16]);

/* ---------------- threads ---------------- */
/* OpenMP build (libhweno_oracle_omp.so): sets the thread count when n > 0 and
 * returns the count in use; the plain build returns 1. */
int hwo_set_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
