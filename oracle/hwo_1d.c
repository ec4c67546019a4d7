/*
 * ORACLE -- test infrastructure only (see hweno_oracle.h).
 *
 * One-dimensional new hybrid HWENO scheme with artificial linear weights,
 * Zhao & Qiu, arXiv:2002.08816, Sec. 2.1, taken step by step in FP64:
 *   semi-discrete moment scheme      Eq. (odeH), Sec. 2.1
 *   Lax-Friedrichs flux, 4-point Gauss-Lobatto cell integral   Sec. 2.1
 *   Step 1   KXRCF troubled cells, first-moment modification (limiter)
 *   Step 2.1 HWENO interface values on stencils with a troubled cell
 *   Step 2.2 linear interface values elsewhere
 *   Step 2.3 linear values at x_{i +- sqrt5/10}
 *   Step 3   third-order TVD (SSP) Runge-Kutta, Eq. (RK)
 *   Remarks 1-2: indicator variables and local characteristic fields.
 *
 * Every candidate polynomial is built here from the moment conditions the
 * paper states (a dense solve in the reference coordinate xi = (x-x_i)/dx);
 * its smoothness indicator is Eq. (GHYZ) integrated exactly.  Readings where
 * the paper is silent (the KXRCF formula, ghost cells, alpha and dt, the
 * eigen-system state, storing the limited moment) are marked "Reading:".
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "hweno_oracle.h"
#include "hwo_internal.h"

/* ---------------------------------------------------------------------- */
/* Candidate polynomials in xi; cell I_{i+j} is [j - 1/2, j + 1/2].        */
/* ---------------------------------------------------------------------- */

enum { AVG = 0, MOM = 1 };

typedef struct {
  int kind; /* AVG: (1/dx) int p dx;  MOM: (1/dx) int p (x - x_{i+j})/dx dx */
  int j;
} cond1d;

typedef struct {
  int n;            /* number of conditions = degree + 1 */
  double inv[36];   /* inverse of the condition-by-monomial matrix */
} fit1d;

static double cond_on_monomial(cond1d c, int k) {
  double a = c.j - 0.5, b = c.j + 0.5;
  if (c.kind == AVG) return hwo_mono_int(k, a, b);
  return hwo_mono_int(k + 1, a, b) - c.j * hwo_mono_int(k, a, b);
}

static void fit1d_init(fit1d* f, int n, const cond1d* conds) {
  double M[36];
  f->n = n;
  for (int r = 0; r < n; ++r)
    for (int k = 0; k < n; ++k) M[r * n + k] = cond_on_monomial(conds[r], k);
  if (hwo_mat_inverse(n, M, f->inv) != 0) abort();
}

static void fit1d_solve(const fit1d* f, const double* data, double* coef) {
  hwo_matvec(f->n, f->n, f->inv, data, coef);
}

static double poly_eval(int n, const double* c, double xi) {
  double s = 0.0;
  for (int k = n - 1; k >= 0; --k) s = s * xi + c[k];
  return s;
}

/* first moment over I_i of the polynomial */
static double poly_first_moment(int n, const double* c) {
  cond1d m0 = {MOM, 0};
  double s = 0.0;
  for (int k = 0; k < n; ++k) s += c[k] * cond_on_monomial(m0, k);
  return s;
}

/* CELL_MONO[k] = int_{-1/2}^{1/2} xi^k dxi: 1/((k+1) 2^k) for even k, 0 for odd */
static const double CELL_MONO[12] = {1.0, 0.0, 1.0 / 12.0, 0.0, 1.0 / 80.0, 0.0,
                                     1.0 / 448.0, 0.0, 1.0 / 2304.0, 0.0,
                                     1.0 / 11264.0, 0.0};

/* Eq. (GHYZ): beta = sum_{a=1}^{r} int_{I_i} dx^{2a-1} (d^a p/dx^a)^2 dx, which
 * in xi is sum_a int_{-1/2}^{1/2} (d^a p/dxi^a)^2 dxi. */
static double poly_beta(int n, const double* c) {
  double d[8], total = 0.0;
  int deg = n - 1;
  for (int k = 0; k < n; ++k) d[k] = c[k];
  for (int a = 1; a <= deg; ++a) {
    int m = n - a; /* coefficients left after a derivatives */
    for (int k = 0; k < m; ++k) d[k] = d[k + 1] * (double)(k + 1);
    for (int p = 0; p < m; ++p)
      for (int q = 0; q < m; ++q) total += d[p] * d[q] * CELL_MONO[p + q];
  }
  return total;
}

/* Step 1 stencils: quartic p0 on S0 = {I_{i-1}, I_i, I_{i+1}} matching three
 * averages and the first moments of I_{i-1}, I_{i+1}; linear p1, p2 on
 * S1 = {I_{i-1}, I_i}, S2 = {I_i, I_{i+1}} matching two averages. */
static fit1d LIM_P0, LIM_P1, LIM_P2;
/* Step 2.1 stencils: quintic p0 matching three averages and three first
 * moments; quadratics p1, p2 matching two averages and the first moment of I_i. */
static fit1d REC_P0, REC_P1, REC_P2;
static int fits_ready = 0;

static void init_fits(void) {
  if (fits_ready) return;
  const cond1d l0[5] = {{AVG, -1}, {AVG, 0}, {AVG, 1}, {MOM, -1}, {MOM, 1}};
  const cond1d l1[2] = {{AVG, -1}, {AVG, 0}};
  const cond1d l2[2] = {{AVG, 0}, {AVG, 1}};
  const cond1d r0[6] = {{AVG, -1}, {AVG, 0}, {AVG, 1}, {MOM, -1}, {MOM, 0}, {MOM, 1}};
  const cond1d r1[3] = {{AVG, -1}, {AVG, 0}, {MOM, 0}};
  const cond1d r2[3] = {{AVG, 0}, {AVG, 1}, {MOM, 0}};
  fit1d_init(&LIM_P0, 5, l0);
  fit1d_init(&LIM_P1, 2, l1);
  fit1d_init(&LIM_P2, 2, l2);
  fit1d_init(&REC_P0, 6, r0);
  fit1d_init(&REC_P1, 3, r1);
  fit1d_init(&REC_P2, 3, r2);
  fits_ready = 1;
}

/* tau of Eq. (tao5) */
static double tau1d(const double beta[3]) {
  double s = 0.5 * (fabs(beta[0] - beta[1]) + fabs(beta[0] - beta[2]));
  return s * s;
}

/* Step 1: q_n = first moment over I_i of p_n, and beta_n of p_n on I_i. */
void hwo1d_limiter_candidates(const double ub[3], double v_m1, double v_p1,
                              double q[3], double beta[3]) {
  init_fits();
  double d0[5] = {ub[0], ub[1], ub[2], v_m1, v_p1};
  double d1[2] = {ub[0], ub[1]};
  double d2[2] = {ub[1], ub[2]};
  double c0[6], c1[6], c2[6];
  fit1d_solve(&LIM_P0, d0, c0);
  fit1d_solve(&LIM_P1, d1, c1);
  fit1d_solve(&LIM_P2, d2, c2);
  q[0] = poly_first_moment(5, c0);
  q[1] = poly_first_moment(2, c1);
  q[2] = poly_first_moment(2, c2);
  beta[0] = poly_beta(5, c0);
  beta[1] = poly_beta(2, c1);
  beta[2] = poly_beta(2, c2);
}

/* Step 1, last formula: the modified first moment. */
double hwo1d_limit_scalar(const double gam[3], double eps, const double ub[3],
                          double v_m1, double v_p1) {
  double q[3], beta[3], omega[3];
  hwo1d_limiter_candidates(ub, v_m1, v_p1, q, beta);
  hwo_nonlinear_weights(3, gam, eps, beta, tau1d(beta), omega);
  return hwo_combine(3, gam, omega, q);
}

static const double XI_PTS[4] = {-0.5, 0.5, 0.0, 0.0}; /* +-sqrt5/10 filled below */

static void recon_points(double pts[4]) {
  pts[0] = XI_PTS[0];
  pts[1] = XI_PTS[1];
  pts[2] = -sqrt(5.0) / 10.0;
  pts[3] = sqrt(5.0) / 10.0;
}

/* Step 2.1 candidates: val[n*4 + p] = p_n at xi in {-1/2, +1/2, -sqrt5/10,
 * +sqrt5/10}; beta_n of p_n on I_i. */
void hwo1d_recon_candidates(const double ub[3], const double vb[3],
                            double val[12], double beta[3]) {
  init_fits();
  double d0[6] = {ub[0], ub[1], ub[2], vb[0], vb[1], vb[2]};
  double d1[3] = {ub[0], ub[1], vb[1]};
  double d2[3] = {ub[1], ub[2], vb[1]};
  double c0[6], c1[6], c2[6], pts[4];
  recon_points(pts);
  fit1d_solve(&REC_P0, d0, c0);
  fit1d_solve(&REC_P1, d1, c1);
  fit1d_solve(&REC_P2, d2, c2);
  for (int p = 0; p < 4; ++p) {
    val[0 * 4 + p] = poly_eval(6, c0, pts[p]);
    val[1 * 4 + p] = poly_eval(3, c1, pts[p]);
    val[2 * 4 + p] = poly_eval(3, c2, pts[p]);
  }
  beta[0] = poly_beta(6, c0);
  beta[1] = poly_beta(3, c1);
  beta[2] = poly_beta(3, c2);
}

/* out = (u^+_{i-1/2}, u^-_{i+1/2}, u_{i-sqrt5/10}, u_{i+sqrt5/10}).
 * hweno = 0: Steps 2.2-2.3 (p0 everywhere).  hweno = 1: Step 2.1 at the two
 * interface points (one set of nonlinear weights for both: the candidates and
 * their beta are the same polynomials on I_i), Step 2.3 inside. */
void hwo1d_recon_scalar(const double gam[3], double eps, const double ub[3],
                        const double vb[3], int hweno, double out[4]) {
  double val[12], beta[3], omega[3];
  if (!hweno) {
    double d0[6] = {ub[0], ub[1], ub[2], vb[0], vb[1], vb[2]};
    double c0[6], pts[4];
    init_fits();
    recon_points(pts);
    fit1d_solve(&REC_P0, d0, c0);
    for (int p = 0; p < 4; ++p) out[p] = poly_eval(6, c0, pts[p]);
    return;
  }
  hwo1d_recon_candidates(ub, vb, val, beta);
  for (int p = 0; p < 4; ++p) out[p] = val[p];
  hwo_nonlinear_weights(3, gam, eps, beta, tau1d(beta), omega);
  for (int p = 0; p < 2; ++p) {
    double v[3] = {val[0 * 4 + p], val[1 * 4 + p], val[2 * 4 + p]};
    out[p] = hwo_combine(3, gam, omega, v);
  }
}

/* ---------------------------------------------------------------------- */
/* Physics: Burgers f = u^2/2; Euler Eq. (euler1).                         */
/* ---------------------------------------------------------------------- */

void hwo_euler1d_flux(double g, const double U[3], double F[3]) {
  double rho = U[0], mu = U[1] / U[0], E = U[2];
  double p = (g - 1.0) * (E - 0.5 * rho * mu * mu);
  F[0] = rho * mu;
  F[1] = rho * mu * mu + p;
  F[2] = mu * (E + p);
}

/* Right eigenvectors of the flux Jacobian at U (columns: mu-c, mu, mu+c);
 * the left eigenvectors are obtained by inverting R numerically. */
void hwo_euler1d_eigen(double g, const double U[3], double R[9], double L[9]) {
  double rho = U[0], mu = U[1] / U[0], E = U[2];
  double p = (g - 1.0) * (E - 0.5 * rho * mu * mu);
  double c = sqrt(g * p / rho), H = (E + p) / rho;
  double cols[3][3] = {{1.0, mu - c, H - mu * c}, {1.0, mu, 0.5 * mu * mu},
                       {1.0, mu + c, H + mu * c}};
  for (int r = 0; r < 3; ++r)
    for (int k = 0; k < 3; ++k) R[r * 3 + k] = cols[k][r];
  if (hwo_mat_inverse(3, R, L) != 0)
    for (int k = 0; k < 9; ++k) L[k] = NAN;
}

int hwo1d_ncomp(int system) { return system == HWO_EULER ? 3 : 1; }

static void phys_flux(const hwo1d_cfg* cfg, const double* U, double* F) {
  if (cfg->system == HWO_EULER)
    hwo_euler1d_flux(cfg->gas_gamma, U, F);
  else
    F[0] = 0.5 * U[0] * U[0];
}

/* max |f'(u)| at one state: |u| (Burgers), |mu| + c (Euler) */
static double wave_speed(const hwo1d_cfg* cfg, const double* U) {
  if (cfg->system != HWO_EULER) return fabs(U[0]);
  double g = cfg->gas_gamma, rho = U[0], mu = U[1] / U[0];
  double p = (g - 1.0) * (U[2] - 0.5 * rho * mu * mu);
  if (!(rho > 0.0) || !(p > 0.0)) return NAN;
  return fabs(mu) + sqrt(g * p / rho);
}

/* Reading: alpha = max over the cell averages of the stage input. */
double hwo1d_alpha(const hwo1d_cfg* cfg, const double* u) {
  int C = hwo1d_ncomp(cfg->system), N = cfg->nx;
  double a = 0.0;
  for (int i = 0; i < N; ++i) {
    double U[3];
    for (int c = 0; c < C; ++c) U[c] = u[(c * 2 + 0) * N + i];
    double s = wave_speed(cfg, U);
    if (!(s == s)) return NAN;
    if (s > a) a = s;
  }
  return a;
}

/* ---------------------------------------------------------------------- */
/* One evaluation of the right-hand side of Eq. (odeH).                    */
/* ---------------------------------------------------------------------- */

#define G1 3 /* ghost cells per side: the stencil of one stage reaches 3 cells */

/* Reading: periodic ghosts wrap; outflow ghosts copy the boundary cell's
 * average and first moment; reflective ghosts (1D Euler) are the mirror images
 * of the interior cells (*mirror = 1). */
static int ghost_src(const hwo1d_cfg* cfg, int i, int* mirror) {
  int N = cfg->nx;
  *mirror = 0;
  if (cfg->bc == HWO_BC_PERIODIC) return ((i % N) + N) % N;
  if (cfg->bc == HWO_BC_REFLECTIVE && (i < 0 || i >= N)) {
    *mirror = 1;
    return i < 0 ? -1 - i : 2 * N - 1 - i;
  }
  return i < 0 ? 0 : (i >= N ? N - 1 : i);
}

/* Sign of a mirrored ghost's moment: q(x) -> s q(2 x_w - x) keeps the average
 * times s and the first moment times -s; s = -1 for the momentum, +1 for the
 * density and the energy. */
static double mirror_sign(int c, int m) {
  double s = c == 1 ? -1.0 : 1.0;
  return m == 0 ? s : -s;
}

/* Reading of the KXRCF indicator (Krivodonova et al., with the degree-1 cell
 * polynomial u_i(x) = ubar_i + 12 vbar_i (x - x_i)/dx, k = 1, h = dx/2):
 *   I_i = |u_i - u_nb| at the inflow face / (h * max(|ubar_i|, 1e-12)).
 * The inflow face is the left one when the velocity is >= 0, else the right. */
static double kxrcf1d(const double* ub, const double* vb, int e, double vel,
                      double h) {
  double jump;
  if (vel >= 0.0)
    jump = (ub[e] - 6.0 * vb[e]) - (ub[e - 1] + 6.0 * vb[e - 1]);
  else
    jump = (ub[e] + 6.0 * vb[e]) - (ub[e + 1] - 6.0 * vb[e + 1]);
  double nrm = fabs(ub[e]);
  if (nrm < 1e-12) nrm = 1e-12;
  return fabs(jump) / (h * nrm);
}

int hwo1d_rhs(const hwo1d_cfg* cfg, const double* u, double alpha, double* rhs,
              double* ulim, unsigned char* flags, double* indicator) {
  return hwo1d_rhs_ex(cfg, u, alpha, rhs, ulim, flags, indicator, NULL);
}

/* Step 2.1 for the Euler cell at extended index e in the characteristic fields
 * of the x-Jacobian at the state U: the interface values at x_{e-1/2} (pm) and
 * x_{e+1/2} (pp). */
static void char_faces1d(const hwo1d_cfg* cfg, const double* ub, const double* vl, int NE,
                         int e, const double U[3], double pm[3], double pp[3]) {
  double R[9], L[9];
  hwo_euler1d_eigen(cfg->gas_gamma, U, R, L);
  double Wu[3][3], Wv[3][3]; /* [field][cell] */
  for (int k = 0; k < 3; ++k) {
    double su[3], sv[3], wu[3], wv[3];
    for (int c = 0; c < 3; ++c) {
      su[c] = ub[c * NE + e - 1 + k];
      sv[c] = vl[c * NE + e - 1 + k];
    }
    hwo_matvec(3, 3, L, su, wu);
    hwo_matvec(3, 3, L, sv, wv);
    for (int f = 0; f < 3; ++f) {
      Wu[f][k] = wu[f];
      Wv[f][k] = wv[f];
    }
  }
  double cm[3], cp[3];
  for (int f = 0; f < 3; ++f) {
    double out[4];
    hwo1d_recon_scalar(cfg->lin_w, cfg->eps, Wu[f], Wv[f], 1, out);
    cm[f] = out[0];
    cp[f] = out[1];
  }
  hwo_matvec(3, 3, R, cm, pm);
  hwo_matvec(3, 3, R, cp, pp);
}

/* As hwo1d_rhs; faces (nullable, [C][2][nx]) receives u^+_{i-1/2}, u^-_{i+1/2}. */
int hwo1d_rhs_ex(const hwo1d_cfg* cfg, const double* u, double alpha, double* rhs,
                 double* ulim, unsigned char* flags, double* indicator,
                 double* faces) {
  const int N = cfg->nx, C = hwo1d_ncomp(cfg->system), NE = N + 2 * G1;
  const double dx = (cfg->x1 - cfg->x0) / N;
  const int euler = cfg->system == HWO_EULER;
  if (N < 3) return -1;
  if (cfg->bc == HWO_BC_REFLECTIVE && !euler) return -1;
  init_fits();
  if (alpha < 0.0) alpha = hwo1d_alpha(cfg, u);
  if (!(alpha == alpha)) return -2;

  double* ub = (double*)malloc(sizeof(double) * C * NE);
  double* vb = (double*)malloc(sizeof(double) * C * NE);
  double* vl = (double*)malloc(sizeof(double) * C * NE);
  double* ind = (double*)malloc(sizeof(double) * NE);
  unsigned char* fl = (unsigned char*)calloc(NE, 1);
  double* fm = (double*)malloc(sizeof(double) * C * NE); /* u^+_{i-1/2} */
  double* fp = (double*)malloc(sizeof(double) * C * NE); /* u^-_{i+1/2} */
  double* gm = (double*)malloc(sizeof(double) * C * NE); /* u_{i-sqrt5/10} */
  double* gp = (double*)malloc(sizeof(double) * C * NE); /* u_{i+sqrt5/10} */
  double* fh = (double*)malloc(sizeof(double) * C * NE); /* flux at e+1/2 */
  int status = 0;

  for (int e = 0; e < NE; ++e) {
    int mir;
    int s = ghost_src(cfg, e - G1, &mir);
    for (int c = 0; c < C; ++c) {
      ub[c * NE + e] = u[(c * 2 + 0) * N + s] * (mir ? mirror_sign(c, 0) : 1.0);
      vb[c * NE + e] = u[(c * 2 + 1) * N + s] * (mir ? mirror_sign(c, 1) : 1.0);
    }
  }

  /* Step 1, troubled cells (Remark 1: u for Burgers with velocity f'(u);
   * rho and E for Euler with the velocity mu). */
  for (int e = 0; e < NE; ++e) ind[e] = 0.0;
#pragma omp parallel for schedule(static)
  for (int e = 1; e < NE - 1; ++e) {
    double I;
    if (euler) {
      double vel = ub[1 * NE + e] / ub[0 * NE + e];
      double Ir = kxrcf1d(ub + 0 * NE, vb + 0 * NE, e, vel, 0.5 * dx);
      double Ie = kxrcf1d(ub + 2 * NE, vb + 2 * NE, e, vel, 0.5 * dx);
      I = Ir > Ie ? Ir : Ie;
    } else {
      I = kxrcf1d(ub, vb, e, ub[e], 0.5 * dx);
    }
    ind[e] = I;
    if (cfg->troubled_mode == HWO_TROUBLED_ALL)
      fl[e] = 1;
    else if (cfg->troubled_mode == HWO_TROUBLED_NONE)
      fl[e] = 0;
    else
      fl[e] = I > cfg->kxrcf_threshold;
  }

  /* Step 1, modify the first moment of troubled cells (Remark 2: in the local
   * characteristic fields for Euler; Reading: eigen-system at the cell's own
   * average).  All cells are modified from the unmodified moments. */
  memcpy(vl, vb, sizeof(double) * C * NE);
#pragma omp parallel for schedule(static)
  for (int e = 1; e < NE - 1; ++e) {
    if (!fl[e]) continue;
    if (!euler) {
      double u3[3] = {ub[e - 1], ub[e], ub[e + 1]};
      vl[e] = hwo1d_limit_scalar(cfg->lin_w, cfg->eps, u3, vb[e - 1], vb[e + 1]);
    } else {
      double R[9], L[9], U[3], W[3][5], q[3];
      for (int c = 0; c < 3; ++c) U[c] = ub[c * NE + e];
      hwo_euler1d_eigen(cfg->gas_gamma, U, R, L);
      /* project u_{i-1}, u_i, u_{i+1}, v_{i-1}, v_{i+1} */
      double src[5][3];
      for (int c = 0; c < 3; ++c) {
        src[0][c] = ub[c * NE + e - 1];
        src[1][c] = ub[c * NE + e];
        src[2][c] = ub[c * NE + e + 1];
        src[3][c] = vb[c * NE + e - 1];
        src[4][c] = vb[c * NE + e + 1];
      }
      for (int k = 0; k < 5; ++k) {
        double w[3];
        hwo_matvec(3, 3, L, src[k], w);
        for (int f = 0; f < 3; ++f) W[f][k] = w[f];
      }
      for (int f = 0; f < 3; ++f)
        q[f] = hwo1d_limit_scalar(cfg->lin_w, cfg->eps, W[f], W[f][3], W[f][4]);
      double v[3];
      hwo_matvec(3, 3, R, q, v);
      for (int c = 0; c < 3; ++c) vl[c * NE + e] = v[c];
    }
  }

  /* Step 2: point values for cells -1..N (extended index 2..NE-3). */
#pragma omp parallel for schedule(static)
  for (int e = 2; e < NE - 2; ++e) {
    int hw = fl[e - 1] | fl[e] | fl[e + 1];
    if (!euler || !hw) {
      for (int c = 0; c < C; ++c) {
        double u3[3] = {ub[c * NE + e - 1], ub[c * NE + e], ub[c * NE + e + 1]};
        double v3[3] = {vl[c * NE + e - 1], vl[c * NE + e], vl[c * NE + e + 1]};
        double out[4];
        hwo1d_recon_scalar(cfg->lin_w, cfg->eps, u3, v3, hw, out);
        fm[c * NE + e] = out[0];
        fp[c * NE + e] = out[1];
        gm[c * NE + e] = out[2];
        gp[c * NE + e] = out[3];
      }
    } else {
      /* Step 2.1 in characteristic fields for the interface values (of the
       * cell average, or with char_state of the mean state at each interface);
       * Step 2.3 component by component for the interior values. */
      double pm[3], pp[3], tmp[3];
      if (!cfg->char_state) {
        double U[3];
        for (int c = 0; c < 3; ++c) U[c] = ub[c * NE + e];
        char_faces1d(cfg, ub, vl, NE, e, U, pm, pp);
      } else {
        double Um[3], Up[3];
        for (int c = 0; c < 3; ++c) {
          Um[c] = 0.5 * (ub[c * NE + e - 1] + ub[c * NE + e]);
          Up[c] = 0.5 * (ub[c * NE + e] + ub[c * NE + e + 1]);
        }
        char_faces1d(cfg, ub, vl, NE, e, Um, pm, tmp);
        char_faces1d(cfg, ub, vl, NE, e, Up, tmp, pp);
      }
      for (int c = 0; c < 3; ++c) {
        double u3[3] = {ub[c * NE + e - 1], ub[c * NE + e], ub[c * NE + e + 1]};
        double v3[3] = {vl[c * NE + e - 1], vl[c * NE + e], vl[c * NE + e + 1]};
        double out[4];
        hwo1d_recon_scalar(cfg->lin_w, cfg->eps, u3, v3, 0, out);
        fm[c * NE + e] = pm[c];
        fp[c * NE + e] = pp[c];
        gm[c * NE + e] = out[2];
        gp[c * NE + e] = out[3];
      }
    }
  }

  /* Lax-Friedrichs flux at x_{e+1/2} from u^- (cell e) and u^+ (cell e+1). */
#pragma omp parallel for schedule(static)
  for (int e = G1 - 1; e < G1 + N; ++e) {
    double a[3], b[3], fa[3], fb[3];
    for (int c = 0; c < C; ++c) {
      a[c] = fp[c * NE + e];
      b[c] = fm[c * NE + e + 1];
    }
    phys_flux(cfg, a, fa);
    phys_flux(cfg, b, fb);
    for (int c = 0; c < C; ++c)
      fh[c * NE + e] = 0.5 * (fa[c] + fb[c]) - 0.5 * alpha * (b[c] - a[c]);
  }

  /* Eq. (odeH) with F_i by the 4-point Gauss-Lobatto rule. */
#pragma omp parallel for schedule(static) reduction(min : status)
  for (int i = 0; i < N; ++i) {
    int e = i + G1;
    double pts[4][3], fq[4][3];
    for (int c = 0; c < C; ++c) {
      pts[0][c] = fm[c * NE + e];
      pts[1][c] = gm[c * NE + e];
      pts[2][c] = gp[c * NE + e];
      pts[3][c] = fp[c * NE + e];
    }
    for (int l = 0; l < 4; ++l) phys_flux(cfg, pts[l], fq[l]);
    for (int c = 0; c < C; ++c) {
      double F = (1.0 / 12.0) * fq[0][c] + (5.0 / 12.0) * fq[1][c] +
                 (5.0 / 12.0) * fq[2][c] + (1.0 / 12.0) * fq[3][c];
      double fl_ = fh[c * NE + e - 1], fr_ = fh[c * NE + e];
      rhs[(c * 2 + 0) * N + i] = -(fr_ - fl_) / dx;
      rhs[(c * 2 + 1) * N + i] = -(fl_ + fr_) / (2.0 * dx) + F / dx;
      if (!(rhs[(c * 2 + 0) * N + i] == rhs[(c * 2 + 0) * N + i]) ||
          !(rhs[(c * 2 + 1) * N + i] == rhs[(c * 2 + 1) * N + i]))
        status = -3;
    }
    if (ulim)
      for (int c = 0; c < C; ++c) {
        ulim[(c * 2 + 0) * N + i] = ub[c * NE + e];
        ulim[(c * 2 + 1) * N + i] = vl[c * NE + e];
      }
    if (faces)
      for (int c = 0; c < C; ++c) {
        faces[(c * 2 + 0) * N + i] = fm[c * NE + e];
        faces[(c * 2 + 1) * N + i] = fp[c * NE + e];
      }
    if (flags) flags[i] = fl[e];
    if (indicator) indicator[i] = ind[e];
  }

  free(ub); free(vb); free(vl); free(ind); free(fl);
  free(fm); free(fp); free(gm); free(gp); free(fh);
  return status;
}

/* ---------------------------------------------------------------------- */
/* Step 3: third-order TVD Runge-Kutta, Eq. (RK).                          */
/* ---------------------------------------------------------------------- */

/* Reading: dt = CFL dx / alpha(u^n), clipped to the final time; dt = 0 once
 * t >= t_final (t_final <= 0: no clipping). */
double hwo1d_dt(const hwo1d_cfg* cfg, const double* u, double cfl, double t,
                double t_final) {
  double dx = (cfg->x1 - cfg->x0) / cfg->nx;
  double dt = cfl * dx / hwo1d_alpha(cfg, u);
  if (t_final > 0.0) {
    double rem = t_final - t;
    if (rem <= 0.0) return 0.0;
    if (dt > rem) dt = rem;
  }
  return dt;
}

/* Reading: alpha of each stage from that stage's input; with limit_in_place
 * the convex combinations use the stage inputs with their limited moments. */
int hwo1d_step(const hwo1d_cfg* cfg, double* u, double dt, long* n_troubled) {
  const int C = hwo1d_ncomp(cfg->system), N = cfg->nx;
  const size_t S = (size_t)C * 2 * N;
  if (!(dt > 0.0)) return 0;
  double* L = (double*)malloc(sizeof(double) * S);
  double* b0 = (double*)malloc(sizeof(double) * S);
  double* bk = (double*)malloc(sizeof(double) * S);
  double* uk = (double*)malloc(sizeof(double) * S);
  unsigned char* fl = (unsigned char*)malloc(N);
  int st = 0;
  long nt = 0;

  /* u1 = u^n + dt L(u^n) */
  st = hwo1d_rhs(cfg, u, -1.0, L, b0, fl, NULL);
  for (int i = 0; i < N; ++i) nt += fl[i];
  if (!cfg->limit_in_place) memcpy(b0, u, sizeof(double) * S);
  for (size_t k = 0; k < S && !st; ++k) uk[k] = b0[k] + dt * L[k];
  /* u2 = 3/4 u^n + 1/4 u1 + 1/4 dt L(u1) */
  if (!st) st = hwo1d_rhs(cfg, uk, -1.0, L, bk, fl, NULL);
  for (int i = 0; i < N && !st; ++i) nt += fl[i];
  if (!cfg->limit_in_place) memcpy(bk, uk, sizeof(double) * S);
  for (size_t k = 0; k < S && !st; ++k)
    uk[k] = 0.75 * b0[k] + 0.25 * bk[k] + 0.25 * dt * L[k];
  /* u^{n+1} = 1/3 u^n + 2/3 u2 + 2/3 dt L(u2) */
  if (!st) st = hwo1d_rhs(cfg, uk, -1.0, L, bk, fl, NULL);
  for (int i = 0; i < N && !st; ++i) nt += fl[i];
  if (!cfg->limit_in_place) memcpy(bk, uk, sizeof(double) * S);
  for (size_t k = 0; k < S && !st; ++k)
    u[k] = (1.0 / 3.0) * b0[k] + (2.0 / 3.0) * bk[k] + (2.0 / 3.0) * dt * L[k];

  if (n_troubled) *n_troubled += nt;
  free(L); free(b0); free(bk); free(uk); free(fl);
  return st;
}

/* Reading of the final step: a step clipped to t_final (dt >= t_final - t)
 * is the last one and ends exactly at t_final.  Without it, rounding of t
 * can leave a remainder of a few ulps and one more, vanishing, step, which
 * would still modify the first moments of troubled cells once more. */
int hwo1d_run(const hwo1d_cfg* cfg, double* u, int nsteps, double cfl,
              double t0, double t_final, double dt_fixed,
              const double* lin_w_per_step, double* t_out, long* n_troubled) {
  const double dx = (cfg->x1 - cfg->x0) / cfg->nx;
  double t = t0;
  int st = 0;
  hwo1d_cfg c = *cfg;
  for (int s = 0; nsteps < 0 || s < nsteps; ++s) {
    double dt = dt_fixed > 0.0 ? dt_fixed : cfl * dx / hwo1d_alpha(&c, u);
    int last = 0;
    if (t_final > 0.0) {
      double rem = t_final - t;
      if (rem <= 0.0) break;
      if (dt >= rem) {
        dt = rem;
        last = 1;
      }
    }
    if (!(dt > 0.0)) break;
    if (lin_w_per_step)
      for (int k = 0; k < 3; ++k) c.lin_w[k] = lin_w_per_step[3 * s + k];
    st = hwo1d_step(&c, u, dt, n_troubled);
    if (st) break;
    t = last ? t_final : t + dt;
    if (last) break;
  }
  if (t_out) *t_out = t;
  return st;
}
