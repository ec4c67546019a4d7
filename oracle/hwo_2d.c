/*
 * ORACLE -- test infrastructure only (see hweno_oracle.h).
 *
 * Two-dimensional new hybrid HWENO scheme with artificial linear weights,
 * Zhao & Qiu, arXiv:2002.08816, Sec. 2.2, taken step by step in FP64:
 *   semi-discrete moment scheme      Eq. (ode2) with Gauss quadratures
 *   Lax-Friedrichs fluxes in x and y  Sec. 2.2
 *   Step 4   KXRCF troubled cells; first moments modified dimension by
 *            dimension with the 1D Step 1 formula
 *   Step 5.1 HWENO values at the interface Gauss points: quartic p0 on the
 *            3x3 stencil (nine averages and the centre's first moments
 *            exactly, the other first moments of cells 2, 4, 6, 8 in least
 *            squares), four quadratics on the 2x2 stencils, Hu-Shu
 *            smoothness indicators Eq. (2dGHYZ), tau Eq. (tao4), weights (99)
 *   Steps 5.2, 5.3  linear p0 at interface and interior Gauss points
 *   Step 6   third-order TVD Runge-Kutta, Eq. (RK)
 *   Remarks 3-4: indicator variables, local characteristic fields.
 *
 * Cells of the 3x3 stencil are numbered as in the paper's Fig. 1:
 * 1 = (i-1,j-1), 2 = (i,j-1), 3 = (i+1,j-1), 4 = (i-1,j), 5 = (i,j), ...,
 * 9 = (i+1,j+1).  Every candidate polynomial is derived here from its moment
 * conditions (the constrained least-squares p0 by its KKT system) in the
 * reference coordinates xi = (x-x_i)/dx, eta = (y-y_j)/dy.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "hweno_oracle.h"
#include "hwo_internal.h"

/* implemented in hwo_1d.c: the 1D Step 1 formula and the 1D Euler pieces */
double hwo1d_limit_scalar(const double gam[3], double eps, const double ub[3],
                          double v_m1, double v_p1);

/* ---------------------------------------------------------------------- */
/* Bivariate polynomials: monomials xi^a eta^b with a + b <= 4, ordered by  */
/* total degree, then by descending a (1, xi, eta, xi^2, xi eta, eta^2,...) */
/* ---------------------------------------------------------------------- */

#define NM4 15
#define NM2 6
static int MON_A[NM4], MON_B[NM4];
static int mono_ready = 0;

static void init_mono(void) {
  if (mono_ready) return;
  int k = 0;
  for (int d = 0; d <= 4; ++d)
    for (int a = d; a >= 0; --a) {
      MON_A[k] = a;
      MON_B[k] = d - a;
      ++k;
    }
  mono_ready = 1;
}

static const int CELL_DI[10] = {0, -1, 0, 1, -1, 0, 1, -1, 0, 1};
static const int CELL_DJ[10] = {0, -1, -1, -1, 0, 0, 0, 1, 1, 1};

enum { AVG = 0, XM = 1, YM = 2 };

/* one moment condition of cell (di, dj) applied to xi^a eta^b */
static double cond2d(int kind, int di, int dj, int a, int b) {
  double ax = hwo_mono_int(a, di - 0.5, di + 0.5);
  double ay = hwo_mono_int(b, dj - 0.5, dj + 0.5);
  if (kind == AVG) return ax * ay;
  if (kind == XM) return (hwo_mono_int(a + 1, di - 0.5, di + 0.5) - di * ax) * ay;
  return ax * (hwo_mono_int(b + 1, dj - 0.5, dj + 0.5) - dj * ay);
}

/* The 19 data of a stencil, in this order: ubar of cells 1..9; vbar of cells
 * 2, 4, 5, 6, 8; wbar of cells 2, 4, 5, 6, 8. */
#define ND 19
static const int MOM_CELLS[5] = {2, 4, 5, 6, 8};

/* p0: 15 coefficients = M0 (15 x 19) * data; p1..p4: 6 = Mq[n] (6 x 19) * data */
static double M0[NM4 * ND];
static double MQ[4][NM2 * ND];
static int maps_ready = 0;

/* data index of (kind, cell) */
static int data_index(int kind, int cell) {
  if (kind == AVG) return cell - 1;
  for (int k = 0; k < 5; ++k)
    if (MOM_CELLS[k] == cell) return 9 + (kind == XM ? 0 : 5) + k;
  abort();
}

static void init_maps(void) {
  if (maps_ready) return;
  init_mono();
  /* p0: exact rows (11) and least-squares rows (8) */
  int eq_kind[11], eq_cell[11], ls_kind[8], ls_cell[8], ne = 0, nl = 0;
  for (int c = 1; c <= 9; ++c) {
    eq_kind[ne] = AVG;
    eq_cell[ne++] = c;
  }
  eq_kind[ne] = XM; eq_cell[ne++] = 5;
  eq_kind[ne] = YM; eq_cell[ne++] = 5;
  const int ls_c[4] = {2, 4, 6, 8};
  for (int k = 0; k < 4; ++k) { ls_kind[nl] = XM; ls_cell[nl++] = ls_c[k]; }
  for (int k = 0; k < 4; ++k) { ls_kind[nl] = YM; ls_cell[nl++] = ls_c[k]; }
  double E[11 * NM4], A[8 * NM4];
  for (int r = 0; r < 11; ++r)
    for (int k = 0; k < NM4; ++k)
      E[r * NM4 + k] = cond2d(eq_kind[r], CELL_DI[eq_cell[r]], CELL_DJ[eq_cell[r]], MON_A[k], MON_B[k]);
  for (int r = 0; r < 8; ++r)
    for (int k = 0; k < NM4; ++k)
      A[r * NM4 + k] = cond2d(ls_kind[r], CELL_DI[ls_cell[r]], CELL_DJ[ls_cell[r]], MON_A[k], MON_B[k]);
  /* KKT: [A^T A  E^T; E 0] [c; lambda] = [A^T d_ls; d_eq] */
  const int NK = NM4 + 11;
  double K[26 * 26], Ki[26 * 26];
  memset(K, 0, sizeof(K));
  for (int p = 0; p < NM4; ++p)
    for (int q = 0; q < NM4; ++q) {
      double s = 0.0;
      for (int r = 0; r < 8; ++r) s += A[r * NM4 + p] * A[r * NM4 + q];
      K[p * NK + q] = s;
    }
  for (int r = 0; r < 11; ++r)
    for (int k = 0; k < NM4; ++k) {
      K[(NM4 + r) * NK + k] = E[r * NM4 + k];
      K[k * NK + NM4 + r] = E[r * NM4 + k];
    }
  if (hwo_mat_inverse(NK, K, Ki) != 0) abort();
  /* c = Ki[0:15, 0:15] A^T d_ls + Ki[0:15, 15:26] d_eq */
  memset(M0, 0, sizeof(M0));
  for (int p = 0; p < NM4; ++p) {
    for (int r = 0; r < 8; ++r) {
      double s = 0.0;
      for (int q = 0; q < NM4; ++q) s += Ki[p * NK + q] * A[r * NM4 + q];
      M0[p * ND + data_index(ls_kind[r], ls_cell[r])] += s;
    }
    for (int r = 0; r < 11; ++r)
      M0[p * ND + data_index(eq_kind[r], eq_cell[r])] += Ki[p * NK + NM4 + r];
  }
  /* quadratics on S1 = {1,2,4,5}, S2 = {2,3,5,6}, S3 = {4,5,7,8}, S4 = {5,6,8,9} */
  const int sc[4][4] = {{1, 2, 4, 5}, {2, 3, 5, 6}, {4, 5, 7, 8}, {5, 6, 8, 9}};
  for (int n = 0; n < 4; ++n) {
    int kind[6], cell[6];
    for (int k = 0; k < 4; ++k) { kind[k] = AVG; cell[k] = sc[n][k]; }
    kind[4] = XM; cell[4] = 5;
    kind[5] = YM; cell[5] = 5;
    double Q[36], Qi[36];
    for (int r = 0; r < 6; ++r)
      for (int k = 0; k < NM2; ++k)
        Q[r * 6 + k] = cond2d(kind[r], CELL_DI[cell[r]], CELL_DJ[cell[r]], MON_A[k], MON_B[k]);
    if (hwo_mat_inverse(6, Q, Qi) != 0) abort();
    memset(MQ[n], 0, sizeof(MQ[n]));
    for (int p = 0; p < NM2; ++p)
      for (int r = 0; r < 6; ++r) MQ[n][p * ND + data_index(kind[r], cell[r])] += Qi[p * 6 + r];
  }
  maps_ready = 1;
}

/* Eq. (2dGHYZ): beta = sum over l = (l1, l2), 1 <= l1 + l2 <= r, of
 * |I|^{|l|-1} int_I (d^{|l|} p / dx^{l1} dy^{l2})^2 dx dy.  In the reference
 * coordinates the term of l carries (dy/dx)^{l1 - l2}; as a quadratic form in
 * the coefficients, beta = c^T B c with B built here once from that sum. */
static void beta_gram(int nm, int r, double ratio, double* B) {
  for (int p = 0; p < nm * nm; ++p) B[p] = 0.0;
  for (int l1 = 0; l1 <= r; ++l1)
    for (int l2 = 0; l1 + l2 <= r; ++l2) {
      if (l1 + l2 == 0) continue;
      double wl = pow(ratio, l1 - l2);
      for (int p = 0; p < nm; ++p)
        for (int q = 0; q < nm; ++q) {
          int ap = MON_A[p], bp = MON_B[p], aq = MON_A[q], bq = MON_B[q];
          if (ap < l1 || bp < l2 || aq < l1 || bq < l2) continue;
          double fp = 1.0, fq = 1.0;
          for (int t = 0; t < l1; ++t) { fp *= (ap - t); fq *= (aq - t); }
          for (int t = 0; t < l2; ++t) { fp *= (bp - t); fq *= (bq - t); }
          B[p * nm + q] += wl * fp * fq *
                           hwo_mono_int(ap + aq - 2 * l1, -0.5, 0.5) *
                           hwo_mono_int(bp + bq - 2 * l2, -0.5, 0.5);
        }
    }
}

static double quad_form(int nm, const double* B, const double* c) {
  double s = 0.0;
  for (int p = 0; p < nm; ++p)
    for (int q = 0; q < nm; ++q) s += c[p] * B[p * nm + q] * c[q];
  return s;
}

static void gauss_points(int ng, double* x, double* w) {
  if (ng == 2) {
    x[0] = -sqrt(3.0) / 6.0; x[1] = sqrt(3.0) / 6.0;
    w[0] = w[1] = 0.5;
  } else {
    x[0] = -sqrt(15.0) / 10.0; x[1] = 0.0; x[2] = sqrt(15.0) / 10.0;
    w[0] = w[2] = 5.0 / 18.0; w[1] = 4.0 / 9.0;
  }
}

/* Reconstruction points of a cell, in this order: the left face xi = -1/2 at
 * eta_k, the right face xi = +1/2 at eta_k, the bottom face eta = -1/2 at
 * xi_k, the top face eta = +1/2 at xi_k, then the interior (xi_k, eta_l)
 * with k fastest.  PV[ng][p][m] = monomial m at point p. */
#define NPMAX 21
static double PV[4][NPMAX][NM4];
static double W0[4][NPMAX][ND];   /* p0 at the points as a map of the 19 data */
static int tables_ready[4] = {0, 0, 0, 0};

static int npoints(int ng) { return 4 * ng + ng * ng; }

static void init_tables(int ng) {
  init_maps();
  if (tables_ready[ng]) return;
  double gx[3], gw[3];
  gauss_points(ng, gx, gw);
  double px[NPMAX], py[NPMAX];
  int p = 0;
  for (int k = 0; k < ng; ++k) { px[p] = -0.5; py[p++] = gx[k]; }
  for (int k = 0; k < ng; ++k) { px[p] = 0.5; py[p++] = gx[k]; }
  for (int k = 0; k < ng; ++k) { px[p] = gx[k]; py[p++] = -0.5; }
  for (int k = 0; k < ng; ++k) { px[p] = gx[k]; py[p++] = 0.5; }
  for (int l = 0; l < ng; ++l)
    for (int k = 0; k < ng; ++k) { px[p] = gx[k]; py[p++] = gx[l]; }
  for (int q = 0; q < p; ++q)
    for (int m = 0; m < NM4; ++m) PV[ng][q][m] = pow(px[q], MON_A[m]) * pow(py[q], MON_B[m]);
  for (int q = 0; q < p; ++q)
    for (int d = 0; d < ND; ++d) {
      double s = 0.0;
      for (int m = 0; m < NM4; ++m) s += PV[ng][q][m] * M0[m * ND + d];
      W0[ng][q][d] = s;
    }
  tables_ready[ng] = 1;
}

static void gather19(const double ub[9], const double vb[9], const double wb[9], double* d) {
  for (int k = 0; k < 9; ++k) d[k] = ub[k];
  for (int k = 0; k < 5; ++k) {
    d[9 + k] = vb[MOM_CELLS[k] - 1];
    d[14 + k] = wb[MOM_CELLS[k] - 1];
  }
}

/* All five candidates at the points (val[n*np + p]) and their smoothness
 * indicators (B4, B2: the Gram matrices of beta_gram for the cell's aspect
 * ratio). */
static void candidates(const double* d, int ng, const double* B4, const double* B2,
                       double* val, double beta[5]) {
  init_tables(ng);
  const int np = npoints(ng);
  for (int n = 0; n < 5; ++n) {
    double c[NM4];
    int nm = n == 0 ? NM4 : NM2;
    hwo_matvec(nm, ND, n == 0 ? M0 : MQ[n - 1], d, c);
    for (int q = 0; q < np; ++q) {
      double s = 0.0;
      for (int m = 0; m < nm; ++m) s += PV[ng][q][m] * c[m];
      val[n * np + q] = s;
    }
    beta[n] = quad_form(nm, n == 0 ? B4 : B2, c);
  }
}

int hwo2d_recon_candidates(const double ub[9], const double vb[9], const double wb[9],
                           int n_gauss, double* val, double beta[5]) {
  double d[ND], B4[NM4 * NM4], B2[NM2 * NM2];
  gather19(ub, vb, wb, d);
  init_maps();
  beta_gram(NM4, 4, 1.0, B4);
  beta_gram(NM2, 2, 1.0, B2);
  candidates(d, n_gauss, B4, B2, val, beta);
  return npoints(n_gauss);
}

/* coefficients (monomial order of the file header) of p0 (15) and of the
 * quadratic p_n, n = 1..4 (6), from the 19 data */
void hwo2d_p0_coeffs(const double* d19, double* c15) {
  init_maps();
  hwo_matvec(NM4, ND, M0, d19, c15);
}

void hwo2d_quad_coeffs(int n, const double* d19, double* c6) {
  init_maps();
  hwo_matvec(NM2, ND, MQ[n - 1], d19, c6);
}

double hwo2d_beta_of_coeffs(int degree, const double* c, double ratio) {
  init_maps();
  double B[NM4 * NM4];
  int nm = degree == 4 ? NM4 : NM2;
  beta_gram(nm, degree, ratio, B);
  return quad_form(nm, B, c);
}

/* W (np x 19): the linear map from the 19 data to p0 at the points above. */
int hwo2d_linear_weights(int n_gauss, double* W) {
  init_tables(n_gauss);
  const int np = npoints(n_gauss);
  for (int p = 0; p < np; ++p)
    for (int k = 0; k < ND; ++k) W[p * ND + k] = W0[n_gauss][p][k];
  return np;
}

/* ---------------------------------------------------------------------- */
/* Physics: Burgers f = g = u^2/2; Euler Eq. (euler2).                     */
/* ---------------------------------------------------------------------- */

int hwo2d_ncomp(int system) { return system == HWO_EULER ? 4 : 1; }

void hwo_euler2d_flux(double g, const double* U, int dir, double* F) {
  double rho = U[0], mu = U[1] / rho, nu = U[2] / rho, E = U[3];
  double p = (g - 1.0) * (E - 0.5 * rho * (mu * mu + nu * nu));
  double vn = dir == 0 ? mu : nu;
  F[0] = rho * vn;
  F[1] = U[1] * vn + (dir == 0 ? p : 0.0);
  F[2] = U[2] * vn + (dir == 1 ? p : 0.0);
  F[3] = vn * (E + p);
}

/* right eigenvectors of dF/dU (dir 0) or dG/dU (dir 1); L by inversion */
void hwo_euler2d_eigen(double g, const double* U, int dir, double R[16], double L[16]) {
  double rho = U[0], mu = U[1] / rho, nu = U[2] / rho, E = U[3];
  double q2 = mu * mu + nu * nu;
  double p = (g - 1.0) * (E - 0.5 * rho * q2);
  double c = sqrt(g * p / rho), H = (E + p) / rho;
  double cols[4][4];
  if (dir == 0) {
    double c1[4] = {1.0, mu - c, nu, H - mu * c};
    double c2[4] = {1.0, mu, nu, 0.5 * q2};
    double c3[4] = {0.0, 0.0, 1.0, nu};
    double c4[4] = {1.0, mu + c, nu, H + mu * c};
    memcpy(cols[0], c1, sizeof(c1)); memcpy(cols[1], c2, sizeof(c2));
    memcpy(cols[2], c3, sizeof(c3)); memcpy(cols[3], c4, sizeof(c4));
  } else {
    double c1[4] = {1.0, mu, nu - c, H - nu * c};
    double c2[4] = {1.0, mu, nu, 0.5 * q2};
    double c3[4] = {0.0, 1.0, 0.0, mu};
    double c4[4] = {1.0, mu, nu + c, H + nu * c};
    memcpy(cols[0], c1, sizeof(c1)); memcpy(cols[1], c2, sizeof(c2));
    memcpy(cols[2], c3, sizeof(c3)); memcpy(cols[3], c4, sizeof(c4));
  }
  for (int r = 0; r < 4; ++r)
    for (int k = 0; k < 4; ++k) R[r * 4 + k] = cols[k][r];
  if (hwo_mat_inverse(4, R, L) != 0)
    for (int k = 0; k < 16; ++k) L[k] = NAN;
}

static void phys_flux2(const hwo2d_cfg* cfg, const double* U, int dir, double* F) {
  if (cfg->system == HWO_EULER)
    hwo_euler2d_flux(cfg->gas_gamma, U, dir, F);
  else
    F[0] = 0.5 * U[0] * U[0];
}

/* max |f'| (dir 0) or |g'| (dir 1) at a state; NaN if not physical */
static double wave_speed2(const hwo2d_cfg* cfg, const double* U, int dir) {
  if (cfg->system != HWO_EULER) return fabs(U[0]);
  double g = cfg->gas_gamma, rho = U[0], mu = U[1] / rho, nu = U[2] / rho;
  double p = (g - 1.0) * (U[3] - 0.5 * rho * (mu * mu + nu * nu));
  if (!(rho > 0.0) || !(p > 0.0)) return NAN;
  return fabs(dir == 0 ? mu : nu) + sqrt(g * p / rho);
}

/* Reading: alpha (x) and beta (y) of the Lax-Friedrichs fluxes are the
 * maxima over the cell averages of the stage input. */
void hwo2d_alpha(const hwo2d_cfg* cfg, const double* u, double* ax, double* ay) {
  const int C = hwo2d_ncomp(cfg->system), n = cfg->nx * cfg->ny;
  double a = 0.0, b = 0.0;
  for (int i = 0; i < n; ++i) {
    double U[4];
    for (int c = 0; c < C; ++c) U[c] = u[(c * 3 + 0) * n + i];
    double sx = wave_speed2(cfg, U, 0), sy = wave_speed2(cfg, U, 1);
    if (!(sx == sx) || !(sy == sy)) {
      *ax = *ay = NAN;
      return;
    }
    if (sx > a) a = sx;
    if (sy > b) b = sy;
  }
  *ax = a;
  *ay = b;
}

/* ---------------------------------------------------------------------- */
/* One evaluation of the right-hand side of Eq. (ode2).                    */
/* ---------------------------------------------------------------------- */

#define G2 3

static int map1(int i, int n, int bc) {
  if (bc == HWO_BC_PERIODIC) return ((i % n) + n) % n;
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

/* Reading of the KXRCF indicator in 2D (Krivodonova et al., degree-1 cell
 * polynomial ubar + 12 vbar xi + 12 wbar eta): the signed jumps across the
 * inflow faces integrated over those faces (the midpoint jump times the
 * length), divided by h |dI^-| max(|ubar|, 1e-12), h = sqrt(dx^2 + dy^2)/2.
 * The inflow x-face is the left one when the x-velocity is >= 0, the inflow
 * y-face the bottom one when the y-velocity is >= 0. */
static double kxrcf2d(const double* ub, const double* vb, const double* wb, int e, int sx,
                      int sy, double velx, double vely, double dx, double dy) {
  double jx, jy;
  if (velx >= 0.0)
    jx = (ub[e] - 6.0 * vb[e]) - (ub[e - sx] + 6.0 * vb[e - sx]);
  else
    jx = (ub[e] + 6.0 * vb[e]) - (ub[e + sx] - 6.0 * vb[e + sx]);
  if (vely >= 0.0)
    jy = (ub[e] - 6.0 * wb[e]) - (ub[e - sy] + 6.0 * wb[e - sy]);
  else
    jy = (ub[e] + 6.0 * wb[e]) - (ub[e + sy] - 6.0 * wb[e + sy]);
  double h = 0.5 * sqrt(dx * dx + dy * dy);
  double nrm = fabs(ub[e]);
  if (nrm < 1e-12) nrm = 1e-12;
  return fabs(dy * jx + dx * jy) / (h * (dx + dy) * nrm);
}

static void tau_weights5(const double* gam, double eps, const double beta[5], double omega[5]) {
  double s = 0.0;
  for (int n = 1; n < 5; ++n) s += fabs(beta[0] - beta[n]);
  s *= 0.25;
  hwo_nonlinear_weights(5, gam, eps, beta, s * s, omega);
}

int hwo2d_rhs(const hwo2d_cfg* cfg, const double* u, double alpha_x, double alpha_y,
              double* rhs, double* ulim, unsigned char* flags, double* indicator) {
  return hwo2d_rhs_fx(cfg, u, alpha_x, alpha_y, NULL, rhs, ulim, flags, indicator, NULL);
}

/* As hwo2d_rhs; points (nullable, [C][4 ng + ng^2][ny][nx]) receives the
 * reconstructed values at every point of every cell (order of
 * hwo2d_recon_candidates). */
int hwo2d_rhs_ex(const hwo2d_cfg* cfg, const double* u, double alpha_x, double alpha_y,
                 double* rhs, double* ulim, unsigned char* flags, double* indicator,
                 double* points) {
  return hwo2d_rhs_fx(cfg, u, alpha_x, alpha_y, NULL, rhs, ulim, flags, indicator, points);
}

/* As hwo2d_rhs_ex with the troubled cells given (flags_in, [ny][nx], nullable)
 * instead of decided by KXRCF: the operator with its switch held fixed, whose
 * derivative the adjoint computes.  Periodic boundaries only (a ghost cell is
 * troubled iff the cell it wraps to is); -1 otherwise. */
int hwo2d_rhs_fx(const hwo2d_cfg* cfg, const double* u, double alpha_x, double alpha_y,
                 const unsigned char* flags_in, double* rhs, double* ulim,
                 unsigned char* flags, double* indicator, double* points) {
  if (flags_in && cfg->bc != HWO_BC_PERIODIC) return -1;
  const int NX = cfg->nx, NY = cfg->ny, N = NX * NY;
  const int C = hwo2d_ncomp(cfg->system);
  const int EX = NX + 2 * G2, EY = NY + 2 * G2, NE = EX * EY;
  const double dx = (cfg->x1 - cfg->x0) / NX, dy = (cfg->y1 - cfg->y0) / NY;
  const int euler = cfg->system == HWO_EULER;
  const int ng = cfg->n_gauss == 2 ? 2 : 3, np = 4 * ng + ng * ng;
  if (NX < 3 || NY < 3) return -1;
  init_maps();
  if (alpha_x < 0.0 || alpha_y < 0.0) hwo2d_alpha(cfg, u, &alpha_x, &alpha_y);
  if (!(alpha_x == alpha_x) || !(alpha_y == alpha_y)) return -2;
  double gx[3], gw[3];
  gauss_points(ng, gx, gw);
  init_tables(ng);
  double B4[NM4 * NM4], B2[NM2 * NM2];
  beta_gram(NM4, 4, dy / dx, B4);
  beta_gram(NM2, 2, dy / dx, B2);

  double* ub = (double*)malloc(sizeof(double) * C * NE);
  double* vb = (double*)malloc(sizeof(double) * C * NE);
  double* wb = (double*)malloc(sizeof(double) * C * NE);
  double* vl = (double*)malloc(sizeof(double) * C * NE);
  double* wl = (double*)malloc(sizeof(double) * C * NE);
  double* ind = (double*)calloc(NE, sizeof(double));
  unsigned char* fl = (unsigned char*)calloc(NE, 1);
  double* pv = (double*)calloc((size_t)C * NE * np, sizeof(double)); /* point values */
  int status = 0;

  for (int ej = 0; ej < EY; ++ej)
    for (int ei = 0; ei < EX; ++ei) {
      int si = map1(ei - G2, NX, cfg->bc), sj = map1(ej - G2, NY, cfg->bc);
      int e = ej * EX + ei, s = sj * NX + si;
      for (int c = 0; c < C; ++c) {
        ub[c * NE + e] = u[(c * 3 + 0) * N + s];
        vb[c * NE + e] = u[(c * 3 + 1) * N + s];
        wb[c * NE + e] = u[(c * 3 + 2) * N + s];
      }
    }

  /* Step 4: troubled cells (Remark 3: u for Burgers with velocity (f', g');
   * rho and E for Euler with the velocity (mu, nu)). */
#pragma omp parallel for schedule(static)
  for (int ej = 1; ej < EY - 1; ++ej)
    for (int ei = 1; ei < EX - 1; ++ei) {
      int e = ej * EX + ei;
      double I;
      if (euler) {
        double vx = ub[1 * NE + e] / ub[0 * NE + e], vy = ub[2 * NE + e] / ub[0 * NE + e];
        double Ir = kxrcf2d(ub, vb, wb, e, 1, EX, vx, vy, dx, dy);
        double Ie = kxrcf2d(ub + 3 * NE, vb + 3 * NE, wb + 3 * NE, e, 1, EX, vx, vy, dx, dy);
        I = Ir > Ie ? Ir : Ie;
      } else {
        I = kxrcf2d(ub, vb, wb, e, 1, EX, ub[e], ub[e], dx, dy);
      }
      ind[e] = I;
      if (flags_in) {
        fl[e] = flags_in[map1(ej - G2, NY, cfg->bc) * NX + map1(ei - G2, NX, cfg->bc)] != 0;
        continue;
      }
      fl[e] = cfg->troubled_mode == HWO_TROUBLED_ALL ? 1
              : cfg->troubled_mode == HWO_TROUBLED_NONE ? 0
              : I > cfg->kxrcf_threshold;
    }

  /* Step 4: modify vbar from the x-neighbours and wbar from the y-neighbours
   * with the 1D formula (Euler: in the characteristic fields of the x- and of
   * the y-Jacobian at the cell's own average). */
  memcpy(vl, vb, sizeof(double) * C * NE);
  memcpy(wl, wb, sizeof(double) * C * NE);
#pragma omp parallel for schedule(static)
  for (int ej = 1; ej < EY - 1; ++ej)
    for (int ei = 1; ei < EX - 1; ++ei) {
      int e = ej * EX + ei;
      if (!fl[e]) continue;
      for (int dir = 0; dir < 2; ++dir) {
        int s = dir == 0 ? 1 : EX;
        const double* mb = dir == 0 ? vb : wb;
        double* ml = dir == 0 ? vl : wl;
        if (!euler) {
          double u3[3] = {ub[e - s], ub[e], ub[e + s]};
          ml[e] = hwo1d_limit_scalar(cfg->lin_w, cfg->eps, u3, mb[e - s], mb[e + s]);
        } else {
          double R[16], L[16], U[4], src[5][4], W[4][5], q[4], out[4];
          for (int c = 0; c < 4; ++c) U[c] = ub[c * NE + e];
          hwo_euler2d_eigen(cfg->gas_gamma, U, dir, R, L);
          for (int c = 0; c < 4; ++c) {
            src[0][c] = ub[c * NE + e - s];
            src[1][c] = ub[c * NE + e];
            src[2][c] = ub[c * NE + e + s];
            src[3][c] = mb[c * NE + e - s];
            src[4][c] = mb[c * NE + e + s];
          }
          for (int k = 0; k < 5; ++k) {
            double wv[4];
            hwo_matvec(4, 4, L, src[k], wv);
            for (int f = 0; f < 4; ++f) W[f][k] = wv[f];
          }
          for (int f = 0; f < 4; ++f)
            q[f] = hwo1d_limit_scalar(cfg->lin_w, cfg->eps, W[f], W[f][3], W[f][4]);
          hwo_matvec(4, 4, R, q, out);
          for (int c = 0; c < 4; ++c) ml[c * NE + e] = out[c];
        }
      }
    }

  /* Step 5: point values for cells -1..N (extended 2..E-3) */
#pragma omp parallel for schedule(static)
  for (int ej = 2; ej < EY - 2; ++ej)
    for (int ei = 2; ei < EX - 2; ++ei) {
      int e = ej * EX + ei;
      int hw = 0;
      for (int dj = -1; dj <= 1; ++dj)
        for (int di = -1; di <= 1; ++di) hw |= fl[e + dj * EX + di];
      /* gather the 3x3 stencil, component by component */
      double su[4][9], sv[4][9], sw[4][9];
      for (int k = 1; k <= 9; ++k) {
        int ee = e + CELL_DJ[k] * EX + CELL_DI[k];
        for (int c = 0; c < C; ++c) {
          su[c][k - 1] = ub[c * NE + ee];
          sv[c][k - 1] = vl[c * NE + ee];
          sw[c][k - 1] = wl[c * NE + ee];
        }
      }
      double* out = pv + (size_t)e * C * np; /* [c][p] */
      for (int c = 0; c < C; ++c) {
        double d[ND];
        gather19(su[c], sv[c], sw[c], d);
        /* Steps 5.2 and 5.3: the linear p0 at every point */
        for (int p = 0; p < np; ++p) {
          double s = 0.0;
          for (int k = 0; k < ND; ++k) s += W0[ng][p][k] * d[k];
          out[c * np + p] = s;
        }
        if (hw && !euler) {
          /* Step 5.1 at the interface points */
          double val[5 * NPMAX], beta[5], om[5];
          candidates(d, ng, B4, B2, val, beta);
          tau_weights5(cfg->lin_w, cfg->eps, beta, om);
          for (int p = 0; p < 4 * ng; ++p) {
            double v5[5];
            for (int n = 0; n < 5; ++n) v5[n] = val[n * np + p];
            out[c * np + p] = hwo_combine(5, cfg->lin_w, om, v5);
          }
        }
      }
      if (hw && euler) {
        /* Step 5.1 in characteristic fields: x-faces with the x-Jacobian,
         * y-faces with the y-Jacobian, both at the cell average (Remark 4), or
         * with char_state at the mean of the averages on the two sides of the
         * face (one eigen-system per face) */
        for (int dir = 0; dir < 2; ++dir)
        for (int side = 0; side < 2; ++side) {
          const int nb = dir == 0 ? (side == 0 ? 3 : 5) : (side == 0 ? 1 : 7);
          double R[16], L[16], U[4];
          for (int c = 0; c < 4; ++c)
            U[c] = cfg->char_state ? 0.5 * (su[c][4] + su[c][nb]) : su[c][4];
          hwo_euler2d_eigen(cfg->gas_gamma, U, dir, R, L);
          double cu[4][9], cv[4][9], cw[4][9];
          for (int k = 0; k < 9; ++k) {
            double a[4], b[4], d[4], ra[4], rb[4], rd[4];
            for (int c = 0; c < 4; ++c) { a[c] = su[c][k]; b[c] = sv[c][k]; d[c] = sw[c][k]; }
            hwo_matvec(4, 4, L, a, ra);
            hwo_matvec(4, 4, L, b, rb);
            hwo_matvec(4, 4, L, d, rd);
            for (int f = 0; f < 4; ++f) { cu[f][k] = ra[f]; cv[f][k] = rb[f]; cw[f][k] = rd[f]; }
          }
          double chv[4][12];
          for (int f = 0; f < 4; ++f) {
            double val[5 * NPMAX], beta[5], om[5], d[ND];
            gather19(cu[f], cv[f], cw[f], d);
            candidates(d, ng, B4, B2, val, beta);
            tau_weights5(cfg->lin_w, cfg->eps, beta, om);
            for (int p = side * ng; p < (side + 1) * ng; ++p) {
              int pp = dir * 2 * ng + p;
              double v5[5];
              for (int n = 0; n < 5; ++n) v5[n] = val[n * np + pp];
              chv[f][p] = hwo_combine(5, cfg->lin_w, om, v5);
            }
          }
          for (int p = side * ng; p < (side + 1) * ng; ++p) {
            double wv[4], cv4[4];
            for (int f = 0; f < 4; ++f) wv[f] = chv[f][p];
            hwo_matvec(4, 4, R, wv, cv4);
            for (int c = 0; c < 4; ++c) out[c * np + dir * 2 * ng + p] = cv4[c];
          }
        }
      }
    }

  /* fluxes and Eq. (ode2) */
#pragma omp parallel for schedule(static) reduction(min : status)
  for (int j = 0; j < NY; ++j)
    for (int i = 0; i < NX; ++i) {
      int e = (j + G2) * EX + (i + G2);
      const double* me = pv + (size_t)e * C * np;
      const double* ml_ = pv + (size_t)(e - 1) * C * np;
      const double* mr = pv + (size_t)(e + 1) * C * np;
      const double* mbot = pv + (size_t)(e - EX) * C * np;
      const double* mtop = pv + (size_t)(e + EX) * C * np;
      double FL[3][4], FR[3][4], GB[3][4], GT[3][4];
      for (int k = 0; k < ng; ++k) {
        double a[4], b[4], fa[4], fb[4];
        /* left face x_{i-1/2}: u^- from cell i-1 (its right face), u^+ own left face */
        for (int c = 0; c < C; ++c) { a[c] = ml_[c * np + ng + k]; b[c] = me[c * np + k]; }
        phys_flux2(cfg, a, 0, fa); phys_flux2(cfg, b, 0, fb);
        for (int c = 0; c < C; ++c) FL[k][c] = 0.5 * (fa[c] + fb[c]) - 0.5 * alpha_x * (b[c] - a[c]);
        /* right face x_{i+1/2}: u^- own right face, u^+ from cell i+1 (its left face) */
        for (int c = 0; c < C; ++c) { a[c] = me[c * np + ng + k]; b[c] = mr[c * np + k]; }
        phys_flux2(cfg, a, 0, fa); phys_flux2(cfg, b, 0, fb);
        for (int c = 0; c < C; ++c) FR[k][c] = 0.5 * (fa[c] + fb[c]) - 0.5 * alpha_x * (b[c] - a[c]);
        /* bottom face y_{j-1/2}: u^- from cell j-1 (its top face), u^+ own bottom */
        for (int c = 0; c < C; ++c) { a[c] = mbot[c * np + 3 * ng + k]; b[c] = me[c * np + 2 * ng + k]; }
        phys_flux2(cfg, a, 1, fa); phys_flux2(cfg, b, 1, fb);
        for (int c = 0; c < C; ++c) GB[k][c] = 0.5 * (fa[c] + fb[c]) - 0.5 * alpha_y * (b[c] - a[c]);
        /* top face y_{j+1/2}: u^- own top face, u^+ from cell j+1 (its bottom) */
        for (int c = 0; c < C; ++c) { a[c] = me[c * np + 3 * ng + k]; b[c] = mtop[c * np + 2 * ng + k]; }
        phys_flux2(cfg, a, 1, fa); phys_flux2(cfg, b, 1, fb);
        for (int c = 0; c < C; ++c) GT[k][c] = 0.5 * (fa[c] + fb[c]) - 0.5 * alpha_y * (b[c] - a[c]);
      }
      /* volume integrals of f and g by the tensor Gauss rule */
      double Fv[4] = {0, 0, 0, 0}, Gv[4] = {0, 0, 0, 0};
      for (int l = 0; l < ng; ++l)
        for (int k = 0; k < ng; ++k) {
          double U[4], f[4], g[4];
          for (int c = 0; c < C; ++c) U[c] = me[c * np + 4 * ng + l * ng + k];
          phys_flux2(cfg, U, 0, f);
          phys_flux2(cfg, U, 1, g);
          for (int c = 0; c < C; ++c) {
            Fv[c] += gw[k] * gw[l] * f[c];
            Gv[c] += gw[k] * gw[l] * g[c];
          }
        }
      for (int c = 0; c < C; ++c) {
        double sfx = 0, sfs = 0, sfxe = 0, sgy = 0, sgs = 0, sgyx = 0;
        for (int k = 0; k < ng; ++k) {
          sfx += gw[k] * (FR[k][c] - FL[k][c]);
          sfs += gw[k] * (FL[k][c] + FR[k][c]);
          sfxe += gw[k] * gx[k] * (FR[k][c] - FL[k][c]);
          sgy += gw[k] * (GT[k][c] - GB[k][c]);
          sgs += gw[k] * (GB[k][c] + GT[k][c]);
          sgyx += gw[k] * gx[k] * (GT[k][c] - GB[k][c]);
        }
        int s = j * NX + i;
        /* Eq. (ode2); the w-equation's volume term carries 1/(dx dy^2) */
        rhs[(c * 3 + 0) * N + s] = -sfx / dx - sgy / dy;
        rhs[(c * 3 + 1) * N + s] = -sfs / (2.0 * dx) + Fv[c] / dx - sgyx / dy;
        rhs[(c * 3 + 2) * N + s] = -sfxe / dx - sgs / (2.0 * dy) + Gv[c] / dy;
        for (int m = 0; m < 3; ++m)
          if (!(rhs[(c * 3 + m) * N + s] == rhs[(c * 3 + m) * N + s])) status = -3;
        if (ulim) {
          ulim[(c * 3 + 0) * N + s] = ub[c * NE + e];
          ulim[(c * 3 + 1) * N + s] = vl[c * NE + e];
          ulim[(c * 3 + 2) * N + s] = wl[c * NE + e];
        }
      }
      if (flags) flags[j * NX + i] = fl[e];
      if (indicator) indicator[j * NX + i] = ind[e];
      if (points)
        for (int c = 0; c < C; ++c)
          for (int p = 0; p < np; ++p) points[((size_t)(c * np + p) * NY + j) * NX + i] = me[c * np + p];
    }

  free(ub); free(vb); free(wb); free(vl); free(wl); free(ind); free(fl); free(pv);
  return status;
}

/* Reading: dt = CFL / (alpha_x/dx + alpha_y/dy) from u^n; a step clipped to
 * t_final is the last one (as in 1D). */
double hwo2d_dt(const hwo2d_cfg* cfg, const double* u, double cfl, double t,
                double t_final) {
  double dx = (cfg->x1 - cfg->x0) / cfg->nx, dy = (cfg->y1 - cfg->y0) / cfg->ny;
  double ax, ay;
  hwo2d_alpha(cfg, u, &ax, &ay);
  double dt = cfl / (ax / dx + ay / dy);
  if (t_final > 0.0) {
    double rem = t_final - t;
    if (rem <= 0.0) return 0.0;
    if (dt > rem) dt = rem;
  }
  return dt;
}

int hwo2d_step(const hwo2d_cfg* cfg, double* u, double dt, long* n_troubled) {
  const int C = hwo2d_ncomp(cfg->system), N = cfg->nx * cfg->ny;
  const size_t S = (size_t)C * 3 * N;
  if (!(dt > 0.0)) return 0;
  double* L = (double*)malloc(sizeof(double) * S);
  double* b0 = (double*)malloc(sizeof(double) * S);
  double* bk = (double*)malloc(sizeof(double) * S);
  double* uk = (double*)malloc(sizeof(double) * S);
  unsigned char* fl = (unsigned char*)malloc(N);
  long nt = 0;
  int st = hwo2d_rhs(cfg, u, -1.0, -1.0, L, b0, fl, NULL);
  for (int i = 0; i < N; ++i) nt += fl[i];
  if (!cfg->limit_in_place) memcpy(b0, u, sizeof(double) * S);
  for (size_t k = 0; k < S && !st; ++k) uk[k] = b0[k] + dt * L[k];
  if (!st) st = hwo2d_rhs(cfg, uk, -1.0, -1.0, L, bk, fl, NULL);
  for (int i = 0; i < N && !st; ++i) nt += fl[i];
  if (!cfg->limit_in_place) memcpy(bk, uk, sizeof(double) * S);
  for (size_t k = 0; k < S && !st; ++k) uk[k] = 0.75 * b0[k] + 0.25 * bk[k] + 0.25 * dt * L[k];
  if (!st) st = hwo2d_rhs(cfg, uk, -1.0, -1.0, L, bk, fl, NULL);
  for (int i = 0; i < N && !st; ++i) nt += fl[i];
  if (!cfg->limit_in_place) memcpy(bk, uk, sizeof(double) * S);
  for (size_t k = 0; k < S && !st; ++k)
    u[k] = (1.0 / 3.0) * b0[k] + (2.0 / 3.0) * bk[k] + (2.0 / 3.0) * dt * L[k];
  if (n_troubled) *n_troubled += nt;
  free(L); free(b0); free(bk); free(uk); free(fl);
  return st;
}

int hwo2d_run(const hwo2d_cfg* cfg, double* u, int nsteps, double cfl, double t0,
              double t_final, double dt_fixed, const double* lin_w_per_step, double* t_out,
              long* n_troubled) {
  double t = t0;
  int st = 0;
  hwo2d_cfg c = *cfg;
  const double dx = (cfg->x1 - cfg->x0) / cfg->nx, dy = (cfg->y1 - cfg->y0) / cfg->ny;
  for (int s = 0; nsteps < 0 || s < nsteps; ++s) {
    double dt;
    if (dt_fixed > 0.0) {
      dt = dt_fixed;
    } else {
      double ax, ay;
      hwo2d_alpha(&c, u, &ax, &ay);
      dt = cfl / (ax / dx + ay / dy);
    }
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
      for (int k = 0; k < 5; ++k) c.lin_w[k] = lin_w_per_step[5 * s + k];
    st = hwo2d_step(&c, u, dt, n_troubled);
    if (st) break;
    t = last ? t_final : t + dt;
    if (last) break;
  }
  if (t_out) *t_out = t;
  return st;
}
