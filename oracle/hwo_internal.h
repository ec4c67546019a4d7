/*
 * ORACLE -- test infrastructure only.  Helpers shared by the 1D and 2D oracle
 * translation units (never by the CUDA path).
 */
#ifndef HWO_INTERNAL_H
#define HWO_INTERNAL_H

/* integral of xi^k over [a, b] */
double hwo_mono_int(int k, double a, double b);

/* Gauss-Jordan inverse with partial pivoting of the n x n row-major matrix a;
 * returns 0, or -1 when a pivot vanishes. */
int hwo_mat_inverse(int n, const double* a, double* inv);

/* y = A x for an m x n row-major A */
void hwo_matvec(int m, int n, const double* A, const double* x, double* y);

/* Nonlinear weights of the HWENO combination (Sec. 2.1 Step 1, Eq. for
 * omega_n; Sec. 2.2 Eq. (99)):
 *   wbar_n = gamma_n (1 + tau / (beta_n + eps)),  omega_n = wbar_n / sum wbar */
void hwo_nonlinear_weights(int ncand, const double* gam, double eps,
                           const double* beta, double tau, double* omega);

/* omega_0 (val_0/gamma_0 - sum_{n>=1} gamma_n/gamma_0 val_n) + sum_{n>=1}
 * omega_n val_n  (Sec. 2.1 Step 1 last formula, Step 2.1, Step 5.1) */
double hwo_combine(int ncand, const double* gam, const double* omega,
                   const double* val);

#endif
