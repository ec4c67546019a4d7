/*
 * ORACLE -- test infrastructure only.  Small dense linear algebra, monomial
 * integrals and the HWENO nonlinear combination, written out plainly.
 */
#include <math.h>
#include <string.h>

#include "hwo_internal.h"

double hwo_mono_int(int k, double a, double b) {
  return (pow(b, k + 1) - pow(a, k + 1)) / (double)(k + 1);
}

int hwo_mat_inverse(int n, const double* a, double* inv) {
  double m[64 * 128];
  int w = 2 * n;
  if (n > 64) return -1;
  for (int r = 0; r < n; ++r) {
    for (int c = 0; c < n; ++c) m[r * w + c] = a[r * n + c];
    for (int c = 0; c < n; ++c) m[r * w + n + c] = (r == c) ? 1.0 : 0.0;
  }
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (fabs(m[r * w + col]) > fabs(m[piv * w + col])) piv = r;
    if (fabs(m[piv * w + col]) < 1e-300) return -1;
    if (piv != col)
      for (int c = 0; c < w; ++c) {
        double t = m[col * w + c];
        m[col * w + c] = m[piv * w + c];
        m[piv * w + c] = t;
      }
    double p = m[col * w + col];
    for (int c = 0; c < w; ++c) m[col * w + c] /= p;
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      double f = m[r * w + col];
      if (f == 0.0) continue;
      for (int c = 0; c < w; ++c) m[r * w + c] -= f * m[col * w + c];
    }
  }
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) inv[r * n + c] = m[r * w + n + c];
  return 0;
}

void hwo_matvec(int m, int n, const double* A, const double* x, double* y) {
  for (int r = 0; r < m; ++r) {
    double s = 0.0;
    for (int c = 0; c < n; ++c) s += A[r * n + c] * x[c];
    y[r] = s;
  }
}

void hwo_nonlinear_weights(int ncand, const double* gam, double eps,
                           const double* beta, double tau, double* omega) {
  double wbar[8], sum = 0.0;
  for (int n = 0; n < ncand; ++n) {
    wbar[n] = gam[n] * (1.0 + tau / (beta[n] + eps));
    sum += wbar[n];
  }
  for (int n = 0; n < ncand; ++n) omega[n] = wbar[n] / sum;
}

double hwo_combine(int ncand, const double* gam, const double* omega,
                   const double* val) {
  double big = val[0] / gam[0];
  for (int n = 1; n < ncand; ++n) big -= gam[n] / gam[0] * val[n];
  double out = omega[0] * big;
  for (int n = 1; n < ncand; ++n) out += omega[n] * val[n];
  return out;
}

/* Threads of the OpenMP build (the per-cell loops of Eq. (odeH) and Eq. (ode2)
 * carry "omp parallel for" pragmas; the plain build ignores them): sets the
 * count when n > 0 and returns the count in use (1 in the plain build).  The
 * arithmetic of every cell is the same in both builds. */
#ifdef _OPENMP
#include <omp.h>
#endif
int hwo_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}
