/* Textbook dense linear algebra for the oracle: Householder QR (Golub & Van Loan, Alg. 5.2.1) and
 * Gaussian elimination with partial pivoting.  TEST INFRASTRUCTURE ONLY. */
#include <math.h>
#include <string.h>
#include "orc.h"

int orc_qr_factor(int m, int n, const double* A, orc_qr* f) {
  double W[24 * 9];
  if (m > 24 || n > 9 || m < n) return -1;
  memcpy(W, A, sizeof(double) * m * n);
  f->m = m;
  f->n = n;
  memset(f->V, 0, sizeof(f->V));
  memset(f->R, 0, sizeof(f->R));
  for (int k = 0; k < n; ++k) {
    double* x = W + k * m;
    double nrm = 0.0;
    for (int i = k; i < m; ++i) nrm += x[i] * x[i];
    nrm = sqrt(nrm);
    if (nrm == 0.0) return -2; /* rank deficient */
    double alpha = x[k] > 0.0 ? -nrm : nrm;
    double* v = f->V + k * m;
    for (int i = 0; i < m; ++i) v[i] = 0.0;
    for (int i = k; i < m; ++i) v[i] = x[i];
    v[k] -= alpha;
    double vv = 0.0;
    for (int i = k; i < m; ++i) vv += v[i] * v[i];
    f->tau[k] = 2.0 / vv;
    /* apply the reflector to the remaining columns */
    for (int j = k; j < n; ++j) {
      double* a = W + j * m;
      double d = 0.0;
      for (int i = k; i < m; ++i) d += v[i] * a[i];
      d *= f->tau[k];
      for (int i = k; i < m; ++i) a[i] -= d * v[i];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = i; j < n; ++j) f->R[i * n + j] = W[j * m + i];
  for (int i = 0; i < n; ++i)
    if (f->R[i * n + i] == 0.0) return -2;
  return 0;
}

void orc_qr_qt(const orc_qr* f, double* b) {
  for (int k = 0; k < f->n; ++k) {
    const double* v = f->V + k * f->m;
    double d = 0.0;
    for (int i = k; i < f->m; ++i) d += v[i] * b[i];
    d *= f->tau[k];
    for (int i = k; i < f->m; ++i) b[i] -= d * v[i];
  }
}

void orc_qr_q(const orc_qr* f, double* b) {
  for (int k = f->n - 1; k >= 0; --k) {
    const double* v = f->V + k * f->m;
    double d = 0.0;
    for (int i = k; i < f->m; ++i) d += v[i] * b[i];
    d *= f->tau[k];
    for (int i = k; i < f->m; ++i) b[i] -= d * v[i];
  }
}

int orc_ge_solve(int n, const double* A, const double* b, double* x) {
  double a[9][10];
  if (n > 9) return -1;
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) a[i][j] = A[i * n + j];
    a[i][n] = b[i];
  }
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (fabs(a[i][k]) > fabs(a[p][k])) p = i;
    if (a[p][k] == 0.0) return -2;
    if (p != k)
      for (int j = 0; j <= n; ++j) {
        double t = a[k][j];
        a[k][j] = a[p][j];
        a[p][j] = t;
      }
    for (int i = k + 1; i < n; ++i) {
      double l = a[i][k] / a[k][k];
      for (int j = k; j <= n; ++j) a[i][j] -= l * a[k][j];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = a[i][n];
    for (int j = i + 1; j < n; ++j) s -= a[i][j] * x[j];
    x[i] = s / a[i][i];
  }
  return 0;
}
