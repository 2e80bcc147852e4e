/* Oracle CGKS residual, explicit step and multigrid V-cycle.  TEST INFRASTRUCTURE ONLY.
 *
 * Fine level (Sec. 2.2, 2.4 and 3 of the paper): HWENO reconstruction -> gas-kinetic flux and
 * interface state at every face Gauss point -> finite-volume residual and Gauss-Green gradient update
 * with the gradient compression factor.  Coarse levels (Sec. 4.2): first-order KFVS with forward-Euler
 * smoothing, FAS forcing, volume-weighted restriction and injection prolongation.
 *
 * Readings (paper silent/garbled):
 *  - Eq. smo: W^{n+1} = W^n + (dt_i/|Omega_i|) Res_i with Res_i = -(total outward flux of cell i);
 *  - local time step dt_i = CFL |Omega_i| / sum_p S_p (|U_i.n_p| + c_i + 2 nu_i S_p/|Omega_i|),
 *    nu = mu/rho (0 for inviscid flow and on the KFVS levels), the face uses min(dt_L, dt_R);
 *    dt_mode 1 uses the global minimum instead;
 *  - the residual restricted after the pre-smoothing step is a second fine residual evaluated at
 *    W^{n+1} (its gradient and compression-factor outputs are discarded);
 *  - the level-3 defect is the sum over level-2 cells of Res_2(W_2^{k}) + F_2 (FAS recursion);
 *  - only W is corrected on the fine level; a correction or a coarse forward-Euler update that would
 *    make rho or p non-positive in a cell is skipped for that cell (counted);
 *  - HWENO: sigma = |beta~_2 - beta~_1| (the printed beta~_0 does not exist), beta_2 from p^2,
 *    beta_1 = min(beta_GG of the alpha-scaled Green-Gauss p^1, beta_LS of the unweighted
 *    least-squares gradient), Omega = |Omega_0|, reconstruction of conservative variables;
 *  - Green-Gauss p^1 with the missing 1/|Omega_0|; p^1 uses the compression factor of the previous
 *    step; the compression factor is evaluated on interior (and periodic) faces only;
 *  - ghost cells for the boundary faces of the stencil: the cell mirrored in the face plane, with the
 *    boundary-condition transform of its average and gradient.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "orc.h"

typedef struct orc_solver {
  orc_mesh* M;
  orc_params P;
  orc_phys ph;
  double *W, *G, *alpha; /* [nc][5], [nc][15], [nc] */
  double r1;             /* first residual norm of the run */
  int64_t iters;
  int64_t skipped_corrections;
  int32_t* colors[8]; /* LU-SGS cell colours per level (computed on first use) */
  int ncolors[8];
} orc_solver;

int orc_build_levels(orc_mesh* M, const orc_params* P, char* err);

/* ------------------------------------------------------------------------------------------- */
/* reconstruction                                                                               */

typedef struct {
  int nf;
  double dlt[ORC_MAXNF][3]; /* neighbour centroid - own centroid (translated / mirrored) */
  double m2n[ORC_MAXNF][6]; /* neighbour central second-moment averages */
  double Sn[ORC_MAXNF][3];  /* outward area vectors */
  double Qn[ORC_MAXNF][5], Gn[ORC_MAXNF][15];
} stencil;

static void face_sum(const orc_mesh* M, int64_t f, double Sn[3], double* area, double xc[3]) {
  orc_face_centre(M, f, xc, Sn, area);
}

static void mirror_m2(const double m[6], const double n[3], double out[6]) {
  double A[3][3] = {{m[0], m[3], m[5]}, {m[3], m[1], m[4]}, {m[5], m[4], m[2]}}, R[3][3], T[3][3], B[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) R[i][j] = (i == j) - 2.0 * n[i] * n[j];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T[i][j] = 0.0;
      for (int k = 0; k < 3; ++k) T[i][j] += R[i][k] * A[k][j];
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      B[i][j] = 0.0;
      for (int k = 0; k < 3; ++k) B[i][j] += T[i][k] * R[k][j];
    }
  out[0] = B[0][0];
  out[1] = B[1][1];
  out[2] = B[2][2];
  out[3] = B[0][1];
  out[4] = B[1][2];
  out[5] = B[0][2];
}

static int build_stencil(const orc_solver* S, const double* W, const double* G, int64_t i, stencil* st) {
  const orc_mesh* M = S->M;
  st->nf = orc_nfaces(M->ctype[i]);
  for (int m = 0; m < st->nf; ++m) {
    int64_t f = M->cf[6 * i + m];
    int side = M->cside[6 * i + m];
    double sg = side ? -1.0 : 1.0, Sn[3], area, xc[3];
    face_sum(M, f, Sn, &area, xc);
    for (int d = 0; d < 3; ++d) st->Sn[m][d] = sg * Sn[d];
    if (M->fR[f] >= 0) {
      int64_t nb = side ? M->fL[f] : M->fR[f];
      for (int d = 0; d < 3; ++d)
        st->dlt[m][d] = M->ctr[3 * nb + d] + sg * M->shift[3 * f + d] - M->ctr[3 * i + d];
      memcpy(st->m2n[m], M->m2 + 6 * nb, 6 * sizeof(double));
      memcpy(st->Qn[m], W + 5 * nb, 5 * sizeof(double));
      memcpy(st->Gn[m], G + 15 * nb, 15 * sizeof(double));
    } else {
      double nrm = sqrt(Sn[0] * Sn[0] + Sn[1] * Sn[1] + Sn[2] * Sn[2]);
      double n[3] = {Sn[0] / nrm, Sn[1] / nrm, Sn[2] / nrm};
      const double* c = M->ctr + 3 * i;
      double h = (c[0] - xc[0]) * n[0] + (c[1] - xc[1]) * n[1] + (c[2] - xc[2]) * n[2];
      for (int d = 0; d < 3; ++d) st->dlt[m][d] = -2.0 * h * n[d];
      mirror_m2(M->m2 + 6 * i, n, st->m2n[m]);
      if (orc_bc_ghost(&S->ph, M->ftag[f], n, W + 5 * i, G + 15 * i, st->Qn[m], st->Gn[m])) return -1;
    }
  }
  return 0;
}

/* averages over a stencil cell of the nine non-constant basis functions X,Y,Z,X^2,Y^2,Z^2,XY,YZ,XZ
   (X = x - x_0) given its centroid offset and central moments */
static void basis_avg(const double dl[3], const double m[6], double a[9]) {
  a[0] = dl[0];
  a[1] = dl[1];
  a[2] = dl[2];
  a[3] = m[0] + dl[0] * dl[0];
  a[4] = m[1] + dl[1] * dl[1];
  a[5] = m[2] + dl[2] * dl[2];
  a[6] = m[3] + dl[0] * dl[1];
  a[7] = m[4] + dl[1] * dl[2];
  a[8] = m[5] + dl[0] * dl[2];
}
/* averages over a stencil cell of d/dx_d of the basis functions */
static void basis_davg(const double dl[3], int d, double a[9]) {
  for (int j = 0; j < 9; ++j) a[j] = 0.0;
  a[d] = 1.0;
  if (d == 0) {
    a[3] = 2.0 * dl[0];
    a[6] = dl[1];
    a[8] = dl[2];
  } else if (d == 1) {
    a[4] = 2.0 * dl[1];
    a[6] = dl[0];
    a[7] = dl[2];
  } else {
    a[5] = 2.0 * dl[2];
    a[7] = dl[1];
    a[8] = dl[0];
  }
}

/* R coefficients rc[5][10] of one cell in the basis 1,X,Y,Z,X^2,Y^2,Z^2,XY,YZ,XZ (Sec. 3) */
static int reconstruct_cell_mode(const orc_solver* S, const double* W, const double* G, const double* alpha_prev,
                                 int64_t i, double rc[5][10], int mode) {
  const orc_mesh* M = S->M;
  stencil st;
  if (build_stencil(S, W, G, i, &st)) return -1;
  const int nf = st.nf;
  const double V = M->vol[i];
  const double* m0 = M->m2 + 6 * i;
  double a0avg[9] = {0, 0, 0, m0[0], m0[1], m0[2], m0[3], m0[4], m0[5]};
  /* equality constraints C b = dQ (cell averages of the neighbours) and least-squares rows B b ~ g
     (averaged gradients of the neighbours) for the nine non-constant coefficients b of p^2 */
  double C[ORC_MAXNF][9], B[3 * ORC_MAXNF][9];
  for (int m = 0; m < nf; ++m) {
    double a[9];
    basis_avg(st.dlt[m], st.m2n[m], a);
    for (int j = 0; j < 9; ++j) C[m][j] = a[j] - a0avg[j];
    for (int d = 0; d < 3; ++d) basis_davg(st.dlt[m], d, B[3 * m + d]);
  }
  /* null-space method: C^T = Q [R; 0], b = Q1 z1 + Q2 z2, R^T z1 = dQ, min |B Q2 z2 - (g - B Q1 z1)| */
  double Ct[9 * ORC_MAXNF];
  for (int m = 0; m < nf; ++m)
    for (int j = 0; j < 9; ++j) Ct[j + 9 * m] = C[m][j];
  orc_qr qc, qb;
  if (orc_qr_factor(9, nf, Ct, &qc)) return -2;
  double Q[9][9]; /* Q[:, col] */
  for (int col = 0; col < 9; ++col) {
    double e[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    e[col] = 1.0;
    orc_qr_q(&qc, e);
    for (int r = 0; r < 9; ++r) Q[r][col] = e[r];
  }
  const int nz = 9 - nf, mb = 3 * nf;
  double BQ2[3 * ORC_MAXNF * 9];
  for (int c = 0; c < nz; ++c)
    for (int r = 0; r < mb; ++r) {
      double s = 0.0;
      for (int j = 0; j < 9; ++j) s += B[r][j] * Q[j][nf + c];
      BQ2[r + mb * c] = s;
    }
  if (orc_qr_factor(mb, nz, BQ2, &qb)) return -2;
  /* least-squares gradient: min sum_m (Q_m - Q_0 - g . dlt_m)^2 */
  double D[ORC_MAXNF * 3];
  for (int m = 0; m < nf; ++m)
    for (int d = 0; d < 3; ++d) D[m + nf * d] = st.dlt[m][d];
  orc_qr qd;
  if (orc_qr_factor(nf, 3, D, &qd)) return -2;
  const double al = alpha_prev ? alpha_prev[i] : 1.0;
  const double g1 = 0.5, g2 = 0.5, eps = S->P.weno_eps;
  const double V23 = pow(V, 2.0 / 3.0), V13 = pow(V, 1.0 / 3.0), Vm13 = pow(V, -1.0 / 3.0);
  for (int q = 0; q < 5; ++q) {
    const double Q0 = W[5 * i + q];
    double dQ[ORC_MAXNF], gv[3 * ORC_MAXNF];
    for (int m = 0; m < nf; ++m) {
      dQ[m] = st.Qn[m][q] - Q0;
      for (int d = 0; d < 3; ++d) gv[3 * m + d] = st.Gn[m][3 * q + d];
    }
    /* z1 from R^T z1 = dQ */
    double z[9];
    for (int r = 0; r < nf; ++r) {
      double s = dQ[r];
      for (int k = 0; k < r; ++k) s -= qc.R[k * nf + r] * z[k];
      z[r] = s / qc.R[r * nf + r];
    }
    double rhs[3 * ORC_MAXNF];
    for (int r = 0; r < mb; ++r) {
      double s = gv[r];
      for (int j = 0; j < 9; ++j) {
        double q1z = 0.0;
        for (int k = 0; k < nf; ++k) q1z += Q[j][k] * z[k];
        s -= B[r][j] * q1z;
      }
      rhs[r] = s;
    }
    orc_qr_qt(&qb, rhs);
    for (int r = nz - 1; r >= 0; --r) {
      double s = rhs[r];
      for (int k = r + 1; k < nz; ++k) s -= qb.R[r * nz + k] * z[nf + k];
      z[nf + r] = s / qb.R[r * nz + r];
    }
    double b[9];
    for (int j = 0; j < 9; ++j) {
      b[j] = 0.0;
      for (int k = 0; k < 9; ++k) b[j] += Q[j][k] * z[k];
    }
    double a0 = Q0;
    for (int j = 3; j < 9; ++j) a0 -= b[j] * a0avg[j];
    /* Green-Gauss gradient of the sub-stencil */
    double gg[3] = {0, 0, 0};
    for (int m = 0; m < nf; ++m)
      for (int d = 0; d < 3; ++d) gg[d] += 0.5 * (st.Qn[m][q] + Q0) * st.Sn[m][d];
    for (int d = 0; d < 3; ++d) gg[d] = al * gg[d] / V;
    /* least-squares gradient */
    double r3[ORC_MAXNF], gl[3];
    for (int m = 0; m < nf; ++m) r3[m] = dQ[m];
    orc_qr_qt(&qd, r3);
    for (int r = 2; r >= 0; --r) {
      double s = r3[r];
      for (int k = r + 1; k < 3; ++k) s -= qd.R[r * 3 + k] * gl[k];
      gl[r] = s / qd.R[r * 3 + r];
    }
    /* smoothness indicators */
    double bGG = V23 * (gg[0] * gg[0] + gg[1] * gg[1] + gg[2] * gg[2]);
    double bLS = V23 * (gl[0] * gl[0] + gl[1] * gl[1] + gl[2] * gl[2]);
    double beta1 = bGG < bLS ? bGG : bLS;
    double lin[3][4] = {{b[0], 2.0 * b[3], b[6], b[8]}, {b[1], b[6], 2.0 * b[4], b[7]}, {b[2], b[8], b[7], 2.0 * b[5]}};
    double Mm[3][3] = {{m0[0], m0[3], m0[5]}, {m0[3], m0[1], m0[4]}, {m0[5], m0[4], m0[2]}};
    double first = 0.0;
    for (int d = 0; d < 3; ++d) {
      double vMv = 0.0;
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) vMv += lin[d][1 + r] * Mm[r][c] * lin[d][1 + c];
      first += V * (lin[d][0] * lin[d][0] + vMv);
    }
    double second = V * (4.0 * b[3] * b[3] + 4.0 * b[4] * b[4] + 4.0 * b[5] * b[5] + b[6] * b[6] + b[7] * b[7] + b[8] * b[8]);
    double beta2 = Vm13 * first + V13 * second;
    double den = Q0 * Q0 + beta1 + 1e-40;
    double bt1 = beta1 / den, bt2 = beta2 / den;
    double sig = fabs(bt2 - bt1);
    double w1 = g1 * (1.0 + (sig / (eps + bt1)) * (sig / (eps + bt1)));
    double w2 = g2 * (1.0 + (sig / (eps + bt2)) * (sig / (eps + bt2)));
    double ws = w1 + w2;
    w1 /= ws;
    w2 /= ws;
    /* R = w2 P2 + w1 P1 with P2 = p2/g2 - (g1/g2) p1, P1 = p1 */
    double c2 = w2 / g2, c1 = w1 - w2 * g1 / g2;
    if (mode == 1) { /* p^2 alone */
      c2 = 1.0;
      c1 = 0.0;
    } else if (mode == 2) { /* p^1 alone */
      c2 = 0.0;
      c1 = 1.0;
    }
    rc[q][0] = c2 * a0 + c1 * Q0;
    for (int d = 0; d < 3; ++d) rc[q][1 + d] = c2 * b[d] + c1 * gg[d];
    for (int j = 3; j < 9; ++j) rc[q][1 + j] = c2 * b[j];
  }
  return 0;
}

static int reconstruct_cell(const orc_solver* S, const double* W, const double* G, const double* alpha_prev,
                            int64_t i, double rc[5][10]) {
  return reconstruct_cell_mode(S, W, G, alpha_prev, i, rc, 0);
}

/* value and gradient of a reconstruction polynomial at offset X from the cell centroid */
static void eval_poly(const double rc[5][10], const double X[3], double Wv[5], double Gv[15]) {
  for (int q = 0; q < 5; ++q) {
    const double* r = rc[q];
    Wv[q] = r[0] + r[1] * X[0] + r[2] * X[1] + r[3] * X[2] + r[4] * X[0] * X[0] + r[5] * X[1] * X[1] +
            r[6] * X[2] * X[2] + r[7] * X[0] * X[1] + r[8] * X[1] * X[2] + r[9] * X[0] * X[2];
    Gv[3 * q + 0] = r[1] + 2.0 * r[4] * X[0] + r[7] * X[1] + r[9] * X[2];
    Gv[3 * q + 1] = r[2] + 2.0 * r[5] * X[1] + r[7] * X[0] + r[8] * X[2];
    Gv[3 * q + 2] = r[3] + 2.0 * r[6] * X[2] + r[8] * X[1] + r[9] * X[0];
  }
}

/* ------------------------------------------------------------------------------------------- */
/* time steps                                                                                   */

static void local_dt_fine(const orc_solver* S, const double* W, double* dt) {
  const orc_mesh* M = S->M;
  const double g = S->P.gamma;
  for (int64_t i = 0; i < M->nc; ++i) {
    const double* w = W + 5 * i;
    double rho = w[0], u[3] = {w[1] / rho, w[2] / rho, w[3] / rho};
    double p = (g - 1.0) * (w[4] - 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
    double c = sqrt(g * p / rho), nu = S->P.viscous ? orc_viscosity(&S->ph, g * p / rho) / rho : 0.0;
    double sum = 0.0, V = M->vol[i];
    for (int m = 0; m < orc_nfaces(M->ctype[i]); ++m) {
      int64_t f = M->cf[6 * i + m];
      double Sn[3], area, xc[3];
      face_sum(M, f, Sn, &area, xc);
      double nn = sqrt(Sn[0] * Sn[0] + Sn[1] * Sn[1] + Sn[2] * Sn[2]);
      double un = fabs((u[0] * Sn[0] + u[1] * Sn[1] + u[2] * Sn[2]) / nn);
      sum += area * (un + c + 2.0 * nu * area / V);
    }
    dt[i] = S->P.cfl_fine * V / sum;
  }
  if (S->P.dt_mode == 1) {
    double mn = dt[0];
    for (int64_t i = 1; i < M->nc; ++i) mn = dt[i] < mn ? dt[i] : mn;
    for (int64_t i = 0; i < M->nc; ++i) dt[i] = mn;
  }
}

static void local_dt_level(const orc_solver* S, const orc_level* L, const double* W, double* dt) {
  const double g = S->P.gamma;
  for (int64_t i = 0; i < L->nc; ++i) {
    const double* w = W + 5 * i;
    double rho = w[0], u[3] = {w[1] / rho, w[2] / rho, w[3] / rho};
    double p = (g - 1.0) * (w[4] - 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
    double c = sqrt(g * p / rho), sum = 0.0;
    for (int32_t k = L->c2f_ptr[i]; k < L->c2f_ptr[i + 1]; ++k) {
      int32_t f = L->c2f[k];
      const double* Sn = L->Sn + 3 * f;
      double nn = sqrt(Sn[0] * Sn[0] + Sn[1] * Sn[1] + Sn[2] * Sn[2]);
      /* the face's area is the sum of its fine faces' areas; its direction that of the summed
         area vector (none when that vector cancels) */
      double un = nn > 0.0 ? fabs((u[0] * Sn[0] + u[1] * Sn[1] + u[2] * Sn[2]) / nn) : 0.0;
      sum += L->area[f] * (un + c);
    }
    dt[i] = S->P.cfl_coarse * L->vol[i] / sum;
  }
  if (S->P.dt_mode == 1) {
    double mn = dt[0];
    for (int64_t i = 1; i < L->nc; ++i) mn = dt[i] < mn ? dt[i] : mn;
    for (int64_t i = 0; i < L->nc; ++i) dt[i] = mn;
  }
}

/* ------------------------------------------------------------------------------------------- */
/* residuals                                                                                    */

/* magnitudes of the terms the last fine residual summed: per cell and component, the sum over its
   Gauss points of |weight x flux| and of |weight x interface state| / |Omega| (the scales of the
   residual and of the Gauss-Green gradient sums; used by tests as rounding-error denominators) */
static double* g_last_fabs = NULL;
static double* g_last_gabs = NULL;
static int64_t g_last_n = 0;

/* fine CGKS residual: Res [nc][5], new gradients (already scaled by the compression factor) and
   the compression factor; any output may be NULL */
int orc_residual_fine(orc_solver* S, const double* W, const double* G, const double* alpha_prev, double* Res,
                      double* Gnew, double* anew, double* dt_out) {
  const orc_mesh* M = S->M;
  const int64_t nc = M->nc;
  int rc_ = 0;
  double* rc = malloc(sizeof(double) * 50 * nc);
  double* dt = malloc(sizeof(double) * nc);
  double* res = calloc(5 * nc, sizeof(double));
  double* gs = calloc(15 * nc, sizeof(double));
  double* al = malloc(sizeof(double) * nc);
  double *gpF = NULL, *gpW = NULL, *gpa = NULL;
  for (int64_t i = 0; i < nc; ++i) al[i] = 1.0;
  local_dt_fine(S, W, dt);
  /* per-cell reconstruction and per-Gauss-point fluxes are independent (OpenMP); the sums into the
     cells below run sequentially in ascending face order */
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(| : bad)
  for (int64_t i = 0; i < nc; ++i)
    if (reconstruct_cell(S, W, G, alpha_prev, i, (double(*)[10])(rc + 50 * i))) bad |= 1;
  if (bad) {
    rc_ = -1;
    goto out;
  }
  gpF = malloc(sizeof(double) * 20 * M->nf);  /* [nf][4][5] flux */
  gpW = malloc(sizeof(double) * 20 * M->nf);  /* [nf][4][5] state at dt */
  gpa = malloc(sizeof(double) * 4 * M->nf);   /* [nf][4] compression factor */
#pragma omp parallel for schedule(dynamic, 64) reduction(| : bad)
  for (int64_t f = 0; f < M->nf; ++f) {
    int64_t L = M->fL[f], R = M->fR[f];
    for (int k = 0; k < M->fngp[f]; ++k) {
      const double* x = M->gx + 12 * f + 3 * k;
      const double* dA = M->gA + 12 * f + 3 * k;
      double w = sqrt(dA[0] * dA[0] + dA[1] * dA[1] + dA[2] * dA[2]);
      double n[3] = {dA[0] / w, dA[1] / w, dA[2] / w};
      double XL[3], WL[5], GL[15], WR[5], GR[15];
      for (int d = 0; d < 3; ++d) XL[d] = x[d] - M->ctr[3 * L + d];
      eval_poly((const double(*)[10])(rc + 50 * L), XL, WL, GL);
      double dtf, ak = 1.0;
      if (R >= 0) {
        double XR[3];
        for (int d = 0; d < 3; ++d) XR[d] = x[d] - M->shift[3 * f + d] - M->ctr[3 * R + d];
        eval_poly((const double(*)[10])(rc + 50 * R), XR, WR, GR);
        dtf = dt[L] < dt[R] ? dt[L] : dt[R];
        ak = S->P.compression_factor ? orc_cf_alpha(&S->ph, WL, WR, n) : 1.0;
      } else {
        if (orc_bc_ghost(&S->ph, M->ftag[f], n, WL, GL, WR, GR)) bad |= 1;
        dtf = dt[L];
      }
      if (orc_gks_point(&S->ph, WL, GL, WR, GR, n, dtf, gpF + 20 * f + 5 * k, gpW + 20 * f + 5 * k)) bad |= 1;
      gpa[4 * f + k] = ak;
    }
  }
  if (bad) {
    rc_ = -1;
    goto out;
  }
  if (g_last_n != nc) {
    free(g_last_fabs);
    free(g_last_gabs);
    g_last_fabs = malloc(sizeof(double) * 5 * nc);
    g_last_gabs = malloc(sizeof(double) * 5 * nc);
    g_last_n = nc;
  }
  memset(g_last_fabs, 0, sizeof(double) * 5 * nc);
  memset(g_last_gabs, 0, sizeof(double) * 5 * nc);
  for (int64_t f = 0; f < M->nf; ++f) {
    int64_t L = M->fL[f], R = M->fR[f];
    for (int k = 0; k < M->fngp[f]; ++k) {
      const double* dA = M->gA + 12 * f + 3 * k;
      const double* F = gpF + 20 * f + 5 * k;
      const double* Wt = gpW + 20 * f + 5 * k;
      double w = sqrt(dA[0] * dA[0] + dA[1] * dA[1] + dA[2] * dA[2]);
      for (int q = 0; q < 5; ++q) {
        res[5 * L + q] -= w * F[q];
        for (int d = 0; d < 3; ++d) gs[15 * L + 3 * q + d] += Wt[q] * dA[d];
        g_last_fabs[5 * L + q] += fabs(w * F[q]);
        g_last_gabs[5 * L + q] += fabs(w * Wt[q]) / M->vol[L];
      }
      al[L] *= gpa[4 * f + k];
      if (R >= 0) {
        for (int q = 0; q < 5; ++q) {
          res[5 * R + q] += w * F[q];
          for (int d = 0; d < 3; ++d) gs[15 * R + 3 * q + d] -= Wt[q] * dA[d];
          g_last_fabs[5 * R + q] += fabs(w * F[q]);
          g_last_gabs[5 * R + q] += fabs(w * Wt[q]) / M->vol[R];
        }
        al[R] *= gpa[4 * f + k];
      }
    }
  }
  if (Res) memcpy(Res, res, sizeof(double) * 5 * nc);
  if (Gnew)
    for (int64_t i = 0; i < nc; ++i)
      for (int j = 0; j < 15; ++j) Gnew[15 * i + j] = al[i] * gs[15 * i + j] / M->vol[i];
  if (anew) memcpy(anew, al, sizeof(double) * nc);
  if (dt_out) memcpy(dt_out, dt, sizeof(double) * nc);
out:
  free(rc);
  free(dt);
  free(res);
  free(gs);
  free(al);
  free(gpF);
  free(gpW);
  free(gpa);
  return rc_;
}

/* first-order KFVS residual of one level */
int orc_residual_kfvs(orc_solver* S, int lev, const double* W, double* Res) {
  const orc_level* L = &S->M->lev[lev];
  memset(Res, 0, sizeof(double) * 5 * L->nc);
  for (int64_t f = 0; f < L->nf; ++f) {
    const double* Sn = L->Sn + 3 * f;
    double s = sqrt(Sn[0] * Sn[0] + Sn[1] * Sn[1] + Sn[2] * Sn[2]);
    /* an agglomerate wrapping around its neighbour can leave a coarse face whose summed area
       vector is exactly zero: no net area, no flux, and no normal to evaluate one with */
    if (s == 0.0) continue;
    double n[3] = {Sn[0] / s, Sn[1] / s, Sn[2] / s}, F[5], Wg[5];
    int32_t a = L->fL[f], b = L->fR[f];
    if (b >= 0) {
      if (orc_kfvs_point(&S->ph, W + 5 * a, W + 5 * b, n, F)) return -1;
    } else {
      if (orc_bc_ghost(&S->ph, L->ftag[f], n, W + 5 * a, NULL, Wg, NULL)) return -1;
      if (orc_kfvs_point(&S->ph, W + 5 * a, Wg, n, F)) return -1;
    }
    for (int q = 0; q < 5; ++q) {
      Res[5 * a + q] -= s * F[q];
      if (b >= 0) Res[5 * b + q] += s * F[q];
    }
  }
  return 0;
}

static double density_norm(const double* Res, const double* vol, int64_t n) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double r = Res[5 * i] / vol[i];
    s += r * r;
  }
  return sqrt(s / (double)n);
}

static int physical(const double w[5], double g) {
  if (!(w[0] > 0.0)) return 0;
  double p = (g - 1.0) * (w[4] - 0.5 * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]) / w[0]);
  return p > 0.0;
}

/* coarse forward-Euler update W += dt/V (R + F); like the correction, an update that would make rho
   or p non-positive in a cell is skipped for that cell (counted) */
static int coarse_update(orc_solver* S, const orc_level* L, double* Wk, const double* R, const double* F,
                         const double* dt) {
  for (int64_t i = 0; i < L->nc; ++i) {
    double w[5];
    for (int q = 0; q < 5; ++q) w[q] = Wk[5 * i + q] + dt[i] / L->vol[i] * (R[5 * i + q] + F[5 * i + q]);
    for (int q = 0; q < 5; ++q)
      if (!isfinite(w[q])) return -1;
    if (physical(w, S->P.gamma))
      memcpy(Wk + 5 * i, w, sizeof(w));
    else
      S->skipped_corrections++;
  }
  return 0;
}

/* W_i += r c_i on the receiving level L: c_i the injected correction Wc - Wc0 of the coarse cell of
   i (prolongation 0), or the volume-weighted mean of the injected corrections of i and its face
   neighbours, in ascending face order (prolongation 1); skipped where rho or p would not stay
   positive (counted) */
static void prolong_correction(orc_solver* S, const orc_level* L, const int32_t* f2c, const double* Wc,
                               const double* Wc0, double* Wf) {
  const double r = S->P.correction_relax;
  for (int64_t i = 0; i < L->nc; ++i) {
    double c[5], w[5];
    int32_t k = f2c[i];
    for (int q = 0; q < 5; ++q) c[q] = Wc[5 * k + q] - Wc0[5 * k + q];
    if (S->P.prolongation == 1) {
      double sv = L->vol[i];
      for (int q = 0; q < 5; ++q) c[q] *= L->vol[i];
      for (int32_t e = L->c2f_ptr[i]; e < L->c2f_ptr[i + 1]; ++e) {
        int32_t f = L->c2f[e], a = L->fL[f], b = L->fR[f];
        if (b < 0 || a == b) continue;
        int64_t j = a == i ? b : a;
        int32_t kj = f2c[j];
        for (int q = 0; q < 5; ++q) c[q] += L->vol[j] * (Wc[5 * kj + q] - Wc0[5 * kj + q]);
        sv += L->vol[j];
      }
      for (int q = 0; q < 5; ++q) c[q] /= sv;
    }
    for (int q = 0; q < 5; ++q) w[q] = Wf[5 * i + q] + r * c[q];
    if (physical(w, S->P.gamma))
      memcpy(Wf + 5 * i, w, sizeof(w));
    else
      S->skipped_corrections++;
  }
}

/* one coarse smoothing step on level l: forward Euler, or LU-SGS on the defect R + F (Sec. 4.3) */
static int coarse_smooth(orc_solver* S, int l, double* Wk, const double* R, const double* F, const double* dt) {
  const orc_level* L = &S->M->lev[l];
  if (S->P.coarse_smoother != 1) return coarse_update(S, L, Wk, R, F, dt);
  if (!S->colors[l]) {
    S->colors[l] = malloc(sizeof(int32_t) * (L->nc ? L->nc : 1));
    S->ncolors[l] = orc_level_colors(L, S->colors[l]);
  }
  double* rhs = malloc(sizeof(double) * 5 * (L->nc ? L->nc : 1));
  for (int64_t j = 0; j < 5 * L->nc; ++j) rhs[j] = R[j] + F[j];
  int rc = orc_lusgs_step(&S->P, L, S->colors[l], S->ncolors[l], Wk, rhs, dt, &S->skipped_corrections);
  free(rhs);
  return rc;
}

/* one explicit fine step (the fine-level smoother, Eq. smo) */
static int fine_step(orc_solver* S, double* norm) {
  const orc_mesh* M = S->M;
  const int64_t nc = M->nc;
  double* res = malloc(sizeof(double) * 5 * nc);
  double* gn = malloc(sizeof(double) * 15 * nc);
  double* an = malloc(sizeof(double) * nc);
  double* dt = malloc(sizeof(double) * nc);
  int rc = orc_residual_fine(S, S->W, S->G, S->alpha, res, gn, an, dt);
  if (!rc) {
    for (int64_t i = 0; i < nc; ++i)
      for (int q = 0; q < 5; ++q) S->W[5 * i + q] += dt[i] / M->vol[i] * res[5 * i + q];
    memcpy(S->G, gn, sizeof(double) * 15 * nc);
    memcpy(S->alpha, an, sizeof(double) * nc);
    if (norm) *norm = density_norm(res, M->vol, nc);
    for (int64_t i = 0; i < nc; ++i)
      if (!physical(S->W + 5 * i, S->P.gamma)) {
        rc = -3;
        break;
      }
  }
  free(res);
  free(gn);
  free(an);
  free(dt);
  return rc;
}

/* coarse-level FAS smoothing with forcing F (Sec. 4.2), recursing to the next level */
static int coarse_cycle(orc_solver* S, int l, double* Wk, const double* Rstar) {
  const orc_level* L = &S->M->lev[l];
  const int64_t n = L->nc;
  int rc = 0;
  double* F = malloc(sizeof(double) * 5 * n);
  double* R = malloc(sizeof(double) * 5 * n);
  double* dt = malloc(sizeof(double) * n);
  double* W0 = malloc(sizeof(double) * 5 * n);
  memcpy(W0, Wk, sizeof(double) * 5 * n);
  if ((rc = orc_residual_kfvs(S, l, Wk, R))) goto out;
  for (int64_t j = 0; j < 5 * n; ++j) F[j] = Rstar[j] - R[j];
  for (int s = 0; s < S->P.coarse_steps; ++s) {
    if ((rc = orc_residual_kfvs(S, l, Wk, R))) goto out;
    local_dt_level(S, L, Wk, dt);
    if ((rc = coarse_smooth(S, l, Wk, R, F, dt))) goto out;
  }
  if (l + 1 < S->M->n_levels) {
    const orc_level* C = &S->M->lev[l + 1];
    const int64_t m = C->nc;
    double* Wc = calloc(5 * m, sizeof(double));
    double* Rc = calloc(5 * m, sizeof(double));
    double* Wc0 = malloc(sizeof(double) * 5 * m);
    if ((rc = orc_residual_kfvs(S, l, Wk, R))) {
      free(Wc);
      free(Rc);
      free(Wc0);
      goto out;
    }
    for (int64_t i = 0; i < n; ++i) {
      int32_t c = C->fine2coarse[i];
      for (int q = 0; q < 5; ++q) {
        Wc[5 * c + q] += L->vol[i] * Wk[5 * i + q];
        Rc[5 * c + q] += R[5 * i + q] + F[5 * i + q];
      }
    }
    for (int64_t c = 0; c < m; ++c)
      for (int q = 0; q < 5; ++q) Wc[5 * c + q] /= C->vol[c];
    memcpy(Wc0, Wc, sizeof(double) * 5 * m);
    rc = coarse_cycle(S, l + 1, Wc, Rc);
    if (!rc) prolong_correction(S, L, C->fine2coarse, Wc, Wc0, Wk);
    free(Wc);
    free(Rc);
    free(Wc0);
    if (rc) goto out;
    for (int s = 0; s < S->P.post; ++s) {
      if ((rc = orc_residual_kfvs(S, l, Wk, R))) goto out;
      local_dt_level(S, L, Wk, dt);
      if ((rc = coarse_smooth(S, l, Wk, R, F, dt))) goto out;
    }
  }
out:
  free(F);
  free(R);
  free(dt);
  free(W0);
  return rc;
}

/* one V-cycle (Sec. 4.2): pre-smoothing CGKS step(s), defect at W^{n+1}, coarse FAS levels,
   injection correction of W, optional post-smoothing */
static int vcycle(orc_solver* S, double* norm) {
  const orc_mesh* M = S->M;
  int rc = 0;
  for (int s = 0; s < (S->P.pre > 0 ? S->P.pre : 1); ++s) {
    double nm;
    if ((rc = fine_step(S, &nm))) return rc;
    if (s == 0 && norm) *norm = nm;
  }
  if (M->n_levels <= 1) return 0;
  const int64_t nc = M->nc;
  const orc_level* C = &M->lev[1];
  const int64_t m = C->nc;
  double* res = malloc(sizeof(double) * 5 * nc);
  double* Wc = calloc(5 * m, sizeof(double));
  double* Rc = calloc(5 * m, sizeof(double));
  double* Wc0 = malloc(sizeof(double) * 5 * m);
  if ((rc = orc_residual_fine(S, S->W, S->G, S->alpha, res, NULL, NULL, NULL))) goto out;
  for (int64_t i = 0; i < nc; ++i) {
    int32_t c = C->fine2coarse[i];
    for (int q = 0; q < 5; ++q) {
      Wc[5 * c + q] += M->cvol[i] * S->W[5 * i + q];
      Rc[5 * c + q] += res[5 * i + q];
    }
  }
  for (int64_t c = 0; c < m; ++c)
    for (int q = 0; q < 5; ++q) Wc[5 * c + q] /= C->vol[c];
  memcpy(Wc0, Wc, sizeof(double) * 5 * m);
  if ((rc = coarse_cycle(S, 1, Wc, Rc))) goto out;
  prolong_correction(S, &M->lev[0], C->fine2coarse, Wc, Wc0, S->W);
  for (int s = 0; s < S->P.post; ++s)
    if ((rc = fine_step(S, NULL))) goto out;
out:
  free(res);
  free(Wc);
  free(Rc);
  free(Wc0);
  return rc;
}

/* ------------------------------------------------------------------------------------------- */
/* solver object                                                                                */

orc_solver* orc_solver_new(orc_mesh* M, const orc_params* P, char* err) {
  orc_solver* S = calloc(1, sizeof(orc_solver));
  S->M = M;
  S->P = *P;
  const double g = P->gamma;
  S->ph.gamma = g;
  S->ph.K = (5.0 - 3.0 * g) / (g - 1.0);
  S->ph.prandtl = P->prandtl;
  S->ph.eps_inviscid = P->eps_inviscid;
  S->ph.c_press = P->c_press;
  S->ph.viscous = P->viscous;
  double a = P->aoa[0] * M_PI / 180.0, b = P->aoa[1] * M_PI / 180.0;
  double u[3] = {P->mach * cos(a) * cos(b), P->mach * sin(b), P->mach * sin(a) * cos(b)};
  double rho = 1.0, p = 1.0 / g;
  S->ph.Winf[0] = rho;
  for (int d = 0; d < 3; ++d) S->ph.Winf[1 + d] = rho * u[d];
  S->ph.Winf[4] = p / (g - 1.0) + 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  S->ph.mu = P->viscous ? rho * P->mach * 1.0 / P->reynolds : 0.0;
  S->ph.sutherland = P->sutherland;
  S->W = calloc(5 * M->nc, sizeof(double));
  S->G = calloc(15 * M->nc, sizeof(double));
  S->alpha = malloc(sizeof(double) * M->nc);
  for (int64_t i = 0; i < M->nc; ++i) S->alpha[i] = 1.0;
  if (orc_build_levels(M, P, err)) {
    free(S->W);
    free(S->G);
    free(S->alpha);
    free(S);
    return NULL;
  }
  return S;
}

const orc_params* orc_solver_params(const orc_solver* S) { return &S->P; }

void orc_solver_delete(orc_solver* S) {
  if (!S) return;
  free(S->W);
  free(S->G);
  free(S->alpha);
  for (int l = 0; l < 8; ++l) free(S->colors[l]);
  free(S);
}

int orc_solver_run(orc_solver* S, int multigrid, int n, double* hist) {
  for (int it = 0; it < n; ++it) {
    double nm = 0.0;
    int rc = multigrid ? vcycle(S, &nm) : fine_step(S, &nm);
    if (rc) return rc;
    if (S->iters == 0) S->r1 = nm;
    S->iters++;
    if (hist) hist[it] = nm;
  }
  return 0;
}

/* the fine-level reconstruction coefficients of every cell ([nc][5][10]); mode 0: R, 1: p^2, 2: p^1 */
int orc_solver_reconstruct(orc_solver* S, double* rc, int mode) {
  for (int64_t i = 0; i < S->M->nc; ++i)
    if (reconstruct_cell_mode(S, S->W, S->G, S->alpha, i, (double(*)[10])(rc + 50 * i), mode)) return -1;
  return 0;
}

void orc_solver_dt(orc_solver* S, double* dt) { local_dt_fine(S, S->W, dt); }
void orc_solver_dt_level(orc_solver* S, int l, const double* W, double* dt) {
  local_dt_level(S, &S->M->lev[l], W, dt);
}
double* orc_solver_W(orc_solver* S) { return S->W; }
double* orc_solver_G(orc_solver* S) { return S->G; }
double* orc_solver_alpha(orc_solver* S) { return S->alpha; }
int64_t orc_solver_skipped(orc_solver* S) { return S->skipped_corrections; }

/* the term magnitudes of the last fine residual, component-major [5][nc] each (nullable) */
int orc_solver_term_scales(orc_solver* S, double* fabs_out, double* gabs_out) {
  const int64_t nc = S->M->nc;
  if (g_last_n != nc || !g_last_fabs) return -1;
  for (int64_t i = 0; i < nc; ++i)
    for (int q = 0; q < 5; ++q) {
      if (fabs_out) fabs_out[q * nc + i] = g_last_fabs[5 * i + q];
      if (gabs_out) gabs_out[q * nc + i] = g_last_gabs[5 * i + q];
    }
  return 0;
}
