/* Oracle: the implicit coarse-level smoother of Sec. 4.3 (backward Euler, first-order Lax-Friedrichs
 * Jacobian splitting, matrix-free symmetric Gauss-Seidel: "LU-SGS").  TEST INFRASTRUCTURE ONLY.
 *
 * One step on a coarse level solves, for the increments dU of all cells,
 *   (|Omega_i|/dt_i + 1/2 sum_p lambda_p S_p) dU_i
 *       + sum_p 1/2 [F_n(U_p + dU_p) - F_n(U_p) - lambda_p dU_p] S_p = Res_i + F_i
 * (the paper's final implicit form, with the FAS forcing F_i on the right), n the unit normal of
 * face p pointing out of cell i, F_n the Euler flux through it, lambda_p = max(|U.n| + c) of the two
 * cells (Sec. 4.3 adds 2 mu S/|Omega|; the coarse levels are inviscid KFVS levels), and S_p the
 * length of the face's summed area vector.  The relaxation is one forward and one backward
 * Gauss-Seidel sweep in a fixed cell order.  Readings:
 *  - the order is by colour, then cell id: colours from Jones-Plassmann rounds (an uncoloured cell
 *    whose priority (splitmix64(id), id) exceeds that of every uncoloured neighbour takes the
 *    smallest colour no coloured neighbour has), so cells of one colour share no face and one
 *    colour can be relaxed at once;
 *  - boundary neighbours (ghost cells) keep dU = 0; their face counts in the diagonal with the
 *    cell's own lambda;
 *  - faces whose summed area vector cancels, and a cell's periodic face with itself, are skipped;
 *  - an increment that would make rho or p non-positive is not applied to that cell (counted).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "orc.h"

uint64_t orc_splitmix64(uint64_t x);

static int other_cell(const orc_level* L, int32_t f, int64_t i) {
  int32_t a = L->fL[f], b = L->fR[f];
  if (b < 0 || a == b) return -1;
  return a == i ? b : a;
}

static int higher_priority(uint64_t pj, int64_t j, uint64_t pi, int64_t i) {
  return pj > pi || (pj == pi && j > i);
}

int orc_level_colors(const orc_level* L, int32_t* color) {
  const int64_t n = L->nc;
  uint64_t* prio = malloc(sizeof(uint64_t) * (n ? n : 1));
  char* sel = malloc(n ? n : 1);
  for (int64_t i = 0; i < n; ++i) {
    prio[i] = orc_splitmix64((uint64_t)i);
    color[i] = -1;
  }
  int64_t left = n;
  int ncol = 0;
  while (left > 0) {
    /* selection on the colouring at the start of the round */
    for (int64_t i = 0; i < n; ++i) {
      sel[i] = 0;
      if (color[i] >= 0) continue;
      int top = 1;
      for (int32_t k = L->c2f_ptr[i]; k < L->c2f_ptr[i + 1] && top; ++k) {
        int j = other_cell(L, L->c2f[k], i);
        if (j >= 0 && color[j] < 0 && higher_priority(prio[j], j, prio[i], i)) top = 0;
      }
      sel[i] = (char)top;
    }
    for (int64_t i = 0; i < n; ++i) {
      if (!sel[i]) continue;
      for (int c = 0;; ++c) {
        int used = 0;
        for (int32_t k = L->c2f_ptr[i]; k < L->c2f_ptr[i + 1] && !used; ++k) {
          int j = other_cell(L, L->c2f[k], i);
          if (j >= 0 && color[j] == c) used = 1;
        }
        if (!used) {
          color[i] = c;
          if (c + 1 > ncol) ncol = c + 1;
          break;
        }
      }
      --left;
    }
  }
  free(prio);
  free(sel);
  return ncol;
}

/* Euler flux through a face with unit normal n */
static void euler_flux_n(const double W[5], const double n[3], double g, double F[5]) {
  double rho = W[0], u[3] = {W[1] / rho, W[2] / rho, W[3] / rho};
  double p = (g - 1.0) * (W[4] - 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
  double un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
  F[0] = rho * un;
  for (int d = 0; d < 3; ++d) F[1 + d] = W[1 + d] * un + p * n[d];
  F[4] = (W[4] + p) * un;
}

static double wave_speed(const double W[5], const double n[3], double g) {
  double rho = W[0], u[3] = {W[1] / rho, W[2] / rho, W[3] / rho};
  double p = (g - 1.0) * (W[4] - 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
  return fabs(u[0] * n[0] + u[1] * n[1] + u[2] * n[2]) + sqrt(g * p / rho);
}

/* 1/2 [F_n(U_j + dU_j) - F_n(U_j) - lambda dU_j] S with n out of cell i */
static void offdiag(const double* Wj, const double* dUj, const double n[3], double lam, double S, double g,
                    double out[5]) {
  double Wp[5], Fp[5], F0[5];
  for (int q = 0; q < 5; ++q) Wp[q] = Wj[q] + dUj[q];
  euler_flux_n(Wp, n, g, Fp);
  euler_flux_n(Wj, n, g, F0);
  for (int q = 0; q < 5; ++q) out[q] = 0.5 * ((Fp[q] - F0[q]) - lam * dUj[q]) * S;
}

static int physical_state(const double w[5], double g) {
  if (!(w[0] > 0.0)) return 0;
  double p = (g - 1.0) * (w[4] - 0.5 * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]) / w[0]);
  return p > 0.0;
}

int orc_lusgs_step(const orc_params* P, const orc_level* L, const int32_t* color, int ncol, double* W,
                   const double* RHS, const double* dt, int64_t* skipped) {
  const int64_t n = L->nc, nf = L->nf;
  const double g = P->gamma;
  double* lam = malloc(sizeof(double) * (nf ? nf : 1));
  double* S = malloc(sizeof(double) * (nf ? nf : 1));
  double* nrm = malloc(sizeof(double) * 3 * (nf ? nf : 1));
  double* D = malloc(sizeof(double) * (n ? n : 1));
  double* dU = malloc(sizeof(double) * 5 * (n ? n : 1));
  int64_t* order = malloc(sizeof(int64_t) * (n ? n : 1));
  int rc = 0;
  /* per face: length of the summed area vector, its unit normal (out of L), lambda */
  for (int64_t f = 0; f < nf; ++f) {
    const double* Sn = L->Sn + 3 * f;
    S[f] = sqrt(Sn[0] * Sn[0] + Sn[1] * Sn[1] + Sn[2] * Sn[2]);
    lam[f] = 0.0;
    for (int d = 0; d < 3; ++d) nrm[3 * f + d] = S[f] > 0.0 ? Sn[d] / S[f] : 0.0;
    if (S[f] == 0.0) continue;
    int32_t a = L->fL[f], b = L->fR[f];
    double la = wave_speed(W + 5 * a, nrm + 3 * f, g);
    if (b >= 0) {
      double lb = wave_speed(W + 5 * b, nrm + 3 * f, g);
      lam[f] = la > lb ? la : lb;
    } else {
      lam[f] = la;
    }
  }
  /* diagonal */
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int32_t k = L->c2f_ptr[i]; k < L->c2f_ptr[i + 1]; ++k) {
      int32_t f = L->c2f[k];
      if (L->fL[f] == L->fR[f]) continue;
      s += lam[f] * S[f];
    }
    D[i] = L->vol[i] / dt[i] + 0.5 * s;
  }
  /* cell order: by colour, then id */
  {
    int64_t m = 0;
    for (int c = 0; c < ncol; ++c)
      for (int64_t i = 0; i < n; ++i)
        if (color[i] == c) order[m++] = i;
  }
  /* forward sweep: neighbours earlier in the order (lower colour) already hold dU* */
  for (int64_t o = 0; o < n; ++o) {
    int64_t i = order[o];
    double acc[5];
    for (int q = 0; q < 5; ++q) acc[q] = RHS[5 * i + q];
    for (int32_t k = L->c2f_ptr[i]; k < L->c2f_ptr[i + 1]; ++k) {
      int32_t f = L->c2f[k];
      int j = other_cell(L, f, i);
      if (j < 0 || S[f] == 0.0 || color[j] >= color[i]) continue;
      double sg = L->fL[f] == i ? 1.0 : -1.0, nn[3], t[5];
      for (int d = 0; d < 3; ++d) nn[d] = sg * nrm[3 * f + d];
      offdiag(W + 5 * j, dU + 5 * j, nn, lam[f], S[f], g, t);
      for (int q = 0; q < 5; ++q) acc[q] -= t[q];
    }
    for (int q = 0; q < 5; ++q) dU[5 * i + q] = acc[q] / D[i];
  }
  /* backward sweep: neighbours later in the order (higher colour) already hold the final dU */
  for (int64_t o = n - 1; o >= 0; --o) {
    int64_t i = order[o];
    double acc[5] = {0, 0, 0, 0, 0};
    for (int32_t k = L->c2f_ptr[i]; k < L->c2f_ptr[i + 1]; ++k) {
      int32_t f = L->c2f[k];
      int j = other_cell(L, f, i);
      if (j < 0 || S[f] == 0.0 || color[j] <= color[i]) continue;
      double sg = L->fL[f] == i ? 1.0 : -1.0, nn[3], t[5];
      for (int d = 0; d < 3; ++d) nn[d] = sg * nrm[3 * f + d];
      offdiag(W + 5 * j, dU + 5 * j, nn, lam[f], S[f], g, t);
      for (int q = 0; q < 5; ++q) acc[q] += t[q];
    }
    for (int q = 0; q < 5; ++q) dU[5 * i + q] -= acc[q] / D[i];
  }
  /* apply */
  for (int64_t i = 0; i < n && !rc; ++i) {
    double w[5];
    for (int q = 0; q < 5; ++q) {
      w[q] = W[5 * i + q] + dU[5 * i + q];
      if (!isfinite(w[q])) rc = -1;
    }
    if (rc) break;
    if (physical_state(w, g))
      memcpy(W + 5 * i, w, sizeof(w));
    else
      ++*skipped;
  }
  free(lam);
  free(S);
  free(nrm);
  free(D);
  free(dU);
  free(order);
  return rc;
}
