// Bodies of the adjoint's transposed-product kernels, per Gauss point and per cell (host+device, so
// that their arithmetic can be exercised without a device); adjoint.cu wraps them in kernels.
#pragma once
#include "fine.cuh"

// point cotangents are one record per Gauss point (41 values padded to 42 doubles, 336 bytes: the
// per-cell kernel gathers its faces' points, so each reads 21 contiguous 16-byte pairs instead of 41
// scattered words); neighbour records are one 20-double record per face side
#define CGKS_PB 42

struct VjpArgs {
  int64_t nc, nf, ngp;
  const int8_t *ctype, *cside;
  const int32_t *cf, *fL, *fR, *gp_face, *gp_ptr;
  const double *gp_x, *gp_A, *fshift, *ctr, *vol, *dt, *Jp, *Jr;
  const double *rbar, *gbar;  // cotangents of Res [5][nc] and Gnew [15][nc]
  double *pbar, *self, *rec;  // [ngp][42] (41 used), [20][nc], [2 nf][20]
  double* cbuf;               // [51][nc]: cotangents of each cell's coefficients and time step
  double *out;                // [20][nc]: cotangents of (W, G)
};

// per Gauss point: cotangents of (flux, interface state) from those of (Res, Gnew) of its two cells,
// times Jp^T -> cotangents of the point inputs
HD void vjp_point_body(int64_t g, const VjpArgs& a) {
  const int64_t ngp = a.ngp, nc = a.nc;
  const int64_t f = a.gp_face[g], L = a.fL[f], R = a.fR[f];
  const double A[3] = {a.gp_A[g], a.gp_A[ngp + g], a.gp_A[2 * ngp + g]};
  // the left cell takes -flux and +A x state / |Omega|; the right cell the opposite
  double ub[10];
  const double rvL = 1.0 / a.vol[L], rvR = R >= 0 ? 1.0 / a.vol[R] : 0.0;
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    ub[q] = -a.rbar[q * nc + L] + (R >= 0 ? a.rbar[q * nc + R] : 0.0);
    double s = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d)
      s += A[d] * (a.gbar[(3 * q + d) * nc + L] * rvL - (R >= 0 ? a.gbar[(3 * q + d) * nc + R] * rvR : 0.0));
    ub[5 + q] = s;
  }
  for (int k = 0; k < CGKS_PJ_IN; ++k) {
    const double* J = a.Jp + (int64_t)(CGKS_PJ_OUT * k) * ngp + g;
    double s = 0.0;
#pragma unroll
    for (int o = 0; o < CGKS_PJ_OUT; ++o) s += J[(int64_t)o * ngp] * ub[o];
    a.pbar[(int64_t)g * CGKS_PB + k] = s;
  }
}

// phase 1, per cell: cotangents of its 50 coefficients and its time step from its faces' points (the
// transposed evaluation of the polynomial and its gradient) -> cbuf [51][nc]
HD void vjp_coef_body(int64_t i, const VjpArgs& a) {
  const int64_t nc = a.nc, nf = a.nf, ngp = a.ngp;
  const int nt = a.ctype[i] == 7 ? 5 : a.ctype[i];
  double cb[CGKS_RJ_OUT];
#pragma unroll
  for (int o = 0; o < CGKS_RJ_OUT; ++o) cb[o] = 0.0;
  for (int m = 0; m < nt; ++m) {
    const int64_t f = a.cf[(int64_t)m * nc + i];
    const int side = a.cside[(int64_t)m * nc + i];
    const int64_t L = a.fL[f], R = a.fR[f];
    const int base = side ? 20 : 0;
    // the face time step is the smaller of the two cells' (shared equally at a tie, as a central
    // difference of the minimum sees it)
    const double own = side ? a.dt[R] : a.dt[L], other = side ? a.dt[L] : a.dt[R];
    const double w_dt = R < 0 ? 1.0 : (own < other ? 1.0 : (own > other ? 0.0 : 0.5));
    for (int64_t g = a.gp_ptr[f]; g < a.gp_ptr[f + 1]; ++g) {
      double X[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) X[d] = a.gp_x[d * ngp + g] - (side ? a.fshift[d * nf + f] : 0.0) - a.ctr[d * nc + i];
      const double2* pb2 = reinterpret_cast<const double2*>(a.pbar + (int64_t)g * CGKS_PB + base);
      double pb[20];
#pragma unroll
      for (int k = 0; k < 10; ++k) {
        const double2 v = pb2[k];
        pb[2 * k] = v.x;
        pb[2 * k + 1] = v.y;
      }
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        const double w = pb[q], gx = pb[5 + 3 * q], gy = pb[6 + 3 * q], gz = pb[7 + 3 * q];
        // basis 1, X, Y, Z, X^2, Y^2, Z^2, XY, YZ, XZ and its gradient
        double* c = cb + 10 * q;
        c[0] += w;
        c[1] += w * X[0] + gx;
        c[2] += w * X[1] + gy;
        c[3] += w * X[2] + gz;
        c[4] += w * X[0] * X[0] + 2.0 * X[0] * gx;
        c[5] += w * X[1] * X[1] + 2.0 * X[1] * gy;
        c[6] += w * X[2] * X[2] + 2.0 * X[2] * gz;
        c[7] += w * X[0] * X[1] + X[1] * gx + X[0] * gy;
        c[8] += w * X[1] * X[2] + X[2] * gy + X[1] * gz;
        c[9] += w * X[0] * X[2] + X[2] * gx + X[0] * gz;
      }
      cb[CGKS_RC] += w_dt * a.pbar[(int64_t)g * CGKS_PB + 40];
    }
  }
#pragma unroll
  for (int o = 0; o < CGKS_RJ_OUT; ++o) a.cbuf[(int64_t)o * nc + i] = cb[o];
}

// phase 2, per cell and row group g with the cell's 51 cotangents cb[o * cs]:
//   g < 20   own-slot input c = g: self[c][i] = sum_o Jr[51 c + o][i] cb[o]
//   g >= 20  neighbour slot s = 1 + (g - 20) / 5, variable q = (g - 20) % 5: its 4 inputs (W_q and the
//            gradient of W_q) into the record of the slot's face for the cell across it (absent
//            slots and boundary faces write nothing)
HD void vjp_slot_body(int64_t i, int g, const VjpArgs& a, const double* cb, int cs) {
  const int64_t nc = a.nc;
  if (g < 20) {
    const double* J = a.Jr + (int64_t)(CGKS_RJ_OUT * g) * nc + i;
    double v = 0.0;
#pragma unroll
    for (int o = 0; o < CGKS_RJ_OUT; ++o) v += J[(int64_t)o * nc] * cb[o * cs];
    a.self[(int64_t)g * nc + i] = v;
    return;
  }
  const int s = 1 + (g - 20) / 5, q = (g - 20) % 5;
  const int nt = a.ctype[i] == 7 ? 5 : a.ctype[i];
  if (s > nt) return;
  const int64_t f = a.cf[(int64_t)(s - 1) * nc + i];
  if (a.fR[f] < 0) return;
  const int side = a.cside[(int64_t)(s - 1) * nc + i];
  double* rec = a.rec + (2 * f + side) * 20;
#pragma unroll
  for (int c4 = 0; c4 < 4; ++c4) {
    const double* J = a.Jr + (int64_t)(CGKS_RJ_SELF + ((s - 1) * 5 + q) * 40 + 10 * c4) * nc + i;
    double v = 0.0;
#pragma unroll
    for (int j = 0; j < 10; ++j) v += J[(int64_t)j * nc] * cb[(10 * q + j) * cs];
    rec[c4 == 0 ? q : 5 + 3 * q + (c4 - 1)] = v;
  }
}


// per cell: own part plus the records its neighbours wrote for it -> cotangents of its (W, G)
HD void vjp_cell_body(int64_t i, const VjpArgs& a) {
  const int64_t nc = a.nc;
  const int nt = a.ctype[i] == 7 ? 5 : a.ctype[i];
  double v[20];
#pragma unroll
  for (int c = 0; c < 20; ++c) v[c] = a.self[(int64_t)c * nc + i];
  for (int m = 0; m < nt; ++m) {
    const int64_t f = a.cf[(int64_t)m * nc + i];
    if (a.fR[f] < 0) continue;
    const int other = 1 - a.cside[(int64_t)m * nc + i];
    const double2* rec = reinterpret_cast<const double2*>(a.rec + (2 * f + other) * 20);
#pragma unroll
    for (int k = 0; k < 10; ++k) {
      const double2 r = rec[k];
      v[2 * k] += r.x;
      v[2 * k + 1] += r.y;
    }
  }
#pragma unroll
  for (int c = 0; c < 20; ++c) a.out[(int64_t)c * nc + i] = v[c];
}
