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


// per cell, the reconstruction's part of the transposed product recomputed from the state instead of
// read from the stored linearisation (adjoint_recompute 1).  cb (stride cs) holds the cotangents of
// the cell's 50 coefficients and of its time step; out: the cotangents of its own (W, grad W) ->
// self, and those of each interior neighbour's (W_q, grad W_q) -> the record of that face side.  The
// reverse mode of reconstruct_cell written out step by step: per variable the WENO combination of
// Sec. 3.4 (weights, smoothness indicators, the minimum in beta_1 taking the smaller branch and half
// of each at a tie, as the forward-mode linearisation does), then the linear maps of p^2 (Sec. 3.1),
// Green-Gauss and least squares; then the ghost states of boundary faces (a function of the cell's own
// W and grad W: their transposed Jacobian from forward-mode duals) and the local time step.
HD void vjp_recon_body(int64_t i, const ReconArgs& a, const VjpArgs& v, const double* cb, int64_t cs) {
  const int64_t nc = a.nc, nf = a.nf;
  const int nt = a.ctype[i] == 7 ? 5 : a.ctype[i];
  const Phys& ph = a.ph;
  double Q0[5], G0[15], self[20];
#pragma unroll
  for (int q = 0; q < 5; ++q) Q0[q] = a.W[q * nc + i];
#pragma unroll
  for (int j = 0; j < 15; ++j) G0[j] = a.G[j * nc + i];
#pragma unroll
  for (int c = 0; c < 20; ++c) self[c] = 0.0;
  // ghost states of boundary slots (primal) and their cotangents
  double gval[6][20], gcot[6][20];
  for (int m = 0; m < nt; ++m) {
    const int64_t f = a.cf[(int64_t)m * nc + i];
    for (int c = 0; c < 20; ++c) gcot[m][c] = 0.0;
    if (a.fR[f] < 0) {
      const double n[3] = {a.fnrm[f], a.fnrm[nf + f], a.fnrm[2 * nf + f]};
      bc_ghost<double>(a.ftag[f], n, Q0, G0, gval[m], gval[m] + 5, ph.gamma, ph.Winf);
    }
  }
  const double V23 = a.aux[i], V43 = a.aux[nc + i], al = a.alpha[i];
  double M2[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) M2[j] = a.aux[(2 + j) * nc + i];
  const double g1 = 0.5, g2 = 0.5;
  for (int q = 0; q < 5; ++q) {
    // stencil of variable q and the forward quantities
    double Qn[6], Gn[6][3], b[9], gg[3] = {0, 0, 0}, gl[3] = {0, 0, 0};
    for (int j = 0; j < 9; ++j) b[j] = 0.0;
    for (int m = 0; m < nt; ++m) {
      const int64_t f = a.cf[(int64_t)m * nc + i];
      if (a.fR[f] >= 0) {
        const int64_t nb = a.cside[(int64_t)m * nc + i] ? a.fL[f] : a.fR[f];
        Qn[m] = a.W[q * nc + nb];
        for (int e = 0; e < 3; ++e) Gn[m][e] = a.G[(3 * q + e) * nc + nb];
      } else {
        Qn[m] = gval[m][q];
        for (int e = 0; e < 3; ++e) Gn[m][e] = gval[m][5 + 3 * q + e];
      }
      const double dQ = Qn[m] - Q0[q];
      for (int j = 0; j < 9; ++j) {  // in the forward reconstruction's order
        b[j] += a.Kop[(j * 24 + m) * nc + i] * dQ;
        b[j] += a.Kop[(j * 24 + 6 + 3 * m) * nc + i] * Gn[m][0];
        b[j] += a.Kop[(j * 24 + 7 + 3 * m) * nc + i] * Gn[m][1];
        b[j] += a.Kop[(j * 24 + 8 + 3 * m) * nc + i] * Gn[m][2];
      }
      for (int d = 0; d < 3; ++d) {
        gg[d] += a.ggw[(3 * m + d) * nc + i] * (Qn[m] + Q0[q]);
        gl[d] += a.lsw[(3 * m + d) * nc + i] * dQ;
      }
    }
    const double a0 = Q0[q] - (b[3] * M2[0] + b[4] * M2[1] + b[5] * M2[2] + b[6] * M2[3] + b[7] * M2[4] + b[8] * M2[5]);
    const double p1[3] = {al * gg[0], al * gg[1], al * gg[2]};
    const double bGG = V23 * (p1[0] * p1[0] + p1[1] * p1[1] + p1[2] * p1[2]);
    const double bLS = V23 * (gl[0] * gl[0] + gl[1] * gl[1] + gl[2] * gl[2]);
    const double beta1 = fmin(bGG, bLS);
    const double vv[3][3] = {{2.0 * b[3], b[6], b[8]}, {b[6], 2.0 * b[4], b[7]}, {b[8], b[7], 2.0 * b[5]}};
    double first = 0.0;
    for (int d = 0; d < 3; ++d) {
      const double* x = vv[d];
      first += b[d] * b[d] + M2[0] * x[0] * x[0] + M2[1] * x[1] * x[1] + M2[2] * x[2] * x[2] +
               2.0 * (M2[3] * x[0] * x[1] + M2[4] * x[1] * x[2] + M2[5] * x[0] * x[2]);
    }
    const double second = 4.0 * (b[3] * b[3] + b[4] * b[4] + b[5] * b[5]) + b[6] * b[6] + b[7] * b[7] + b[8] * b[8];
    const double beta2 = V23 * first + V43 * second;
    const double rden = 1.0 / (Q0[q] * Q0[q] + beta1 + 1e-40);
    const double bt1 = beta1 * rden, bt2 = beta2 * rden, dif = bt2 - bt1;
    const double d1 = ph.weno_eps + bt1, d2 = ph.weno_eps + bt2;
    const double s2 = dif * dif, d11 = d1 * d1, d22 = d2 * d2;
    const double A1 = g1 * (d11 + s2) * d22, A2 = g2 * (d22 + s2) * d11;
    const double inv = 1.0 / (A1 + A2);
    const double w1 = A1 * inv, w2 = A2 * inv;
    const double c2 = w2 * (1.0 / g2), c1 = w1 - w2 * (g1 / g2);
    // reverse: out[0] = c2 a0 + c1 Q0, out[1+d] = c2 b[d] + c1 p1[d] (d < 3), out[1+j] = c2 b[j] (j >= 3)
    double ob[10];
    for (int k = 0; k < 10; ++k) ob[k] = cb[(10 * q + k) * cs];
    double c2b = ob[0] * a0, c1b = ob[0] * Q0[q];
    for (int d = 0; d < 3; ++d) {
      c2b += ob[1 + d] * b[d];
      c1b += ob[1 + d] * p1[d];
    }
    for (int j = 3; j < 9; ++j) c2b += ob[1 + j] * b[j];
    const double a0b = c2 * ob[0];
    double q0b = c1 * ob[0];
    double bb[9], p1b[3];
    for (int d = 0; d < 3; ++d) {
      bb[d] = c2 * ob[1 + d];
      p1b[d] = c1 * ob[1 + d];
    }
    for (int j = 3; j < 9; ++j) bb[j] = c2 * ob[1 + j];
    // weights
    const double w1b = c1b, w2b = c2b * (1.0 / g2) - c1b * (g1 / g2);
    const double t = w1b * w1 + w2b * w2;
    const double A1b = inv * (w1b - t), A2b = inv * (w2b - t);
    const double d11b = A1b * g1 * d22 + A2b * g2 * (d22 + s2);
    const double d22b = A1b * g1 * (d11 + s2) + A2b * g2 * d11;
    const double s2b = A1b * g1 * d22 + A2b * g2 * d11;
    const double bt1b = 2.0 * d1 * d11b - 2.0 * dif * s2b, bt2b = 2.0 * d2 * d22b + 2.0 * dif * s2b;
    double beta1b = bt1b * rden;
    const double beta2b = bt2b * rden;
    const double rdenb = bt1b * beta1 + bt2b * beta2;
    q0b += -rden * rden * 2.0 * Q0[q] * rdenb;
    beta1b += -rden * rden * rdenb;
    // smoothness indicator of p^2
    const double firstb = V23 * beta2b, secondb = V43 * beta2b;
    double vb[3][3];
    for (int d = 0; d < 3; ++d) {
      const double* x = vv[d];
      bb[d] += 2.0 * b[d] * firstb;
      vb[d][0] = firstb * (2.0 * M2[0] * x[0] + 2.0 * M2[3] * x[1] + 2.0 * M2[5] * x[2]);
      vb[d][1] = firstb * (2.0 * M2[1] * x[1] + 2.0 * M2[3] * x[0] + 2.0 * M2[4] * x[2]);
      vb[d][2] = firstb * (2.0 * M2[2] * x[2] + 2.0 * M2[4] * x[1] + 2.0 * M2[5] * x[0]);
    }
    bb[3] += 2.0 * vb[0][0] + 8.0 * b[3] * secondb;
    bb[4] += 2.0 * vb[1][1] + 8.0 * b[4] * secondb;
    bb[5] += 2.0 * vb[2][2] + 8.0 * b[5] * secondb;
    bb[6] += vb[0][1] + vb[1][0] + 2.0 * b[6] * secondb;
    bb[7] += vb[1][2] + vb[2][1] + 2.0 * b[7] * secondb;
    bb[8] += vb[0][2] + vb[2][0] + 2.0 * b[8] * secondb;
    // beta_1 = min(beta_GG, beta_LS)
    const double bGGb = bGG < bLS ? beta1b : (bGG > bLS ? 0.0 : 0.5 * beta1b);
    const double bLSb = bGG < bLS ? 0.0 : (bGG > bLS ? beta1b : 0.5 * beta1b);
    double glb[3], ggb[3];
    for (int d = 0; d < 3; ++d) {
      p1b[d] += 2.0 * V23 * p1[d] * bGGb;
      glb[d] = 2.0 * V23 * gl[d] * bLSb;
      ggb[d] = al * p1b[d];
    }
    // a0 = Q0 - sum_j b_j M2_j
    q0b += a0b;
    for (int j = 3; j < 9; ++j) bb[j] -= a0b * M2[j - 3];
    // the linear maps, slot by slot
    for (int m = 0; m < nt; ++m) {
      const int64_t f = a.cf[(int64_t)m * nc + i];
      double dQb = 0.0, Gnb[3] = {0, 0, 0};
      for (int j = 0; j < 9; ++j) {
        dQb += a.Kop[(j * 24 + m) * nc + i] * bb[j];
        for (int e = 0; e < 3; ++e) Gnb[e] += a.Kop[(j * 24 + 6 + 3 * m + e) * nc + i] * bb[j];
      }
      double ggsum = 0.0;
      for (int d = 0; d < 3; ++d) {
        dQb += a.lsw[(3 * m + d) * nc + i] * glb[d];
        ggsum += a.ggw[(3 * m + d) * nc + i] * ggb[d];
      }
      const double Qnb = dQb + ggsum;
      q0b += ggsum - dQb;
      if (a.fR[f] >= 0) {
        double* rec = v.rec + (2 * f + a.cside[(int64_t)m * nc + i]) * 20;
        rec[q] = Qnb;
        for (int e = 0; e < 3; ++e) rec[5 + 3 * q + e] = Gnb[e];
      } else {
        gcot[m][q] += Qnb;
        for (int e = 0; e < 3; ++e) gcot[m][5 + 3 * q + e] += Gnb[e];
      }
    }
    self[q] += q0b;
  }
  // ghost states: their transposed Jacobian in the cell's own (W, grad W), one dual seed per input
  for (int m = 0; m < nt; ++m) {
    const int64_t f = a.cf[(int64_t)m * nc + i];
    if (a.fR[f] >= 0) continue;
    const DualD n[3] = {DualD(a.fnrm[f]), DualD(a.fnrm[nf + f]), DualD(a.fnrm[2 * nf + f])};
    for (int c = 0; c < 20; ++c) {
      DualD Wd[5], Gd[15], Wg[5], Gg[15];
      for (int q = 0; q < 5; ++q) Wd[q] = DualD(Q0[q], c == q ? 1.0 : 0.0);
      for (int j = 0; j < 15; ++j) Gd[j] = DualD(G0[j], c == 5 + j ? 1.0 : 0.0);
      bc_ghost<DualD>(a.ftag[f], n, Wd, Gd, Wg, Gg, DualD(ph.gamma), ph.Winf);
      double sacc = 0.0;
      for (int q = 0; q < 5; ++q) sacc += Wg[q].d * gcot[m][q];
      for (int j = 0; j < 15; ++j) sacc += Gg[j].d * gcot[m][5 + j];
      self[c] += sacc;
    }
  }
  // local time step
  const double dtb = cb[CGKS_RC * cs];
  for (int c = 0; c < 5; ++c) {
    DualD Qd[5];
    for (int q = 0; q < 5; ++q) Qd[q] = DualD(Q0[q], q == c ? 1.0 : 0.0);
    self[c] += time_step<DualD>(i, a, Qd).d * dtb;
  }
  for (int c = 0; c < 20; ++c) v.self[(int64_t)c * nc + i] = self[c];
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
