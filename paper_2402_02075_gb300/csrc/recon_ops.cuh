// Per-cell precompute of the reconstruction operators (Sec. 3): the constrained least-squares p^2
// map, Green-Gauss and least-squares gradient weights, indicator constants and time-step weights,
// as host+device functions (mesh.cu runs them in a kernel; the host can run them on the same
// arrays).
#pragma once
#include "internal.cuh"

__host__ __device__ __forceinline__ int cell_nfaces(int t) { return t == 7 ? 5 : t; }

// ---- dense helpers of the reconstruction-operator precompute (per thread, column-major) --------

// Householder QR of A (m x n, m >= n, column-major, leading dimension m): R in the upper triangle,
// reflector k stored in A[k+1:, k] with an implicit unit leading entry, scale in tau[k].
__host__ __device__ inline bool house_qr(int m, int n, double* A, double* tau) {
  for (int k = 0; k < n; ++k) {
    double* a = A + k * m;
    double s = 0.0;
    for (int i = k + 1; i < m; ++i) s += a[i] * a[i];
    const double x0 = a[k];
    const double nrm = sqrt(x0 * x0 + s);
    if (nrm == 0.0) return false;
    const double beta = x0 >= 0.0 ? -nrm : nrm;
    const double v0 = x0 - beta;
    for (int i = k + 1; i < m; ++i) a[i] /= v0;
    tau[k] = (beta - x0) / beta;
    a[k] = beta;
    for (int j = k + 1; j < n; ++j) {
      double* b = A + j * m;
      double d = b[k];
      for (int i = k + 1; i < m; ++i) d += a[i] * b[i];
      d *= tau[k];
      b[k] -= d;
      for (int i = k + 1; i < m; ++i) b[i] -= d * a[i];
    }
  }
  return true;
}

// y <- Q y (Q = H_0 H_1 ... H_{n-1}) or y <- Q^T y
__host__ __device__ inline void house_apply(int m, int n, const double* A, const double* tau, double* y, bool transpose) {
  for (int kk = 0; kk < n; ++kk) {
    const int k = transpose ? kk : n - 1 - kk;
    const double* a = A + k * m;
    double d = y[k];
    for (int i = k + 1; i < m; ++i) d += a[i] * y[i];
    d *= tau[k];
    y[k] -= d;
    for (int i = k + 1; i < m; ++i) y[i] -= d * a[i];
  }
}

// p^2 operator, Green-Gauss and least-squares weights, smoothness-indicator constants and
// time-step weights of every cell.  Stencil: the cell and its face neighbours; a boundary face
// contributes the mirror image of the cell in the face plane (ghost cell).
struct ROArgs {
  int64_t nc, nf;
  const int8_t* ctype;
  const int32_t* cf;
  const int8_t* cside;
  const int32_t *fL, *fR;
  const double *vol, *ctr, *m2, *Sn, *area, *fshift, *fctr, *fnrm;
  double *Kop, *ggw, *lsw, *aux, *dtw;
  DevErr* err;
};

__host__ __device__ inline void recon_ops_body(int64_t i, const ROArgs& A_) {
  const int64_t nc = A_.nc, nf = A_.nf;
  const int8_t* ctype = A_.ctype;
  const int32_t* cf = A_.cf;
  const int8_t* cside = A_.cside;
  const int32_t *fL = A_.fL, *fR = A_.fR;
  const double *vol = A_.vol, *ctr = A_.ctr, *m2 = A_.m2, *Sn = A_.Sn, *area = A_.area, *fshift = A_.fshift,
               *fctr = A_.fctr, *fnrm = A_.fnrm;
  double *Kop = A_.Kop, *ggw = A_.ggw, *lsw = A_.lsw, *aux = A_.aux, *dtw = A_.dtw;
  DevErr* err = A_.err;
  const int nt = cell_nfaces(ctype[i]);
  const double V = vol[i];
  double c0[3], M0[6];
  for (int d = 0; d < 3; ++d) c0[d] = ctr[d * nc + i];
  for (int j = 0; j < 6; ++j) M0[j] = m2[j * nc + i];
  double dl[6][3], Mn[6][6];
  for (int m = 0; m < nt; ++m) {
    const int64_t f = cf[(int64_t)m * nc + i];
    const bool side = cside[(int64_t)m * nc + i] != 0;
    const double sg = side ? -1.0 : 1.0;
    double S[3];
    for (int d = 0; d < 3; ++d) S[d] = sg * Sn[d * nf + f];
    const double sn = sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
    for (int d = 0; d < 3; ++d) {
      ggw[(3 * m + d) * nc + i] = S[d] / (2.0 * V);
      dtw[(4 * m + d) * nc + i] = S[d] * (area[f] / sn);
    }
    dtw[(4 * m + 3) * nc + i] = area[f];
    if (fR[f] >= 0) {
      const int64_t nb = side ? fL[f] : fR[f];
      for (int d = 0; d < 3; ++d) dl[m][d] = ctr[d * nc + nb] + sg * fshift[d * nf + f] - c0[d];
      for (int j = 0; j < 6; ++j) Mn[m][j] = m2[j * nc + nb];
    } else {
      double n[3], h = 0.0;
      for (int d = 0; d < 3; ++d) {
        n[d] = fnrm[d * nf + f];
        h += (c0[d] - fctr[d * nf + f]) * n[d];
      }
      for (int d = 0; d < 3; ++d) dl[m][d] = -2.0 * h * n[d];
      // mirrored moments R M R, R = I - 2 n n^T
      const double A[3][3] = {{M0[0], M0[3], M0[5]}, {M0[3], M0[1], M0[4]}, {M0[5], M0[4], M0[2]}};
      double An[3], nAn = 0.0;
      for (int r = 0; r < 3; ++r) {
        An[r] = A[r][0] * n[0] + A[r][1] * n[1] + A[r][2] * n[2];
        nAn += n[r] * An[r];
      }
      double B[3][3];
      for (int r = 0; r < 3; ++r)
        for (int s = 0; s < 3; ++s) B[r][s] = A[r][s] - 2.0 * (n[r] * An[s] + An[r] * n[s]) + 4.0 * nAn * n[r] * n[s];
      Mn[m][0] = B[0][0];
      Mn[m][1] = B[1][1];
      Mn[m][2] = B[2][2];
      Mn[m][3] = B[0][1];
      Mn[m][4] = B[1][2];
      Mn[m][5] = B[0][2];
    }
  }
  for (int m = nt; m < 6; ++m) {
    for (int d = 0; d < 3; ++d) ggw[(3 * m + d) * nc + i] = 0.0;
    for (int d = 0; d < 4; ++d) dtw[(4 * m + d) * nc + i] = 0.0;
  }
  // C (nt x 9): averages of the basis X,Y,Z,X^2,Y^2,Z^2,XY,YZ,XZ over the neighbour minus over the cell;
  // B (3nt x 9): averages of their derivatives over the neighbour
  double Ct[9 * 6];   // C^T, column-major 9 x nt
  double Bm[18 * 9];  // B, column-major (3nt) x 9
  const int mb = 3 * nt;
  for (int m = 0; m < nt; ++m) {
    const double* x = dl[m];
    const double* M = Mn[m];
    const double row[9] = {x[0], x[1], x[2], M[0] + x[0] * x[0] - M0[0], M[1] + x[1] * x[1] - M0[1],
                           M[2] + x[2] * x[2] - M0[2], M[3] + x[0] * x[1] - M0[3], M[4] + x[1] * x[2] - M0[4],
                           M[5] + x[0] * x[2] - M0[5]};
    for (int j = 0; j < 9; ++j) Ct[m * 9 + j] = row[j];
    const double dx[9] = {1, 0, 0, 2 * x[0], 0, 0, x[1], 0, x[2]};
    const double dy[9] = {0, 1, 0, 0, 2 * x[1], 0, x[0], x[2], 0};
    const double dz[9] = {0, 0, 1, 0, 0, 2 * x[2], 0, x[1], x[0]};
    for (int j = 0; j < 9; ++j) {
      Bm[j * mb + 3 * m + 0] = dx[j];
      Bm[j * mb + 3 * m + 1] = dy[j];
      Bm[j * mb + 3 * m + 2] = dz[j];
    }
  }
  double tc[6];
  if (!house_qr(9, nt, Ct, tc)) {
    set_err(err, CGKS_EMESH, (int)i, 50);
    return;
  }
  // Q (9 x 9) explicit
  double Q[81];
  for (int col = 0; col < 9; ++col) {
    double* y = Q + col * 9;
    for (int r = 0; r < 9; ++r) y[r] = r == col ? 1.0 : 0.0;
    house_apply(9, nt, Ct, tc, y, false);
  }
  // A1 = Q1 R^{-T} (9 x nt): each row x of A1 solves R x^T = (row of Q1)^T, back substitution;
  // R[k][j] is stored at Ct[j*9 + k]
  double A1[9 * 6];
  for (int r = 0; r < 9; ++r)
    for (int k = nt - 1; k >= 0; --k) {
      double s = Q[k * 9 + r];
      for (int j = k + 1; j < nt; ++j) s -= Ct[j * 9 + k] * A1[j * 9 + r];
      A1[k * 9 + r] = s / Ct[k * 9 + k];
    }
  // BQ2 (mb x nz)
  const int nz = 9 - nt;
  double BQ2[18 * 5], tb[5];
  for (int c = 0; c < nz; ++c)
    for (int r = 0; r < mb; ++r) {
      double s = 0.0;
      for (int j = 0; j < 9; ++j) s += Bm[j * mb + r] * Q[(nt + c) * 9 + j];
      BQ2[c * mb + r] = s;
    }
  if (!house_qr(mb, nz, BQ2, tb)) {
    set_err(err, CGKS_EMESH, (int)i, 51);
    return;
  }
  // P2 = (BQ2)^+ = Rb^{-1} Qb^T (nz x mb), column by column of the identity
  double P2[5 * 18];
  for (int col = 0; col < mb; ++col) {
    double y[18];
    for (int r = 0; r < mb; ++r) y[r] = r == col ? 1.0 : 0.0;
    house_apply(mb, nz, BQ2, tb, y, true);
    for (int r = nz - 1; r >= 0; --r) {
      double s = y[r];
      for (int j = r + 1; j < nz; ++j) s -= BQ2[j * mb + r] * P2[col * 5 + j];
      P2[col * 5 + r] = s / BQ2[r * mb + r];
    }
  }
  // Kg = Q2 P2 (9 x mb); KdQ = A1 - Kg (B A1) (9 x nt)
  double Kg[9 * 18];
  for (int col = 0; col < mb; ++col)
    for (int r = 0; r < 9; ++r) {
      double s = 0.0;
      for (int j = 0; j < nz; ++j) s += Q[(nt + j) * 9 + r] * P2[col * 5 + j];
      Kg[col * 9 + r] = s;
    }
  for (int k = 0; k < nt; ++k) {
    double BA[18];
    for (int r = 0; r < mb; ++r) {
      double s = 0.0;
      for (int j = 0; j < 9; ++j) s += Bm[j * mb + r] * A1[k * 9 + j];
      BA[r] = s;
    }
    for (int r = 0; r < 9; ++r) {
      double s = A1[k * 9 + r];
      for (int j = 0; j < mb; ++j) s -= Kg[j * 9 + r] * BA[j];
      Kop[(r * 24 + k) * nc + i] = s;
    }
  }
  for (int r = 0; r < 9; ++r) {
    for (int k = nt; k < 6; ++k) Kop[(r * 24 + k) * nc + i] = 0.0;
    for (int col = 0; col < 18; ++col) Kop[(r * 24 + 6 + col) * nc + i] = col < mb ? Kg[col * 9 + r] : 0.0;
  }
  // least-squares gradient weights: D^+ with D = [dl_m] (nt x 3)
  double D[6 * 3], td[3];
  for (int d = 0; d < 3; ++d)
    for (int m = 0; m < nt; ++m) D[d * nt + m] = dl[m][d];
  if (!house_qr(nt, 3, D, td)) {
    set_err(err, CGKS_EMESH, (int)i, 52);
    return;
  }
  for (int m = 0; m < 6; ++m) {
    double y[6] = {0, 0, 0, 0, 0, 0}, g[3];
    if (m < nt) {
      y[m] = 1.0;
      house_apply(nt, 3, D, td, y, true);
      for (int r = 2; r >= 0; --r) {
        double s = y[r];
        for (int j = r + 1; j < 3; ++j) s -= D[j * nt + r] * g[j];
        g[r] = s / D[r * nt + r];
      }
    } else {
      g[0] = g[1] = g[2] = 0.0;
    }
    for (int d = 0; d < 3; ++d) lsw[(3 * m + d) * nc + i] = g[d];
  }
  const double c13 = cbrt(V);
  aux[0 * nc + i] = c13 * c13;  // |Omega|^(2/3)
  aux[1 * nc + i] = V * c13;    // |Omega|^(4/3)
  for (int j = 0; j < 6; ++j) aux[(2 + j) * nc + i] = M0[j];
}

