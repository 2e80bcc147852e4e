// Bodies of the fine-level CGKS kernels (Sec. 2-3 of the paper), FP64, written as host+device
// functions over argument structs; fine.cu wraps them in kernels.
//   reconstruct_body : per cell, HWENO p^2 (constrained least-squares operator), Green-Gauss p^1
//                      scaled by the compression factor, least-squares gradient, smoothness
//                      indicators, non-linear WENO weights -> 10 coefficients per variable; local dt
//   gks_point_body   : per face Gauss point, the time-dependent gas distribution of Eq. 2nd-flux:
//                      flux averaged over dt, interface state at dt (Sec. 2.4), compression factor
//                      alpha_{p,k} (Sec. 3.3)
//   gather_body      : per cell, fixed-order sums of the Gauss-point records -> residual,
//                      Gauss-Green gradient times the compression factor, optional explicit update
// The FP64 pipe bounds this path: micro-slopes use the closed-form solution of the 5x5 moment
// system, moment matrices are applied to combined slopes, and full-space moments of time
// derivatives come from Euler-flux Jacobians (the derivative of an equilibrium moment along a slope).
#pragma once
#include "internal.cuh"
#include "kinetic.cuh"

struct ReconArgs {
  int64_t nc, nf;
  const int8_t* ctype;
  const int32_t *cf, *fL, *fR, *ftag;
  const int8_t* cside;
  const double *fnrm, *Kop, *ggw, *lsw, *aux, *dtw, *vol, *W, *G, *alpha;
  double *rc, *dt;
  Phys ph;
  DevErr* err;
};

HD void reconstruct_body(int64_t i, const ReconArgs& a) {
  const int64_t nc = a.nc, nf = a.nf;
  const int nt = a.ctype[i];
  const Phys& ph = a.ph;
  double Q0[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) Q0[q] = a.W[q * nc + i];
  // p^2 coefficients b[q][j] of X,Y,Z,X^2,Y^2,Z^2,XY,YZ,XZ; Green-Gauss and least-squares gradients
  double b[5][9], gg[5][3], gl[5][3];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
#pragma unroll
    for (int j = 0; j < 9; ++j) b[q][j] = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) gg[q][d] = gl[q][d] = 0.0;
  }
  for (int m = 0; m < nt; ++m) {
    const int64_t f = a.cf[(int64_t)m * nc + i];
    double Qn[5], Gn[15];
    if (a.fR[f] >= 0) {
      const int64_t nb = a.cside[(int64_t)m * nc + i] ? a.fL[f] : a.fR[f];
#pragma unroll
      for (int q = 0; q < 5; ++q) Qn[q] = a.W[q * nc + nb];
#pragma unroll
      for (int j = 0; j < 15; ++j) Gn[j] = a.G[j * nc + nb];
    } else {
      double G0[15];
#pragma unroll
      for (int j = 0; j < 15; ++j) G0[j] = a.G[j * nc + i];
      const double n[3] = {a.fnrm[f], a.fnrm[nf + f], a.fnrm[2 * nf + f]};
      if (!bc_ghost<double>(a.ftag[f], n, Q0, G0, Qn, Gn, ph.gamma, ph.Winf)) set_err(a.err, CGKS_ENAN, (int)i, 1);
    }
    double dQ[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) dQ[q] = Qn[q] - Q0[q];
    // the difference column and the three gradient columns of this neighbour
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      const double k0 = a.Kop[(j * 24 + m) * nc + i];
      const double kx = a.Kop[(j * 24 + 6 + 3 * m) * nc + i];
      const double ky = a.Kop[(j * 24 + 7 + 3 * m) * nc + i];
      const double kz = a.Kop[(j * 24 + 8 + 3 * m) * nc + i];
#pragma unroll
      for (int q = 0; q < 5; ++q) b[q][j] += k0 * dQ[q] + kx * Gn[3 * q] + ky * Gn[3 * q + 1] + kz * Gn[3 * q + 2];
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double wg = a.ggw[(3 * m + d) * nc + i], wl = a.lsw[(3 * m + d) * nc + i];
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        gg[q][d] += wg * (Qn[q] + Q0[q]);
        gl[q][d] += wl * dQ[q];
      }
    }
  }
  const double V23 = a.aux[i], V43 = a.aux[nc + i];
  double M2[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) M2[j] = a.aux[(2 + j) * nc + i];
  const double al = a.alpha[i];
  const double g1 = 0.5, g2 = 0.5;
  __align__(16) double out[CGKS_RC];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const double* bq = b[q];
    const double a0 = Q0[q] - (bq[3] * M2[0] + bq[4] * M2[1] + bq[5] * M2[2] + bq[6] * M2[3] + bq[7] * M2[4] + bq[8] * M2[5]);
    const double p1[3] = {al * gg[q][0], al * gg[q][1], al * gg[q][2]};
    const double bGG = V23 * (p1[0] * p1[0] + p1[1] * p1[1] + p1[2] * p1[2]);
    const double bLS = V23 * (gl[q][0] * gl[q][0] + gl[q][1] * gl[q][1] + gl[q][2] * gl[q][2]);
    const double beta1 = fmin(bGG, bLS);
    // |Omega|^(2/3) sum_d (avg of (d_d p2)^2) + |Omega|^(4/3) sum_{|a|=2} (D^a p2)^2
    const double v[3][3] = {{2.0 * bq[3], bq[6], bq[8]}, {bq[6], 2.0 * bq[4], bq[7]}, {bq[8], bq[7], 2.0 * bq[5]}};
    double first = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double* x = v[d];
      const double vMv = M2[0] * x[0] * x[0] + M2[1] * x[1] * x[1] + M2[2] * x[2] * x[2] +
                         2.0 * (M2[3] * x[0] * x[1] + M2[4] * x[1] * x[2] + M2[5] * x[0] * x[2]);
      first += bq[d] * bq[d] + vMv;
    }
    const double second = 4.0 * (bq[3] * bq[3] + bq[4] * bq[4] + bq[5] * bq[5]) + bq[6] * bq[6] + bq[7] * bq[7] + bq[8] * bq[8];
    const double beta2 = V23 * first + V43 * second;
    const double rden = 1.0 / (Q0[q] * Q0[q] + beta1 + 1e-40);
    const double bt1 = beta1 * rden, bt2 = beta2 * rden;
    const double sig = fabs(bt2 - bt1);
    const double r1 = sig / (ph.weno_eps + bt1), r2 = sig / (ph.weno_eps + bt2);
    const double w1 = g1 * (1.0 + r1 * r1), w2 = g2 * (1.0 + r2 * r2);
    const double ws = 1.0 / (w1 + w2);
    const double c2 = (w2 * ws) / g2, c1 = w1 * ws - (w2 * ws) * (g1 / g2);
    out[10 * q + 0] = c2 * a0 + c1 * Q0[q];
#pragma unroll
    for (int d = 0; d < 3; ++d) out[10 * q + 1 + d] = c2 * bq[d] + c1 * p1[d];
#pragma unroll
    for (int j = 3; j < 9; ++j) out[10 * q + 1 + j] = c2 * bq[j];
  }
  double2* dst = reinterpret_cast<double2*>(a.rc + (int64_t)CGKS_RC * i);
#pragma unroll
  for (int k = 0; k < CGKS_RC / 2; ++k) dst[k] = make_double2(out[2 * k], out[2 * k + 1]);
  // local time step: CFL |Omega| / sum_p S_p (|U.n_p| + c + 2 nu S_p / |Omega|)
  const double r = 1.0 / Q0[0];
  const double u[3] = {Q0[1] * r, Q0[2] * r, Q0[3] * r};
  const double p = (ph.gamma - 1.0) * (Q0[4] - 0.5 * Q0[0] * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
  const double c = sqrt(ph.gamma * p * r);
  const double nu = ph.viscous ? ph.mu * r : 0.0;
  const double V = a.vol[i];
  double s = 0.0;
  for (int m = 0; m < nt; ++m) {
    const double S = a.dtw[(4 * m + 3) * nc + i];
    const double un = fabs(u[0] * a.dtw[(4 * m) * nc + i] + u[1] * a.dtw[(4 * m + 1) * nc + i] +
                           u[2] * a.dtw[(4 * m + 2) * nc + i]);
    s += un + S * c + 2.0 * nu * S * S / V;
  }
  a.dt[i] = ph.cfl_fine * V / s;
  if (!(Q0[0] > 0.0) || !(p > 0.0) || !isfinite(Q0[4])) set_err(a.err, CGKS_ENAN, (int)i, 2);
}

// ---- gas-kinetic point flux -------------------------------------------------------------------

struct Mom {
  double m[7];        // u-moments (half or full space) times rho
  double v[6], w[6];  // tangential moments <v^k>, <w^k>
  double x2, x4;      // <xi^2>, <xi^4>
};

HD void tang_moments(double V, double h, double* v) {
  v[0] = 1.0;
  v[1] = V;
#pragma unroll
  for (int n = 0; n + 2 < 6; ++n) v[n + 2] = V * v[n + 1] + (n + 1) * h * v[n];
}

HD void make_mom(const Prim<double>& g, int side, double K, Mom& M) {
  u_moments<double, 6>(g.U, g.lam, side, M.m);
#pragma unroll
  for (int k = 0; k < 7; ++k) M.m[k] *= g.rho;
  const double h = 0.5 / g.lam;
  tang_moments(g.V, h, M.v);
  tang_moments(g.W, h, M.w);
  M.x2 = K * h;
  M.x4 = K * (K + 2.0) * h * h;
}

// out = <u^KU v^KV w^KW (s . psi) psi>, psi = (1, u, v, w, (u^2 + v^2 + w^2 + xi^2)/2)
template <int KU, int KV, int KW>
HD void psi_apply(const Mom& M, const double s[5], double out[5]) {
  const double* m = M.m;
  const double* v = M.v;
  const double* w = M.w;
#define MM(a, b, c) (m[KU + (a)] * (v[KV + (b)] * w[KW + (c)]))
  const double e00 = MM(0, 0, 0), e01 = MM(1, 0, 0), e11 = MM(2, 0, 0);
  const double e02 = MM(0, 1, 0), e12 = MM(1, 1, 0), e22 = MM(0, 2, 0);
  const double e03 = MM(0, 0, 1), e13 = MM(1, 0, 1), e23 = MM(0, 1, 1), e33 = MM(0, 0, 2);
  const double e04 = 0.5 * (e11 + e22 + e33 + M.x2 * e00);
  const double e14 = 0.5 * (MM(3, 0, 0) + MM(1, 2, 0) + MM(1, 0, 2) + M.x2 * e01);
  const double e24 = 0.5 * (MM(2, 1, 0) + MM(0, 3, 0) + MM(0, 1, 2) + M.x2 * e02);
  const double e34 = 0.5 * (MM(2, 0, 1) + MM(0, 2, 1) + MM(0, 0, 3) + M.x2 * e03);
  const double e44 = 0.25 * (MM(4, 0, 0) + MM(0, 4, 0) + MM(0, 0, 4) + M.x4 * e00 +
                             2.0 * (MM(2, 2, 0) + MM(2, 0, 2) + MM(0, 2, 2)) + 2.0 * M.x2 * (e11 + e22 + e33));
#undef MM
  out[0] = e00 * s[0] + e01 * s[1] + e02 * s[2] + e03 * s[3] + e04 * s[4];
  out[1] = e01 * s[0] + e11 * s[1] + e12 * s[2] + e13 * s[3] + e14 * s[4];
  out[2] = e02 * s[0] + e12 * s[1] + e22 * s[2] + e23 * s[3] + e24 * s[4];
  out[3] = e03 * s[0] + e13 * s[1] + e23 * s[2] + e33 * s[3] + e34 * s[4];
  out[4] = e04 * s[0] + e14 * s[1] + e24 * s[2] + e34 * s[3] + e44 * s[4];
}

// micro-slope s with <s psi> = dW under the full Maxwellian g (closed form of the 5x5 system)
HD void slope_solve(const Prim<double>& g, double K, const double dW[5], double s[5]) {
  const double r = 1.0 / g.rho;
  const double d0 = dW[0] * r, d1 = dW[1] * r, d2 = dW[2] * r, d3 = dW[3] * r, d4 = dW[4] * r;
  const double q2 = g.U * g.U + g.V * g.V + g.W * g.W + (K + 3.0) * 0.5 / g.lam;
  const double R4 = 2.0 * d4 - q2 * d0;
  const double R1 = d1 - g.U * d0, R2 = d2 - g.V * d0, R3 = d3 - g.W * d0;
  const double l2 = 2.0 * g.lam;
  s[4] = (l2 * l2 / (K + 3.0)) * (R4 - 2.0 * (g.U * R1 + g.V * R2 + g.W * R3));
  s[1] = l2 * R1 - g.U * s[4];
  s[2] = l2 * R2 - g.V * s[4];
  s[3] = l2 * R3 - g.W * s[4];
  s[0] = d0 - g.U * s[1] - g.V * s[2] - g.W * s[3] - 0.5 * s[4] * q2;
}

// directional derivative of the Euler flux through the k-th axis of the face frame along dW:
// equals <u_k (a . psi) psi> under the full Maxwellian when <a psi> = dW
HD void euler_jvp(const double w[5], const Prim<double>& g, double gm1, int k, const double dW[5], double out[5]) {
  const double r = 1.0 / w[0];
  const double u[3] = {g.U, g.V, g.W};
  const double du[3] = {(dW[1] - u[0] * dW[0]) * r, (dW[2] - u[1] * dW[0]) * r, (dW[3] - u[2] * dW[0]) * r};
  const double p = 0.5 * w[0] / g.lam;
  const double dp = gm1 * (dW[4] - (u[0] * dW[1] + u[1] * dW[2] + u[2] * dW[3]) +
                           0.5 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) * dW[0]);
  const double mk = w[1 + k], dmk = dW[1 + k];
  out[0] = dmk;
#pragma unroll
  for (int j = 0; j < 3; ++j) out[1 + j] = dmk * u[j] + mk * du[j];
  out[1 + k] += dp;
  out[4] = du[k] * (w[4] + p) + u[k] * (dW[4] + dp);
}

// gradient (global frame) of a reconstruction polynomial at offset X from its centroid
HD void eval_gradient(const double* rcp, const double X[3], double Gq[15]) {
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const double2* c2 = reinterpret_cast<const double2*>(rcp + 10 * q);
    const double2 A = c2[0], B = c2[1], C = c2[2], D = c2[3], E = c2[4];
    // (r0 r1) (r2 r3) (r4 r5) (r6 r7) (r8 r9): 1 X Y Z X^2 Y^2 Z^2 XY YZ XZ
    Gq[3 * q + 0] = A.y + 2.0 * C.x * X[0] + D.y * X[1] + E.y * X[2];
    Gq[3 * q + 1] = B.x + 2.0 * C.y * X[1] + D.y * X[0] + E.x * X[2];
    Gq[3 * q + 2] = B.y + 2.0 * D.x * X[2] + E.x * X[1] + E.y * X[0];
  }
}

HD void eval_value(const double* rcp, const double X[3], double Wv[5]) {
  const double xx = X[0] * X[0], yy = X[1] * X[1], zz = X[2] * X[2], xy = X[0] * X[1], yz = X[1] * X[2], xz = X[0] * X[2];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const double2* c2 = reinterpret_cast<const double2*>(rcp + 10 * q);
    const double2 A = c2[0], B = c2[1], C = c2[2], D = c2[3], E = c2[4];
    Wv[q] = A.x + A.y * X[0] + B.x * X[1] + B.y * X[2] + C.x * xx + C.y * yy + D.x * zz + D.y * xy + E.x * yz + E.y * xz;
  }
}

// directional derivatives along (n, t1, t2) of the frame-rotated conservative variables
HD void rotate_gradient(const double Gq[15], const double* e[3], double D[3][5]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double* dir = e[k];
    double gs[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) gs[q] = Gq[3 * q] * dir[0] + Gq[3 * q + 1] * dir[1] + Gq[3 * q + 2] * dir[2];
    D[k][0] = gs[0];
    D[k][4] = gs[4];
#pragma unroll
    for (int j = 0; j < 3; ++j) D[k][1 + j] = e[j][0] * gs[1] + e[j][1] * gs[2] + e[j][2] * gs[3];
  }
}

// one side of the interface: micro-slopes of the initial distribution, its contribution to the
// equilibrium slopes, the time-integrated flux, the state at dt and the time-integrated state
template <int SIDE>
HD void side_terms(const double D[3][5], const double w[5], const Prim<double>& g, double K, double gm1, double tau,
                   double q4, double q5, double edt, double dtf, double dWc[3][5], double Facc[5], double Wacc[5],
                   double Iacc[5]) {
  double a[3][5];
#pragma unroll
  for (int k = 0; k < 3; ++k) slope_solve(g, K, D[k], a[k]);
  // time slope A from <A + a.u> = 0 under the full Maxwellian: <(a.u) psi> = sum_k J_k dW_k
  double au[5] = {0, 0, 0, 0, 0};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double t[5];
    euler_jvp(w, g, gm1, k, D[k], t);
#pragma unroll
    for (int q = 0; q < 5; ++q) au[q] -= t[q];
  }
  double A[5];
  slope_solve(g, K, au, A);
  Mom M;
  make_mom(g, SIDE, K, M);
  double t0[5], t1[5], t2[5];
  psi_apply<0, 0, 0>(M, a[0], t0);
  psi_apply<0, 0, 0>(M, a[1], t1);
  psi_apply<0, 0, 0>(M, a[2], t2);
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    dWc[0][q] += t0[q];
    dWc[1][q] += t1[q];
    dWc[2][q] += t2[q];
  }
  const double one[5] = {1.0, 0.0, 0.0, 0.0, 0.0};
  double Va[5], VA[5], V0[5], Fa[5], FA[5], F0[5];
  {
    double x[5], y[5], z[5];
    psi_apply<1, 0, 0>(M, a[0], x);
    psi_apply<0, 1, 0>(M, a[1], y);
    psi_apply<0, 0, 1>(M, a[2], z);
#pragma unroll
    for (int q = 0; q < 5; ++q) Va[q] = x[q] + y[q] + z[q];
    psi_apply<2, 0, 0>(M, a[0], x);
    psi_apply<1, 1, 0>(M, a[1], y);
    psi_apply<1, 0, 1>(M, a[2], z);
#pragma unroll
    for (int q = 0; q < 5; ++q) Fa[q] = x[q] + y[q] + z[q];
  }
  psi_apply<0, 0, 0>(M, A, VA);
  psi_apply<0, 0, 0>(M, one, V0);
  psi_apply<1, 0, 0>(M, A, FA);
  psi_apply<1, 0, 0>(M, one, F0);
  const double tq4 = tau * q4;
  const double etd = edt * (tau + dtf), etau = edt * tau;
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    Facc[q] += q4 * F0[q] - q5 * Fa[q] - tq4 * FA[q];
    Wacc[q] += edt * V0[q] - etd * Va[q] - etau * VA[q];
    Iacc[q] += q4 * V0[q] - q5 * Va[q] - tq4 * VA[q];
  }
}

struct PointArgs {
  int64_t ngp, nf, nc;
  const int32_t *gp_face, *fL, *fR, *ftag;
  const double *gp_x, *gp_A, *fshift, *ctr, *rc, *dt;
  double *gpF, *gpW, *gpa;
  Phys ph;
  DevErr* err;
};

HD void gks_point_body(int64_t g, const PointArgs& a) {
  const Phys& ph = a.ph;
  const int64_t ngp = a.ngp, nf = a.nf, nc = a.nc;
  const int64_t f = a.gp_face[g];
  const int64_t L = a.fL[f], R = a.fR[f];
  const double x[3] = {a.gp_x[g], a.gp_x[ngp + g], a.gp_x[2 * ngp + g]};
  const double Av[3] = {a.gp_A[g], a.gp_A[ngp + g], a.gp_A[2 * ngp + g]};
  const double wgt = sqrt(Av[0] * Av[0] + Av[1] * Av[1] + Av[2] * Av[2]);
  const double n[3] = {Av[0] / wgt, Av[1] / wgt, Av[2] / wgt};
  double t1[3], t2[3];
  face_frame(n, t1, t2);
  const double* e[3] = {n, t1, t2};
  const double K = ph.K, gm1 = ph.gamma - 1.0;
  const bool bnd = R < 0;
  // left and right states and gradients at the point (global frame)
  const double* rcL = a.rc + (int64_t)CGKS_RC * L;
  const double XL[3] = {x[0] - a.ctr[L], x[1] - a.ctr[nc + L], x[2] - a.ctr[2 * nc + L]};
  double WLg[5], WRg[5], GLg[15], GRg[15], dtf;
  eval_value(rcL, XL, WLg);
  eval_gradient(rcL, XL, GLg);
  if (!bnd) {
    const double* rcR = a.rc + (int64_t)CGKS_RC * R;
    double XR[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) XR[d] = x[d] - a.fshift[d * nf + f] - a.ctr[d * nc + R];
    eval_value(rcR, XR, WRg);
    eval_gradient(rcR, XR, GRg);
    dtf = fmin(a.dt[L], a.dt[R]);
  } else {
    if (!bc_ghost<double>(a.ftag[f], n, WLg, GLg, WRg, GRg, ph.gamma, ph.Winf)) set_err(a.err, CGKS_ENAN, (int)f, 3);
    dtf = a.dt[L];
  }
  double wl[5], wr[5];
  rotate_in(WLg, n, t1, t2, wl);
  rotate_in(WRg, n, t1, t2, wr);
  Prim<double> gl, gr;
  const bool okl = prim_local(wl, gm1, gl), okr = prim_local(wr, gm1, gr);
  if (!(okl && okr)) set_err(a.err, CGKS_ENAN, (int)f, 4);
  // interface equilibrium W^c = int_{u>0} psi g^l + int_{u<0} psi g^r (Eq. compatibility2)
  double wc[5];
  {
    double ml[3], mr[3];
    u_moments<double, 2>(gl.U, gl.lam, 1, ml);
    u_moments<double, 2>(gr.U, gr.lam, -1, mr);
    const double ql = gl.V * gl.V + gl.W * gl.W + (K + 2.0) * 0.5 / gl.lam;
    const double qr = gr.V * gr.V + gr.W * gr.W + (K + 2.0) * 0.5 / gr.lam;
    wc[0] = gl.rho * ml[0] + gr.rho * mr[0];
    wc[1] = gl.rho * ml[1] + gr.rho * mr[1];
    wc[2] = gl.rho * gl.V * ml[0] + gr.rho * gr.V * mr[0];
    wc[3] = gl.rho * gl.W * ml[0] + gr.rho * gr.W * mr[0];
    wc[4] = 0.5 * (gl.rho * (ml[2] + ml[0] * ql) + gr.rho * (mr[2] + mr[0] * qr));
  }
  Prim<double> gc;
  if (!prim_local(wc, gm1, gc)) set_err(a.err, CGKS_ENAN, (int)f, 5);
  // collision times (Sec. 2.3)
  const double pl = 0.5 * gl.rho / gl.lam, pr = 0.5 * gr.rho / gr.lam, pc = 0.5 * gc.rho / gc.lam;
  const double jump = fabs((pl - pr) / (pl + pr));
  double tau, tn;
  if (ph.viscous) {
    tau = ph.mu / pc;
    tn = tau + ph.c_press * jump * dtf;
  } else {
    tn = ph.eps_inviscid * dtf + ph.c_press * jump * dtf;
    tau = tn;
  }
  // exact integrals over [0, dt] of the time coefficients of Eq. 2nd-flux
  const double edt = exp(-dtf / tn), om = 1.0 - edt;
  const double q1 = dtf - tn * om;
  const double q2 = (tn * tn + tau * tn) * om - tn * dtf * edt - tau * dtf;
  const double q3 = 0.5 * dtf * dtf - tau * dtf + tau * tn * om;
  const double q4 = tn * om;
  const double q5 = (tau * tn + tn * tn) * om - tn * dtf * edt;
  // compression factor of this Gauss point (interior faces only)
  double alpha = 1.0;
  if (!bnd) {
    const double cl = sqrt(ph.gamma * pl / gl.rho), cr = sqrt(ph.gamma * pr / gr.rho);
    const double dp = fabs(pl - pr);
    const double dn = gl.U / cl - gr.U / cr, d1 = gl.V / cl - gr.V / cr, d2 = gl.W / cl - gr.W / cr;
    const double A = dp / pl + dp / pr + dn * dn + (d1 * d1 + d2 * d2);
    alpha = 1.0 / (1.0 + A * A);
  }
  double dWc[3][5], Facc[5], Wacc[5], Iacc[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    dWc[0][q] = dWc[1][q] = dWc[2][q] = 0.0;
    Facc[q] = Wacc[q] = Iacc[q] = 0.0;
  }
  {
    double D[3][5];
    rotate_gradient(GLg, e, D);
    side_terms<1>(D, wl, gl, K, gm1, tau, q4, q5, edt, dtf, dWc, Facc, Wacc, Iacc);
    rotate_gradient(GRg, e, D);
    side_terms<-1>(D, wr, gr, K, gm1, tau, q4, q5, edt, dtf, dWc, Facc, Wacc, Iacc);
  }
  // equilibrium part: slopes a^c from the kinetic-weighted interface gradients; A^c from
  // <A + a.u> = 0; full-space moments through the Euler-flux Jacobians
  double ac[3][5];
#pragma unroll
  for (int k = 0; k < 3; ++k) slope_solve(gc, K, dWc[k], ac[k]);
  double cu[5] = {0, 0, 0, 0, 0};  // <(a^c . u) psi>_c = sum_k J_k dW^c_k
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double t[5];
    euler_jvp(wc, gc, gm1, k, dWc[k], t);
#pragma unroll
    for (int q = 0; q < 5; ++q) cu[q] += t[q];
  }
  double Fc0[5], FcA[5], Fca[5];
  {
    // <u psi>_c is the Euler flux of W^c; <u A^c psi>_c = J_n <A^c psi>_c = -J_n <(a^c . u) psi>_c
    const double u0 = gc.U, pcc = pc;
    Fc0[0] = wc[1];
    Fc0[1] = wc[1] * u0 + pcc;
    Fc0[2] = wc[2] * u0;
    Fc0[3] = wc[3] * u0;
    Fc0[4] = (wc[4] + pcc) * u0;
    euler_jvp(wc, gc, gm1, 0, cu, FcA);
#pragma unroll
    for (int q = 0; q < 5; ++q) FcA[q] = -FcA[q];
    Mom M;
    make_mom(gc, 0, K, M);
    double xx[5], yy[5], zz[5];
    psi_apply<2, 0, 0>(M, ac[0], xx);
    psi_apply<1, 1, 0>(M, ac[1], yy);
    psi_apply<1, 0, 1>(M, ac[2], zz);
#pragma unroll
    for (int q = 0; q < 5; ++q) Fca[q] = xx[q] + yy[q] + zz[q];
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    Facc[q] += q1 * Fc0[q] + q2 * Fca[q] + q3 * FcA[q];
    Wacc[q] += om * (wc[q] - dtf * cu[q]);
    Iacc[q] += q1 * wc[q] + (q2 - q3) * cu[q];
  }
  if (ph.viscous && ph.prandtl != 1.0) {
    // heat flux about U^c of the time-integrated distribution, scaled by (1/Pr - 1)
    const double Ub[3] = {gc.U, gc.V, gc.W};
    const double U2 = Ub[0] * Ub[0] + Ub[1] * Ub[1] + Ub[2] * Ub[2];
    const double qn = Facc[4] - (Ub[0] * Facc[1] + Ub[1] * Facc[2] + Ub[2] * Facc[3]) + 0.5 * U2 * Facc[0] -
                      Ub[0] * (Iacc[4] - (Ub[0] * Iacc[1] + Ub[1] * Iacc[2] + Ub[2] * Iacc[3]) + 0.5 * U2 * Iacc[0]);
    Facc[4] += (1.0 / ph.prandtl - 1.0) * qn;
  }
  const double sdt = wgt / dtf;
#pragma unroll
  for (int q = 0; q < 5; ++q) Facc[q] *= sdt;
  double Fg[5], Wg[5];
  rotate_out(Facc, n, t1, t2, Fg);
  rotate_out(Wacc, n, t1, t2, Wg);
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    a.gpF[q * ngp + g] = Fg[q];
    a.gpW[q * ngp + g] = Wg[q];
  }
  a.gpa[g] = alpha;
}

struct GatherArgs {
  int64_t nc, ngp;
  const int8_t *ctype, *cside;
  const int32_t *cf, *gp_ptr;
  const double *gp_A, *gpF, *gpW, *gpa, *vol, *dt, *W_in;
  double *W_out, *res, *G_out, *alpha_out;
  int update;
  double gamma;
  DevErr* err;
};

HD void gather_body(int64_t i, const GatherArgs& a) {
  const int64_t nc = a.nc, ngp = a.ngp;
  double r[5] = {0, 0, 0, 0, 0}, gs[15];
#pragma unroll
  for (int j = 0; j < 15; ++j) gs[j] = 0.0;
  double al = 1.0;
  const int nt = a.ctype[i];
  for (int m = 0; m < nt; ++m) {
    const int64_t f = a.cf[(int64_t)m * nc + i];
    const double s = a.cside[(int64_t)m * nc + i] ? -1.0 : 1.0;
    for (int64_t g = a.gp_ptr[f]; g < a.gp_ptr[f + 1]; ++g) {
      const double A[3] = {s * a.gp_A[g], s * a.gp_A[ngp + g], s * a.gp_A[2 * ngp + g]};
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        r[q] -= s * a.gpF[q * ngp + g];
        const double wq = a.gpW[q * ngp + g];
#pragma unroll
        for (int d = 0; d < 3; ++d) gs[3 * q + d] += wq * A[d];
      }
      al *= a.gpa[g];
    }
  }
  const double rv = 1.0 / a.vol[i];
  if (a.res)
#pragma unroll
    for (int q = 0; q < 5; ++q) a.res[q * nc + i] = r[q];
  if (a.G_out)
#pragma unroll
    for (int j = 0; j < 15; ++j) a.G_out[j * nc + i] = al * gs[j] * rv;
  if (a.alpha_out) a.alpha_out[i] = al;
  if (a.update) {
    const double h = a.dt[i] * rv;
    double w[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      w[q] = a.W_in[q * nc + i] + h * r[q];
      a.W_out[q * nc + i] = w[q];
    }
    const double p = (a.gamma - 1.0) * (w[4] - 0.5 * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]) / w[0]);
    if (!(w[0] > 0.0) || !(p > 0.0) || !isfinite(p)) set_err(a.err, CGKS_ENAN, (int)i, 6);
  }
}
