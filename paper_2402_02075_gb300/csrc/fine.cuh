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
// The FP64 pipe bounds this path (FP64 runs at 1/62 of the FP32 rate on this GPU), so the code is
// written for few FP64 instructions: one reciprocal and one square-root family per Maxwellian,
// micro-slopes from the closed-form solution of the 5x5 moment system, the half-space erfc/exp
// seeds computed once per side, moment matrices applied to the slopes, and full-space moments of
// time derivatives from Euler-flux Jacobian products (the derivative of an equilibrium moment along
// a slope direction).
#pragma once
#include <cstring>

#include "internal.cuh"
#include "kinetic.cuh"

// sizes of the stored linearisation (the adjoint): inputs and outputs of one Gauss point; of one
// cell's reconstruction: its own slot dense (20 inputs (W, grad W) x 51 outputs, the coefficients and
// the time step), and per neighbour slot (up to 6) one block per variable q, 4 inputs (W_q and its
// gradient) x its 10 coefficients -- each variable is reconstructed on its own, so a neighbour's
// variable q reaches no other variable's coefficients (only the cell's own ghosts couple them)
#define CGKS_PJ_IN 41
#define CGKS_PJ_OUT 10
#define CGKS_RJ_OUT 51
#define CGKS_RJ_SELF (20 * CGKS_RJ_OUT)
#define CGKS_RJ_NB (5 * 4 * 10)
#define CGKS_RJ_ROWS (CGKS_RJ_SELF + 6 * CGKS_RJ_NB)

HD double rsqrt_hd(double x) {
#ifdef __CUDA_ARCH__
  return rsqrt(x);
#else
  return 1.0 / sqrt(x);
#endif
}
HD DualD rsqrt_hd(DualD x) {
  const double r = rsqrt_hd(x.v);
  return DualD(r, -0.5 * r * r * r * x.d);
}

// dynamic viscosity at temperature ratio t = T/T_inf = gamma p/rho (free stream rho 1, p 1/gamma):
// constant, or Sutherland's law mu_inf t^(3/2) (1 + s)/(t + s)
template <typename T>
HD T viscosity(const Phys& ph, T t) {
  if (ph.suth == 0.0) return T(ph.mu);
  return ph.mu * t * sqrt(t) * (1.0 + ph.suth) / (t + ph.suth);
}

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

// value of stencil input c of slot s as T: with T = DualD the one seeded input carries derivative 1
template <typename T>
struct Seed {
  HD static T at(double v, bool) { return v; }
};
template <>
struct Seed<DualD> {
  HD static DualD at(double v, bool on) { return DualD(v, on ? 1.0 : 0.0); }
};

// reconstruction of cell i: 10 coefficients per variable.  Seeds of the
// forward-mode linearisation: 20 s + c is component c of (W 5, grad W 15) of stencil slot s (slot 0
// the cell, slot 1 + m its neighbour through local face m); seed < 0 for none
template <typename T>
HD void reconstruct_cell(int64_t i, const ReconArgs& a, int seed, T out[CGKS_RC]) {
  const int64_t nc = a.nc, nf = a.nf;
  const int nt = a.ctype[i] == 7 ? 5 : a.ctype[i];  // faces: pyramids (type 7) have 5
  const Phys& ph = a.ph;
  T Q0[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) Q0[q] = Seed<T>::at(a.W[q * nc + i], seed == q);
  // p^2 coefficients b[q][j] of X,Y,Z,X^2,Y^2,Z^2,XY,YZ,XZ; Green-Gauss and least-squares gradients
  T b[5][9], gg[5][3], gl[5][3];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
#pragma unroll
    for (int j = 0; j < 9; ++j) b[q][j] = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) gg[q][d] = gl[q][d] = 0.0;
  }
  for (int m = 0; m < nt; ++m) {
    const int64_t f = a.cf[(int64_t)m * nc + i];
    T Qn[5], Gn[15];
    if (a.fR[f] >= 0) {
      const int64_t nb = a.cside[(int64_t)m * nc + i] ? a.fL[f] : a.fR[f];
      const int s0 = 20 * (m + 1);
#pragma unroll
      for (int q = 0; q < 5; ++q) Qn[q] = Seed<T>::at(a.W[q * nc + nb], seed == s0 + q);
#pragma unroll
      for (int j = 0; j < 15; ++j) Gn[j] = Seed<T>::at(a.G[j * nc + nb], seed == s0 + 5 + j);
    } else {
      T G0[15];
#pragma unroll
      for (int j = 0; j < 15; ++j) G0[j] = Seed<T>::at(a.G[j * nc + i], seed == 5 + j);
      const T n[3] = {a.fnrm[f], a.fnrm[nf + f], a.fnrm[2 * nf + f]};
      if (!bc_ghost<T>(a.ftag[f], n, Q0, G0, Qn, Gn, T(ph.gamma), ph.Winf)) set_err(a.err, CGKS_ENAN, (int)i, 1);
    }
    T dQ[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) dQ[q] = Qn[q] - Q0[q];
    // the difference column and the three gradient columns of this neighbour, each added into the
    // coefficient on its own (one fused multiply-add per operator entry)
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      const double k0 = a.Kop[(j * 24 + m) * nc + i];
      const double kx = a.Kop[(j * 24 + 6 + 3 * m) * nc + i];
      const double ky = a.Kop[(j * 24 + 7 + 3 * m) * nc + i];
      const double kz = a.Kop[(j * 24 + 8 + 3 * m) * nc + i];
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        b[q][j] += k0 * dQ[q];
        b[q][j] += kx * Gn[3 * q];
        b[q][j] += ky * Gn[3 * q + 1];
        b[q][j] += kz * Gn[3 * q + 2];
      }
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
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const T* bq = b[q];
    const T a0 = Q0[q] - (bq[3] * M2[0] + bq[4] * M2[1] + bq[5] * M2[2] + bq[6] * M2[3] + bq[7] * M2[4] + bq[8] * M2[5]);
    const T p1[3] = {al * gg[q][0], al * gg[q][1], al * gg[q][2]};
    const T bGG = V23 * (p1[0] * p1[0] + p1[1] * p1[1] + p1[2] * p1[2]);
    const T bLS = V23 * (gl[q][0] * gl[q][0] + gl[q][1] * gl[q][1] + gl[q][2] * gl[q][2]);
    const T beta1 = fmin(bGG, bLS);
    // |Omega|^(2/3) sum_d (avg of (d_d p2)^2) + |Omega|^(4/3) sum_{|a|=2} (D^a p2)^2
    const T v[3][3] = {{2.0 * bq[3], bq[6], bq[8]}, {bq[6], 2.0 * bq[4], bq[7]}, {bq[8], bq[7], 2.0 * bq[5]}};
    T first = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const T* x = v[d];
      const T vMv = M2[0] * x[0] * x[0] + M2[1] * x[1] * x[1] + M2[2] * x[2] * x[2] +
                    2.0 * (M2[3] * x[0] * x[1] + M2[4] * x[1] * x[2] + M2[5] * x[0] * x[2]);
      first += bq[d] * bq[d] + vMv;
    }
    const T second = 4.0 * (bq[3] * bq[3] + bq[4] * bq[4] + bq[5] * bq[5]) + bq[6] * bq[6] + bq[7] * bq[7] + bq[8] * bq[8];
    const T beta2 = V23 * first + V43 * second;
    const T rden = 1.0 / (Q0[q] * Q0[q] + beta1 + 1e-40);
    const T bt1 = beta1 * rden, bt2 = beta2 * rden;
    const T sig = fabs(bt2 - bt1);
    // w_m = g_m (1 + (sig/d_m)^2) with d_m = eps + beta~_m, normalised with one division:
    // w_1 : w_2 = g_1 (d_1^2 + sig^2) d_2^2 : g_2 (d_2^2 + sig^2) d_1^2
    const T d1 = ph.weno_eps + bt1, d2 = ph.weno_eps + bt2;
    const T s2 = sig * sig, d11 = d1 * d1, d22 = d2 * d2;
    const T A1 = g1 * (d11 + s2) * d22, A2 = g2 * (d22 + s2) * d11;
    const T inv = 1.0 / (A1 + A2);
    const T w1 = A1 * inv, w2 = A2 * inv;
    const T c2 = w2 * (1.0 / g2), c1 = w1 - w2 * (g1 / g2);
    out[10 * q + 0] = c2 * a0 + c1 * Q0[q];
#pragma unroll
    for (int d = 0; d < 3; ++d) out[10 * q + 1 + d] = c2 * bq[d] + c1 * p1[d];
#pragma unroll
    for (int j = 3; j < 9; ++j) out[10 * q + 1 + j] = c2 * bq[j];
  }
}

// local time step of cell i from its average Q0: CFL |Omega| / sum_p S_p (|U.n_p| + c + 2 nu S_p / |Omega|)
template <typename T>
HD T time_step(int64_t i, const ReconArgs& a, const T Q0[5]) {
  const int64_t nc = a.nc;
  const int nt = a.ctype[i] == 7 ? 5 : a.ctype[i];
  const Phys& ph = a.ph;
  const T r = 1.0 / Q0[0];
  const T u[3] = {Q0[1] * r, Q0[2] * r, Q0[3] * r};
  const T p = (ph.gamma - 1.0) * (Q0[4] - 0.5 * Q0[0] * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
  const T c = sqrt(ph.gamma * p * r);
  const double V = a.vol[i];
  const T nu2 = ph.viscous ? 2.0 * viscosity<T>(ph, ph.gamma * p * r) * r / V : T(0.0);
  T s = 0.0;
  for (int m = 0; m < nt; ++m) {
    const double S = a.dtw[(4 * m + 3) * nc + i];
    const T un = fabs(u[0] * a.dtw[(4 * m) * nc + i] + u[1] * a.dtw[(4 * m + 1) * nc + i] +
                      u[2] * a.dtw[(4 * m + 2) * nc + i]);
    s += un + S * c + nu2 * S * S;
  }
  if (!(Q0[0] > 0.0) || !(p > 0.0) || !isfinite(Q0[4])) set_err(a.err, CGKS_ENAN, (int)i, 2);
  return ph.cfl_fine * V / s;
}

HD void reconstruct_body(int64_t i, const ReconArgs& a) {
  {
    __align__(16) double out[CGKS_RC];
    reconstruct_cell<double>(i, a, -1, out);
    double2* dst = reinterpret_cast<double2*>(a.rc + (int64_t)CGKS_RC * i);
#pragma unroll
    for (int k = 0; k < CGKS_RC / 2; ++k) dst[k] = make_double2(out[2 * k], out[2 * k + 1]);
  }
  double Q0[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) Q0[q] = a.W[q * a.nc + i];
  a.dt[i] = time_step<double>(i, a, Q0);
}

// forward-mode linearisation of the reconstruction of cell i into Jr [CGKS_RJ_ROWS][nc]: rows
// 51 c + o of the own slot (input c of (W, grad W), output o of (50 coefficients, time step)), then
// for neighbour slot s = 1..6 the rows CGKS_RJ_SELF + ((s - 1) 5 + q) 40 + 10 c4 + j: input c4 of
// (W_q, d/dx, d/dy, d/dz of W_q), output coefficient j of variable q; absent slots (boundary faces,
// fewer faces) are zero
HD void recon_jacobian_body(int64_t i, const ReconArgs& a, double* Jr) {
  const int64_t nc = a.nc;
  const int nt = a.ctype[i] == 7 ? 5 : a.ctype[i];
  for (int k = 0; k < 20; ++k) {
    DualD out[CGKS_RC];
    reconstruct_cell<DualD>(i, a, k, out);
    for (int o = 0; o < CGKS_RC; ++o) Jr[(int64_t)(CGKS_RJ_OUT * k + o) * nc + i] = out[o].d;
    double ddt = 0.0;
    if (k < 5) {
      DualD Q0[5];
      for (int q = 0; q < 5; ++q) Q0[q] = DualD(a.W[q * nc + i], q == k ? 1.0 : 0.0);
      ddt = time_step<DualD>(i, a, Q0).d;
    }
    Jr[(int64_t)(CGKS_RJ_OUT * k + CGKS_RC) * nc + i] = ddt;
  }
  for (int s = 1; s <= 6; ++s) {
    const bool live = s <= nt && a.fR[a.cf[(int64_t)(s - 1) * nc + i]] >= 0;
    for (int c = 0; c < 20; ++c) {
      const int q = c < 5 ? c : (c - 5) / 3, c4 = c < 5 ? 0 : 1 + (c - 5) % 3;
      DualD out[CGKS_RC];
      if (live) reconstruct_cell<DualD>(i, a, 20 * s + c, out);
      const int64_t row = CGKS_RJ_SELF + ((s - 1) * 5 + q) * 40 + 10 * c4;
      for (int j = 0; j < 10; ++j) Jr[(row + j) * nc + i] = live ? out[10 * q + j].d : 0.0;
    }
  }
}

// ---- gas-kinetic point flux -------------------------------------------------------------------

// a Maxwellian in the face frame with the reciprocals and products the moments and slopes need
template <typename T>
struct Maxw {
  T rho, U, V, W;  // density, velocity (normal, tangential 1, tangential 2)
  T r, p, h;       // 1/rho, pressure, h = p/rho = 1/(2 lambda)
  T l2, q2;        // 2 lambda = 1/h, |U|^2 + (K+3) h
  T lr, ckr, hq2;  // 2 lambda / rho, 4 lambda^2 / ((K+3) rho), q2 / 2: the slope solve's coefficients
  T hu2, rH;       // |U|^2 / 2, (E + p) / rho: the Euler-flux derivative's
};

// iK3 = 1/(K+3)
template <typename T>
HD bool make_maxw(const T w[5], T gm1, T K, T iK3, Maxw<T>& g) {
  g.rho = w[0];
  g.r = 1.0 / w[0];
  g.U = w[1] * g.r;
  g.V = w[2] * g.r;
  g.W = w[3] * g.r;
  g.p = gm1 * (w[4] - 0.5 * (w[1] * g.U + w[2] * g.V + w[3] * g.W));
  g.h = g.p * g.r;
  g.l2 = 1.0 / g.h;
  const T u2 = g.U * g.U + g.V * g.V + g.W * g.W;
  g.q2 = u2 + (K + 3.0) * g.h;
  g.lr = g.l2 * g.r;
  g.ckr = g.l2 * g.l2 * iK3 * g.r;
  g.hq2 = 0.5 * g.q2;
  g.hu2 = 0.5 * u2;
  g.rH = (w[4] + g.p) * g.r;
  return w[0] > 0.0 && g.p > 0.0;
}

// <u^0>, <u^1> over u > 0 (side +1) or u < 0 (side -1), normalised by rho:
// 1/2 erfc(-s sqrt(lambda) U) and U <u^0> + s exp(-lambda U^2) / (2 sqrt(pi lambda))
template <typename T>
HD void half_seeds(const Maxw<T>& g, T side, T& m0, T& m1) {
  const T lam = 0.5 * g.l2;
  const T isl = rsqrt_hd(lam);
  const T sl = lam * isl;
  m0 = 0.5 * erfc(-side * sl * g.U);
  m1 = g.U * m0 + side * (0.5 * 0.56418958354775628695) * exp(-lam * g.U * g.U) * isl;
}

// micro-slope s with <s psi> = dW under the full Maxwellian g (closed form of the 5x5 system, with
// d = dW / rho: s4 = 4 lambda^2/(K+3) (2 d4 - q2 d0 - 2 U.(d - U d0)), s_i = 2 lambda (d_i - U_i d0)
// - U_i s4, s0 = d0 - U.s - q2 s4 / 2); the 1/rho of d rides in the coefficients lr and ckr
template <typename T>
HD void slope_solve(const Maxw<T>& g, const T dW[5], T s[5]) {
  const T R1 = dW[1] - g.U * dW[0], R2 = dW[2] - g.V * dW[0], R3 = dW[3] - g.W * dW[0];
  const T R4 = 2.0 * dW[4] - g.q2 * dW[0];
  s[4] = g.ckr * (R4 - 2.0 * (g.U * R1 + g.V * R2 + g.W * R3));
  s[1] = g.lr * R1 - g.U * s[4];
  s[2] = g.lr * R2 - g.V * s[4];
  s[3] = g.lr * R3 - g.W * s[4];
  s[0] = g.r * dW[0] - g.U * s[1] - g.V * s[2] - g.W * s[3] - g.hq2 * s[4];
}

// directional derivative of the Euler flux through the k-th axis of the face frame along dW:
// equals <u_k (a . psi) psi> under the full Maxwellian when <a psi> = dW.  With e_j = rho du_j =
// dW_{1+j} - u_j dW_0: d(rho u_k u_j) = dW_{1+k} u_j + u_k e_j, d(u_k (E + p)) = e_k (E + p)/rho +
// u_k (dE + dp)
template <typename T>
HD void euler_jvp(const Maxw<T>& g, T gm1, int k, const T dW[5], T out[5]) {
  const T u[3] = {g.U, g.V, g.W};
  const T e[3] = {dW[1] - u[0] * dW[0], dW[2] - u[1] * dW[0], dW[3] - u[2] * dW[0]};
  const T dp = gm1 * (dW[4] - (u[0] * dW[1] + u[1] * dW[2] + u[2] * dW[3]) + g.hu2 * dW[0]);
  const T dmk = dW[1 + k];
  out[0] = dmk;
#pragma unroll
  for (int j = 0; j < 3; ++j) out[1 + j] = dmk * u[j] + u[k] * e[j];
  out[1 + k] += dp;
  out[4] = e[k] * g.rH + u[k] * (dW[4] + dp);
}

// gradient (global frame) of a reconstruction polynomial at offset X from its centroid
HD void eval_gradient(const double* rcp, const double X[3], double Gq[15]) {
  const double X2[3] = {2.0 * X[0], 2.0 * X[1], 2.0 * X[2]};
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const double2* c2 = reinterpret_cast<const double2*>(rcp + 10 * q);
    const double2 A = c2[0], B = c2[1], C = c2[2], D = c2[3], E = c2[4];
    // (r0 r1) (r2 r3) (r4 r5) (r6 r7) (r8 r9): 1 X Y Z X^2 Y^2 Z^2 XY YZ XZ
    Gq[3 * q + 0] = A.y + C.x * X2[0] + D.y * X[1] + E.y * X[2];
    Gq[3 * q + 1] = B.x + C.y * X2[1] + D.y * X[0] + E.x * X[2];
    Gq[3 * q + 2] = B.y + D.x * X2[2] + E.x * X[1] + E.y * X[0];
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
template <typename T>
HD void rotate_gradient(const T Gq[15], const T* e[3], T D[3][5]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const T* dir = e[k];
    T gs[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) gs[q] = Gq[3 * q] * dir[0] + Gq[3 * q + 1] * dir[1] + Gq[3 * q + 2] * dir[2];
    D[k][0] = gs[0];
    D[k][4] = gs[4];
#pragma unroll
    for (int j = 0; j < 3; ++j) D[k][1 + j] = e[j][0] * gs[1] + e[j][1] * gs[2] + e[j][2] * gs[3];
  }
}

// ---- moments in the frame moving with the tangential velocity --------------------------------
// With c = v - V, d = w - W (full-space Gaussians of variance h), psi = T psi' where
// psi' = (1, u, c, d, (u^2 + c^2 + d^2 + xi^2)/2) and T adds V, W, (V^2 + W^2)/2 terms.  Odd moments of
// c and d vanish, so the matrices <u^k psi' psi'^T>, <u^k c psi' psi'^T>, <u^k d psi' psi'^T> are sparse;
// a slope s becomes s' = T^T s and a moment vector o' becomes T o'.
template <typename T>
struct MomP {
  T M[7];            // rho <u^k>, k = 0..6 (half or full space)
  T h, sig, tau4;    // h = p/rho, sig = h + <xi^2>/2, tau4 = 2 h^2 + h <xi^2> + <xi^4>/4
  T hs;              // h (2 h + <xi^2>/2)
  T V, W, E;         // tangential velocity and (V^2 + W^2)/2
  // the matrix entries the products below share, formed once per moment set: P_k = M_{k+2}/2 +
  // sig M_k (<u^k psi'_0 psi'_4>; <u^k psi'_1 psi'_4> is P_{k+1}), R_k = M_{k+4}/4 + sig M_{k+2} +
  // tau4 M_k (<u^k psi'_4 psi'_4>), h M_k, and S_k = h M_{k+2}/2 + hs M_k (<u^k c psi'_2 psi'_4>)
  T Pm[4], Rm[3], hM[4], S4[2];
};

template <typename T>
HD void make_momp(const Maxw<T>& g, T m0, T m1, T K, MomP<T>& P) {
  T* M = P.M;
  const T h = g.h;
  M[0] = g.rho * m0;
  M[1] = g.rho * m1;
#pragma unroll
  for (int n = 0; n + 2 < 7; ++n) M[n + 2] = g.U * M[n + 1] + T(n + 1) * h * M[n];
  const T x2 = K * h, x4 = K * (K + 2.0) * h * h;
  P.h = h;
  P.sig = h + 0.5 * x2;
  P.tau4 = 2.0 * h * h + h * x2 + 0.25 * x4;
  P.hs = h * (2.0 * h + 0.5 * x2);
  P.V = g.V;
  P.W = g.W;
  P.E = 0.5 * (g.V * g.V + g.W * g.W);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    P.Pm[k] = 0.5 * M[k + 2] + P.sig * M[k];
    P.hM[k] = h * M[k];
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) P.Rm[k] = 0.25 * M[k + 4] + P.sig * M[k + 2] + P.tau4 * M[k];
#pragma unroll
  for (int k = 0; k < 2; ++k) P.S4[k] = 0.5 * P.hM[k + 2] + P.hs * M[k];
}

// s' = T^T s
template <typename T>
HD void to_primed(const MomP<T>& P, const T s[5], T sp[5]) {
  sp[0] = s[0] + P.V * s[2] + P.W * s[3] + P.E * s[4];
  sp[1] = s[1];
  sp[2] = s[2] + P.V * s[4];
  sp[3] = s[3] + P.W * s[4];
  sp[4] = s[4];
}

// out += T o' (the energy row added term by term, one fused multiply-add each)
template <typename T>
HD void add_from_primed(const MomP<T>& P, const T o[5], T out[5]) {
  out[0] += o[0];
  out[1] += o[1];
  out[2] += P.V * o[0] + o[2];
  out[3] += P.W * o[0] + o[3];
  out[4] += P.E * o[0];
  out[4] += P.V * o[2];
  out[4] += P.W * o[3];
  out[4] += o[4];
}

// out = T o'
template <typename T>
HD void from_primed(const MomP<T>& P, const T o[5], T out[5]) {
  out[0] = o[0];
  out[1] = o[1];
  out[2] = P.V * o[0] + o[2];
  out[3] = P.W * o[0] + o[3];
  out[4] = P.E * o[0] + P.V * o[2] + P.W * o[3] + o[4];
}

// o' = <u^k (s' . psi') psi'>
template <typename T, int k>
HD void papp(const MomP<T>& P, const T s[5], T o[5]) {
  const T* M = P.M;
  const T Pk = P.Pm[k], Qk = P.Pm[k + 1], Rk = P.Rm[k], hM = P.hM[k];
  o[0] = M[k] * s[0] + M[k + 1] * s[1] + Pk * s[4];
  o[1] = M[k + 1] * s[0] + M[k + 2] * s[1] + Qk * s[4];
  o[2] = hM * s[2];
  o[3] = hM * s[3];
  o[4] = Pk * s[0] + Qk * s[1] + Rk * s[4];
}

// o' += <u^k c (s' . psi') psi'> (J = 2) or <u^k d (s' . psi') psi'> (J = 3)
template <typename T, int k, int J>
HD void papp_t_add(const MomP<T>& P, const T s[5], T o[5]) {
  const T hM0 = P.hM[k], hM1 = P.hM[k + 1], S4 = P.S4[k];
  o[0] += hM0 * s[J];
  o[1] += hM1 * s[J];
  o[J] += hM0 * s[0];
  o[J] += hM1 * s[1];
  o[J] += S4 * s[4];
  o[4] += S4 * s[J];
}

// o' = <u^k (a . u) psi'> with the three slopes in primed form: u a_n + v a_t1 + w a_t2,
// v = V + c, w = W + d
template <typename T, int k>
HD void papp_au(const MomP<T>& P, const T an[5], const T a1[5], const T a2[5], T o[5]) {
  T comb[5], t[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) comb[q] = P.V * a1[q] + P.W * a2[q];
  papp<T, k + 1>(P, an, o);
  papp<T, k>(P, comb, t);
#pragma unroll
  for (int q = 0; q < 5; ++q) o[q] += t[q];
  papp_t_add<T, k, 2>(P, a1, o);
  papp_t_add<T, k, 3>(P, a2, o);
}

// one side of the interface: micro-slopes of the initial distribution, its contribution to the
// equilibrium slopes, the time-integrated flux, the state at dt (STATE) and the time-integrated state
template <typename T, bool STATE = true>
HD void side_terms(const T D[3][5], const Maxw<T>& g, T m0, T m1, T K, T gm1, T tau, T q4, T q5, T edt, T dtf, T dWc[3][5],
                   T Facc[5], T Wacc[5], T Iacc[5]) {
  MomP<T> P;
  make_momp<T>(g, m0, m1, K, P);
  T a[3][5];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    T s[5];
    slope_solve<T>(g, D[k], s);
    to_primed<T>(P, s, a[k]);
  }
  // time slope A from <A + a.u> = 0 under the full Maxwellian: <(a.u) psi> = sum_k J_k dW_k
  T Ap[5];
  {
    T t0[5], t1[5], t2[5], au[5], A[5];
    euler_jvp<T>(g, gm1, 0, D[0], t0);
    euler_jvp<T>(g, gm1, 1, D[1], t1);
    euler_jvp<T>(g, gm1, 2, D[2], t2);
#pragma unroll
    for (int q = 0; q < 5; ++q) au[q] = -(t0[q] + t1[q] + t2[q]);
    slope_solve<T>(g, au, A);
    to_primed<T>(P, A, Ap);
  }
  // half-space moments: equilibrium-slope contributions <a_k psi>
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    T t[5];
    papp<T, 0>(P, a[k], t);
    add_from_primed<T>(P, t, dWc[k]);
  }
  // <(a.u) psi>, <u (a.u) psi>, <A psi>, <u A psi>, <psi>, <u psi>
  T Va[5], Fa[5], VA[5], FA[5];
  papp_au<T, 0>(P, a[0], a[1], a[2], Va);
  papp_au<T, 1>(P, a[0], a[1], a[2], Fa);
  papp<T, 0>(P, Ap, VA);
  papp<T, 1>(P, Ap, FA);
  const T* M = P.M;
  const T V0[5] = {M[0], M[1], 0.0, 0.0, 0.5 * M[2] + P.sig * M[0]};
  const T F0[5] = {M[1], M[2], 0.0, 0.0, 0.5 * M[3] + P.sig * M[1]};
  const T tq4 = tau * q4;
  const T etd = edt * (tau + dtf), etau = edt * tau;
  T f[5], s[5], i[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    f[q] = q4 * F0[q] - q5 * Fa[q] - tq4 * FA[q];
    if (STATE) s[q] = edt * V0[q] - etd * Va[q] - etau * VA[q];
    i[q] = q4 * V0[q] - q5 * Va[q] - tq4 * VA[q];
  }
  add_from_primed<T>(P, f, Facc);
  if (STATE) add_from_primed<T>(P, s, Wacc);
  add_from_primed<T>(P, i, Iacc);
}

struct PointArgs {
  int64_t ngp, nf, nc;
  const int32_t *gp_face, *fL, *fR, *ftag;
  const double *gp_x, *gp_A, *fshift, *ctr, *rc, *dt;
  double* gpr;  // [ngp][CGKS_GPR] records: flux x weight / dt (5), interface state (5), area vector (3), alpha
  Phys ph;
  DevErr* err;
};

// inputs of one Gauss point: unit normal n, 1/|weight x area|, face, cells, the left and right
// states and gradients at the point (global frame) and the face's time step
struct PointIn {
  double n[3], iw;
  int64_t f, L, R;
  double WL[5], GL[15], WR[5], GR[15], dtf;
};

HD void point_inputs(int64_t g, const PointArgs& a, PointIn& p) {
  const int64_t ngp = a.ngp, nf = a.nf, nc = a.nc;
  const int64_t f = a.gp_face[g];
  const int64_t L = a.fL[f], R = a.fR[f];
  p.f = f;
  p.L = L;
  p.R = R;
  const double x[3] = {a.gp_x[g], a.gp_x[ngp + g], a.gp_x[2 * ngp + g]};
  const double Av[3] = {a.gp_A[g], a.gp_A[ngp + g], a.gp_A[2 * ngp + g]};
  p.iw = rsqrt_hd(Av[0] * Av[0] + Av[1] * Av[1] + Av[2] * Av[2]);
#pragma unroll
  for (int d = 0; d < 3; ++d) p.n[d] = Av[d] * p.iw;
  const double* rcL = a.rc + (int64_t)CGKS_RC * L;
  const double XL[3] = {x[0] - a.ctr[L], x[1] - a.ctr[nc + L], x[2] - a.ctr[2 * nc + L]};
  eval_value(rcL, XL, p.WL);
  eval_gradient(rcL, XL, p.GL);
  if (R >= 0) {
    const double* rcR = a.rc + (int64_t)CGKS_RC * R;
    double XR[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) XR[d] = x[d] - a.fshift[d * nf + f] - a.ctr[d * nc + R];
    eval_value(rcR, XR, p.WR);
    eval_gradient(rcR, XR, p.GR);
    p.dtf = fmin(a.dt[L], a.dt[R]);
  } else {
    p.dtf = a.dt[L];
  }
}

// the gas-kinetic flux of one Gauss point (flux x weight / dt and interface state x area, both in
// the global frame) and its compression factor, from the point's left and right states and
// gradients; on a boundary face (bnd) the right side is the ghost of the left.  STATE false: the flux
// alone (the interface state and the compression factor, which only the Gauss-Green gradient update
// uses, are left out; Wg is not written and alpha is 1)
template <typename T, bool STATE = true>
HD void point_flux(const double nd[3], double iw, bool bnd, int tag, const T WLg[5], const T GLg[15], const T WRi[5],
                   const T GRi[15], T dtf, const Phys& ph, T Fg[5], T Wg[5], T& alpha, DevErr* err, int64_t f) {
  T n[3], t1[3], t2[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) n[d] = nd[d];
  face_frame<T>(n, t1, t2);
  const T* e[3] = {n, t1, t2};
  const T K = ph.K, gm1 = ph.gamma - 1.0, iK3 = 1.0 / (ph.K + 3.0);
  T WRg[5], GRg[15];
  if (!bnd) {
#pragma unroll
    for (int q = 0; q < 5; ++q) WRg[q] = WRi[q];
#pragma unroll
    for (int j = 0; j < 15; ++j) GRg[j] = GRi[j];
  } else if (!bc_ghost<T>(tag, n, WLg, GLg, WRg, GRg, T(ph.gamma), ph.Winf)) {
    set_err(err, CGKS_ENAN, (int)f, 3);
  }
  T wl[5], wr[5];
  rotate_in<T>(WLg, n, t1, t2, wl);
  rotate_in<T>(WRg, n, t1, t2, wr);
  Maxw<T> gl, gr;
  const bool okl = make_maxw<T>(wl, gm1, K, iK3, gl), okr = make_maxw<T>(wr, gm1, K, iK3, gr);
  if (!(okl && okr)) set_err(err, CGKS_ENAN, (int)f, 4);
  // half-space seeds of both sides, and the interface equilibrium
  // W^c = int_{u>0} psi g^l + int_{u<0} psi g^r (Eq. compatibility2)
  T ml0, ml1, mr0, mr1;
  half_seeds<T>(gl, 1.0, ml0, ml1);
  half_seeds<T>(gr, -1.0, mr0, mr1);
  T wc[5];
  {
    const T ml2 = gl.U * ml1 + gl.h * ml0, mr2 = gr.U * mr1 + gr.h * mr0;
    const T ql = gl.V * gl.V + gl.W * gl.W + (ph.K + 2.0) * gl.h;
    const T qr = gr.V * gr.V + gr.W * gr.W + (ph.K + 2.0) * gr.h;
    wc[0] = gl.rho * ml0 + gr.rho * mr0;
    wc[1] = gl.rho * ml1 + gr.rho * mr1;
    wc[2] = gl.rho * gl.V * ml0 + gr.rho * gr.V * mr0;
    wc[3] = gl.rho * gl.W * ml0 + gr.rho * gr.W * mr0;
    wc[4] = 0.5 * (gl.rho * (ml2 + ml0 * ql) + gr.rho * (mr2 + mr0 * qr));
  }
  Maxw<T> gc;
  if (!make_maxw<T>(wc, gm1, K, iK3, gc)) set_err(err, CGKS_ENAN, (int)f, 5);
  // collision times (Sec. 2.3)
  const T jump = fabs((gl.p - gr.p) / (gl.p + gr.p));
  T tau, tn;
  if (ph.viscous) {
    tau = viscosity<T>(ph, ph.gamma * gc.h) * (gc.r * gc.l2);  // mu(T^c) / p^c, p^c/rho^c = 1/(2 lambda^c)
    tn = tau + ph.c_press * jump * dtf;
  } else {
    tn = (ph.eps_inviscid + ph.c_press * jump) * dtf;
    tau = tn;
  }
  // exact integrals over [0, dt] of the time coefficients of Eq. 2nd-flux
  const T edt = exp(-dtf / tn), om = 1.0 - edt;
  const T q1 = dtf - tn * om;
  const T q2 = (tn * tn + tau * tn) * om - tn * dtf * edt - tau * dtf;
  const T q3 = 0.5 * dtf * dtf - tau * dtf + tau * tn * om;
  const T q4 = tn * om;
  const T q5 = (tau * tn + tn * tn) * om - tn * dtf * edt;
  // compression factor of this Gauss point (interior faces only), 1/p = l2 / rho
  alpha = 1.0;
  if (STATE && !bnd && ph.cf) {
    const T icl = rsqrt_hd(ph.gamma * gl.h), icr = rsqrt_hd(ph.gamma * gr.h);
    const T dp = fabs(gl.p - gr.p);
    const T dn = gl.U * icl - gr.U * icr, d1 = gl.V * icl - gr.V * icr, d2 = gl.W * icl - gr.W * icr;
    const T A = dp * (gl.r * gl.l2 + gr.r * gr.l2) + dn * dn + (d1 * d1 + d2 * d2);
    alpha = 1.0 / (1.0 + A * A);
  }
  T dWc[3][5], Facc[5], Wacc[5], Iacc[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    dWc[0][q] = dWc[1][q] = dWc[2][q] = 0.0;
    Facc[q] = Wacc[q] = Iacc[q] = 0.0;
  }
  {
    T D[3][5];
    rotate_gradient<T>(GLg, e, D);
    side_terms<T, STATE>(D, gl, ml0, ml1, K, gm1, tau, q4, q5, edt, dtf, dWc, Facc, Wacc, Iacc);
    rotate_gradient<T>(GRg, e, D);
    side_terms<T, STATE>(D, gr, mr0, mr1, K, gm1, tau, q4, q5, edt, dtf, dWc, Facc, Wacc, Iacc);
  }
  // equilibrium part: slopes a^c from the kinetic-weighted interface gradients; A^c from
  // <A + a.u> = 0; full-space moments through the Euler-flux Jacobians
  T ac[3][5];
#pragma unroll
  for (int k = 0; k < 3; ++k) slope_solve<T>(gc, dWc[k], ac[k]);
  T cu[5];  // <(a^c . u) psi>_c = sum_k J_k dW^c_k
  {
    T u0[5], u1[5], u2[5];
    euler_jvp<T>(gc, gm1, 0, dWc[0], u0);
    euler_jvp<T>(gc, gm1, 1, dWc[1], u1);
    euler_jvp<T>(gc, gm1, 2, dWc[2], u2);
#pragma unroll
    for (int q = 0; q < 5; ++q) cu[q] = u0[q] + u1[q] + u2[q];
  }
  T Fc0[5], FcA[5], Fca[5];
  {
    // <u psi>_c is the Euler flux of W^c; <u A^c psi>_c = J_n <A^c psi>_c = -J_n <(a^c . u) psi>_c
    Fc0[0] = wc[1];
    Fc0[1] = wc[1] * gc.U + gc.p;
    Fc0[2] = wc[2] * gc.U;
    Fc0[3] = wc[3] * gc.U;
    Fc0[4] = (wc[4] + gc.p) * gc.U;
    euler_jvp<T>(gc, gm1, 0, cu, FcA);
#pragma unroll
    for (int q = 0; q < 5; ++q) FcA[q] = -FcA[q];
    // <u (a^c . u) psi>_c in the frame moving with the tangential velocity
    MomP<T> P;
    make_momp<T>(gc, 1.0, gc.U, K, P);
    T a0[5], a1[5], a2[5], o[5];
    to_primed<T>(P, ac[0], a0);
    to_primed<T>(P, ac[1], a1);
    to_primed<T>(P, ac[2], a2);
    papp_au<T, 1>(P, a0, a1, a2, o);
    from_primed<T>(P, o, Fca);
  }
  const T q23 = q2 - q3;
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    Facc[q] += q1 * Fc0[q];
    Facc[q] += q2 * Fca[q];
    Facc[q] += q3 * FcA[q];
    if (STATE) Wacc[q] += om * (wc[q] - dtf * cu[q]);
    Iacc[q] += q1 * wc[q];
    Iacc[q] += q23 * cu[q];
  }
  if (ph.viscous && ph.prandtl != 1.0) {
    // heat flux about U^c of the time-integrated distribution, scaled by (1/Pr - 1)
    const T Ub[3] = {gc.U, gc.V, gc.W};
    const T U2 = Ub[0] * Ub[0] + Ub[1] * Ub[1] + Ub[2] * Ub[2];
    const T qn = Facc[4] - (Ub[0] * Facc[1] + Ub[1] * Facc[2] + Ub[2] * Facc[3]) + 0.5 * U2 * Facc[0] -
                 Ub[0] * (Iacc[4] - (Ub[0] * Iacc[1] + Ub[1] * Iacc[2] + Ub[2] * Iacc[3]) + 0.5 * U2 * Iacc[0]);
    Facc[4] += (1.0 / ph.prandtl - 1.0) * qn;
  }
  const T sdt = 1.0 / (iw * dtf);  // weight / dt
#pragma unroll
  for (int q = 0; q < 5; ++q) Facc[q] *= sdt;
  rotate_out<T>(Facc, n, t1, t2, Fg);
  if (STATE) rotate_out<T>(Wacc, n, t1, t2, Wg);
}

// one contiguous record per point, so that the gather reads a face's points as one segment; STATE
// false (the defect of the V-cycle): the flux alone, in the record's first five entries
template <bool STATE = true>
HD void gks_point_body(int64_t g, const PointArgs& a) {
  PointIn p;
  point_inputs(g, a, p);
  double Fg[5], Wg[5], alpha;
  point_flux<double, STATE>(p.n, p.iw, p.R < 0, a.ftag[p.f], p.WL, p.GL, p.WR, p.GR, p.dtf, a.ph, Fg, Wg, alpha, a.err,
                            p.f);
  const int64_t ngp = a.ngp;
  double2* dst = reinterpret_cast<double2*>(a.gpr + (int64_t)CGKS_GPR * g);
  dst[0] = make_double2(Fg[0], Fg[1]);
  dst[1] = make_double2(Fg[2], Fg[3]);
  if (!STATE) {
    a.gpr[(int64_t)CGKS_GPR * g + 4] = Fg[4];
    return;
  }
  dst[2] = make_double2(Fg[4], Wg[0]);
  dst[3] = make_double2(Wg[1], Wg[2]);
  dst[4] = make_double2(Wg[3], Wg[4]);
  dst[5] = make_double2(a.gp_A[g], a.gp_A[ngp + g]);
  dst[6] = make_double2(a.gp_A[2 * ngp + g], alpha);
}

// forward-mode linearisation of one Gauss point: Jp[(10 k + o) ngp + g] = d out_o / d in_k with
// inputs k = (W_L 5, grad W_L 15, W_R 5, grad W_R 15, dt_f) at the point and outputs o = (flux 5,
// interface state 5) as gks_point_body stores them; the right-side columns of a boundary point
// are zero (its ghost is a function of the left side)
HD void point_jacobian_body(int64_t g, const PointArgs& a, double* Jp) {
  PointIn p;
  point_inputs(g, a, p);
  const bool bnd = p.R < 0;
  const int tag = a.ftag[p.f];
  const int64_t ngp = a.ngp;
  for (int k = 0; k < CGKS_PJ_IN; ++k) {
    double col[10];
    if (bnd && k >= 20 && k < 40) {
#pragma unroll
      for (int o = 0; o < 10; ++o) col[o] = 0.0;
    } else {
      DualD WL[5], GL[15], WR[5], GR[15], Fg[5], Wg[5], al;
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        WL[q] = DualD(p.WL[q], k == q ? 1.0 : 0.0);
        WR[q] = DualD(bnd ? 0.0 : p.WR[q], k == 20 + q ? 1.0 : 0.0);
      }
#pragma unroll
      for (int j = 0; j < 15; ++j) {
        GL[j] = DualD(p.GL[j], k == 5 + j ? 1.0 : 0.0);
        GR[j] = DualD(bnd ? 0.0 : p.GR[j], k == 25 + j ? 1.0 : 0.0);
      }
      const DualD dtf(p.dtf, k == 40 ? 1.0 : 0.0);
      point_flux<DualD>(p.n, p.iw, bnd, tag, WL, GL, WR, GR, dtf, a.ph, Fg, Wg, al, a.err, p.f);
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        col[q] = Fg[q].d;
        col[5 + q] = Wg[q].d;
      }
    }
#pragma unroll
    for (int o = 0; o < 10; ++o) Jp[(int64_t)(10 * k + o) * ngp + g] = col[o];
  }
}

struct GatherArgs {
  int64_t nc, ngp;
  const int8_t *ctype, *cside;
  const int32_t *cf, *gp_ptr;
  const double *gpr, *vol, *dt, *W_in;
  double *W_out, *res, *G_out, *alpha_out;
  int update;
  double gamma;
  DevErr* err;
};

// running sums of one cell: residual, Gauss-Green gradient sums, compression-factor product
struct GatherAcc {
  double r[5], gs[15], al;
};

HD void gather_init(GatherAcc& c) {
#pragma unroll
  for (int q = 0; q < 5; ++q) c.r[q] = 0.0;
#pragma unroll
  for (int j = 0; j < 15; ++j) c.gs[j] = 0.0;
  c.al = 1.0;
}

// x with its sign bit xor-ed with `mask` (0 or the sign bit): an exact change of sign done by an
// integer operation, so that it takes no FP64 issue slot (those bound the gather on GB300)
HD double xor_sign(double x, uint64_t mask) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)mask);
#else
  uint64_t u;
  memcpy(&u, &x, sizeof u);
  u ^= mask;
  memcpy(&x, &u, sizeof x);
  return x;
#endif
}

// adds the ng consecutive Gauss-point records `rec` of one face, seen from its left cell (right:
// false) or from its right cell (the flux and the area vector change sign), in ascending point order
template <bool GRAD = true>
HD void gather_face(const double* rec, int ng, bool right, GatherAcc& c) {
  const uint64_t m = right ? 0x8000000000000000ull : 0ull;
  for (int k = 0; k < ng; ++k) {
    const double* v = rec + (int64_t)CGKS_GPR * k;
    if (!GRAD) {  // the residual alone (the defect of the V-cycle)
#pragma unroll
      for (int q = 0; q < 5; ++q) c.r[q] -= xor_sign(v[q], m);
      continue;
    }
    const double A[3] = {xor_sign(v[10], m), xor_sign(v[11], m), xor_sign(v[12], m)};
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      c.r[q] -= xor_sign(v[q], m);
      const double wq = v[5 + q];
#pragma unroll
      for (int d = 0; d < 3; ++d) c.gs[3 * q + d] += wq * A[d];
    }
    c.al *= v[13];
  }
}

// the cell's outputs from its sums: residual, alpha x Gauss-Green gradient / |Omega|, alpha, and
// the optional explicit update W += dt/|Omega| Res
HD void gather_store(int64_t i, const GatherArgs& a, const GatherAcc& c) {
  const int64_t nc = a.nc;
  const double rv = 1.0 / a.vol[i];
  if (a.res)
#pragma unroll
    for (int q = 0; q < 5; ++q) a.res[q * nc + i] = c.r[q];
  if (a.G_out) {
    const double k = c.al * rv;
#pragma unroll
    for (int j = 0; j < 15; ++j) a.G_out[j * nc + i] = k * c.gs[j];
  }
  if (a.alpha_out) a.alpha_out[i] = c.al;
  if (a.update) {
    const double h = a.dt[i] * rv;
    double w[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      w[q] = a.W_in[q * nc + i] + h * c.r[q];
      a.W_out[q * nc + i] = w[q];
    }
    const double p = (a.gamma - 1.0) * (w[4] - 0.5 * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]) / w[0]);
    if (!(w[0] > 0.0) || !(p > 0.0) || !isfinite(p)) set_err(a.err, CGKS_ENAN, (int)i, 6);
  }
}

// the gather of cell i, one face after the other in local-face order (the reference order: the
// device kernel stages the same records through shared memory and sums them in the same order)
HD void gather_body(int64_t i, const GatherArgs& a) {
  const int64_t nc = a.nc;
  GatherAcc c;
  gather_init(c);
  const int nt = a.ctype[i] == 7 ? 5 : a.ctype[i];  // faces: pyramids (type 7) have 5
  for (int m = 0; m < nt; ++m) {
    const int64_t f = a.cf[(int64_t)m * nc + i];
    const int64_t g0 = a.gp_ptr[f];
    const double* rec = a.gpr + (int64_t)CGKS_GPR * g0;
    const int ng = (int)(a.gp_ptr[f + 1] - g0);
    const bool right = a.cside[(int64_t)m * nc + i] != 0;
    if (a.G_out || a.alpha_out || a.update)
      gather_face<true>(rec, ng, right, c);
    else
      gather_face<false>(rec, ng, right, c);
  }
  gather_store(i, a, c);
}
