/* Oracle gas-kinetic solver at one point of a cell interface (Sec. 2.1 and 2.3 of the paper).
 * TEST INFRASTRUCTURE ONLY.
 *
 * Everything is computed from the definitions: every moment <...> is a sum over explicit monomials
 * u^a v^b w^c (xi^2)^d of the factorised Gaussian moments (Eq. co-moment), the micro-slopes solve the
 * 5x5 moment systems of Eq. co by Gaussian elimination, W^c is the half-space sum of Eq.
 * compatibility2, and the flux is the time integral over [0, dt] of the u-moment of Eq. 2nd-flux,
 * using the exact integrals of its time coefficients.
 *
 * Readings (paper silent/garbled):
 *  - gradients of the equilibrium state at the interface are kinetic-weighted, in the same way as
 *    W^c:  dW^c/dx_i = int_{u>0} psi a^l_i g^l + int_{u<0} psi a^r_i g^r (parity unpinned: the
 *    paper prints no number for this choice; its half-space terms are pinned by quadrature);
 *  - inviscid flow: tau := tau_n (Sec. 2.3 numerical collision time) in every term; viscous flow:
 *    tau = mu / p^c in the polynomial terms, tau_n = tau + C |p_l - p_r|/(p_l + p_r) dt in the
 *    exponentials;
 *  - Prandtl number: the BGK model gives Pr = 1 (Eq. ce-ns); for Pr != 1 the time-integrated
 *    energy flux is corrected by (1/Pr - 1) times the time-integrated heat flux about the
 *    interface velocity U^c (parity unpinned beyond its smooth-flow Chapman-Enskog form);
 *  - local frame (n, t1, t2) by the branchless orthonormal basis of Duff et al. (JCGT 2017).
 */
#include <math.h>
#include <string.h>
#include "orc.h"

typedef struct {
  double c;
  int a, b, e, d;
} term;
static const term PSI[5][4] = {
    {{1.0, 0, 0, 0, 0}},
    {{1.0, 1, 0, 0, 0}},
    {{1.0, 0, 1, 0, 0}},
    {{1.0, 0, 0, 1, 0}},
    {{0.5, 2, 0, 0, 0}, {0.5, 0, 2, 0, 0}, {0.5, 0, 0, 2, 0}, {0.5, 0, 0, 0, 1}},
};
static const int PSI_N[5] = {1, 1, 1, 1, 4};

/* 1D Gaussian moments <u^n> (full or half space in u), <v^n>, <w^n>, <xi^(2d)>, normalised by rho */
void orc_moments(const orc_maxw* g, double K, int space, orc_mom* m) {
  double lam = g->lam, U = g->U;
  m->rho = g->rho;
  if (space == 0) {
    m->mu[0] = 1.0;
    m->mu[1] = U;
  } else if (space > 0) {
    m->mu[0] = 0.5 * erfc(-sqrt(lam) * U);
    m->mu[1] = U * m->mu[0] + 0.5 * exp(-lam * U * U) / sqrt(M_PI * lam);
  } else {
    m->mu[0] = 0.5 * erfc(sqrt(lam) * U);
    m->mu[1] = U * m->mu[0] - 0.5 * exp(-lam * U * U) / sqrt(M_PI * lam);
  }
  for (int n = 0; n + 2 < 9; ++n) m->mu[n + 2] = U * m->mu[n + 1] + (n + 1) / (2.0 * lam) * m->mu[n];
  m->mv[0] = 1.0;
  m->mv[1] = g->V;
  m->mw[0] = 1.0;
  m->mw[1] = g->W;
  for (int n = 0; n + 2 < 7; ++n) {
    m->mv[n + 2] = g->V * m->mv[n + 1] + (n + 1) / (2.0 * lam) * m->mv[n];
    m->mw[n + 2] = g->W * m->mw[n + 1] + (n + 1) / (2.0 * lam) * m->mw[n];
  }
  m->mxi[0] = 1.0;
  m->mxi[1] = K / (2.0 * lam);
  m->mxi[2] = K * (K + 2.0) / (4.0 * lam * lam);
}

static double mono(const orc_mom* m, int a, int b, int c, int d) {
  return m->rho * m->mu[a] * m->mv[b] * m->mw[c] * m->mxi[d];
}

/* int u^ku v^kv w^kw (s . psi) psi_alpha g dXi  (s == NULL means s . psi := 1) */
double orc_mom_term(const orc_mom* m, int ku, int kv, int kw, const double* s, int alpha) {
  double acc = 0.0;
  for (int i = 0; i < PSI_N[alpha]; ++i) {
    const term* ta = &PSI[alpha][i];
    if (!s) {
      acc += ta->c * mono(m, ku + ta->a, kv + ta->b, kw + ta->e, ta->d);
      continue;
    }
    for (int beta = 0; beta < 5; ++beta)
      for (int j = 0; j < PSI_N[beta]; ++j) {
        const term* tb = &PSI[beta][j];
        acc += s[beta] * tb->c * ta->c *
               mono(m, ku + ta->a + tb->a, kv + ta->b + tb->b, kw + ta->e + tb->e, ta->d + tb->d);
      }
  }
  return acc;
}

int orc_prim_from_cons(const double W[5], double gamma, orc_maxw* g) {
  double rho = W[0];
  if (!(rho > 0.0)) return -1;
  double U = W[1] / rho, V = W[2] / rho, Wv = W[3] / rho;
  double p = (gamma - 1.0) * (W[4] - 0.5 * rho * (U * U + V * V + Wv * Wv));
  if (!(p > 0.0)) return -1;
  g->rho = rho;
  g->U = U;
  g->V = V;
  g->W = Wv;
  g->lam = rho / (2.0 * p);
  return 0;
}

/* micro-slope s with <s psi> = dW under the full-space Maxwellian g (Eq. co) */
int orc_slope(const orc_maxw* g, double K, const double dW[5], double s[5]) {
  orc_mom m;
  orc_moments(g, K, 0, &m);
  double M[25];
  for (int a = 0; a < 5; ++a)
    for (int b = 0; b < 5; ++b) {
      double e[5] = {0, 0, 0, 0, 0};
      e[b] = 1.0;
      M[5 * a + b] = orc_mom_term(&m, 0, 0, 0, e, a);
    }
  return orc_ge_solve(5, M, dW, s);
}

void orc_frame(const double n[3], double t1[3], double t2[3]) {
  double sign = copysign(1.0, n[2]);
  double a = -1.0 / (sign + n[2]);
  double b = n[0] * n[1] * a;
  t1[0] = 1.0 + sign * n[0] * n[0] * a;
  t1[1] = sign * b;
  t1[2] = -sign * n[0];
  t2[0] = b;
  t2[1] = sign + n[1] * n[1] * a;
  t2[2] = -n[1];
}

/* exact integrals over [0, dt] of the time coefficients of Eq. 2nd-flux */
double orc_viscosity(const orc_phys* ph, double t) {
  if (ph->sutherland == 0.0) return ph->mu;
  return ph->mu * pow(t, 1.5) * (1.0 + ph->sutherland) / (t + ph->sutherland);
}

void orc_time_integrals(double dt, double tau, double tn, double q[5]) {
  double e = exp(-dt / tn);
  q[0] = dt - tn * (1.0 - e);                                    /* 1 - e^{-t/tn}           */
  q[1] = (tn * tn + tau * tn) * (1.0 - e) - tn * dt * e - tau * dt; /* (t + tau) e^{-t/tn} - tau */
  q[2] = 0.5 * dt * dt - tau * dt + tau * tn * (1.0 - e);        /* t - tau + tau e^{-t/tn} */
  q[3] = tn * (1.0 - e);                                         /* e^{-t/tn}               */
  q[4] = (tau * tn + tn * tn) * (1.0 - e) - tn * dt * e;         /* (tau + t) e^{-t/tn}     */
}

static void rotate_in(const double W[5], const double n[3], const double t1[3], const double t2[3], double Wl[5]) {
  Wl[0] = W[0];
  Wl[1] = W[1] * n[0] + W[2] * n[1] + W[3] * n[2];
  Wl[2] = W[1] * t1[0] + W[2] * t1[1] + W[3] * t1[2];
  Wl[3] = W[1] * t2[0] + W[2] * t2[1] + W[3] * t2[2];
  Wl[4] = W[4];
}
static void rotate_out(const double Fl[5], const double n[3], const double t1[3], const double t2[3], double F[5]) {
  F[0] = Fl[0];
  for (int d = 0; d < 3; ++d) F[1 + d] = Fl[1] * n[d] + Fl[2] * t1[d] + Fl[3] * t2[d];
  F[4] = Fl[4];
}
/* directional derivatives along (n, t1, t2) of the rotated conservative variables */
static void rotate_grad(const double G[15], const double* e[3], double D[3][5]) {
  for (int k = 0; k < 3; ++k) {
    const double* dir = e[k];
    for (int q = 0; q < 5; q += 4) {
      double s = 0.0;
      for (int d = 0; d < 3; ++d) s += G[3 * q + d] * dir[d];
      D[k][q] = s;
    }
    for (int a = 0; a < 3; ++a) {
      double s = 0.0;
      for (int i = 0; i < 3; ++i)
        for (int d = 0; d < 3; ++d) s += e[a][i] * G[3 * (1 + i) + d] * dir[d];
      D[k][1 + a] = s;
    }
  }
}

int orc_gks_point(const orc_phys* ph, const double WL[5], const double GL[15], const double WR[5],
                  const double GR[15], const double n[3], double dt, double F[5], double Wt[5]) {
  const double K = ph->K;
  double t1[3], t2[3];
  orc_frame(n, t1, t2);
  const double* e[3] = {n, t1, t2};
  double wl[5], wr[5], dl[3][5], dr[3][5];
  rotate_in(WL, n, t1, t2, wl);
  rotate_in(WR, n, t1, t2, wr);
  rotate_grad(GL, e, dl);
  rotate_grad(GR, e, dr);
  orc_maxw gl, gr, gc;
  if (orc_prim_from_cons(wl, ph->gamma, &gl) || orc_prim_from_cons(wr, ph->gamma, &gr)) return -1;
  orc_mom ml, mlp, mr, mrn, mc;
  orc_moments(&gl, K, 0, &ml);
  orc_moments(&gl, K, +1, &mlp);
  orc_moments(&gr, K, 0, &mr);
  orc_moments(&gr, K, -1, &mrn);
  /* interface equilibrium state (Eq. compatibility2) */
  double wc[5];
  for (int a = 0; a < 5; ++a) wc[a] = orc_mom_term(&mlp, 0, 0, 0, NULL, a) + orc_mom_term(&mrn, 0, 0, 0, NULL, a);
  if (orc_prim_from_cons(wc, ph->gamma, &gc)) return -1;
  orc_moments(&gc, K, 0, &mc);
  /* micro-slopes of the initial states and their time derivatives (Eq. co) */
  double al[3][5], ar[3][5], Al[5], Ar[5], ac[3][5], Ac[5], rhs[5];
  for (int k = 0; k < 3; ++k) {
    if (orc_slope(&gl, K, dl[k], al[k]) || orc_slope(&gr, K, dr[k], ar[k])) return -2;
  }
  for (int a = 0; a < 5; ++a)
    rhs[a] = -(orc_mom_term(&ml, 1, 0, 0, al[0], a) + orc_mom_term(&ml, 0, 1, 0, al[1], a) +
               orc_mom_term(&ml, 0, 0, 1, al[2], a));
  if (orc_slope(&gl, K, rhs, Al)) return -2;
  for (int a = 0; a < 5; ++a)
    rhs[a] = -(orc_mom_term(&mr, 1, 0, 0, ar[0], a) + orc_mom_term(&mr, 0, 1, 0, ar[1], a) +
               orc_mom_term(&mr, 0, 0, 1, ar[2], a));
  if (orc_slope(&gr, K, rhs, Ar)) return -2;
  /* equilibrium slopes (kinetic-weighted interface gradients) */
  for (int k = 0; k < 3; ++k) {
    double dwc[5];
    for (int a = 0; a < 5; ++a) dwc[a] = orc_mom_term(&mlp, 0, 0, 0, al[k], a) + orc_mom_term(&mrn, 0, 0, 0, ar[k], a);
    if (orc_slope(&gc, K, dwc, ac[k])) return -2;
  }
  for (int a = 0; a < 5; ++a)
    rhs[a] = -(orc_mom_term(&mc, 1, 0, 0, ac[0], a) + orc_mom_term(&mc, 0, 1, 0, ac[1], a) +
               orc_mom_term(&mc, 0, 0, 1, ac[2], a));
  if (orc_slope(&gc, K, rhs, Ac)) return -2;
  /* collision times (Sec. 2.3) */
  double pl = wl[0] / (2.0 * gl.lam), pr = wr[0] / (2.0 * gr.lam), pc = wc[0] / (2.0 * gc.lam);
  double jump = fabs((pl - pr) / (pl + pr));
  double tau, tn;
  if (ph->viscous) {
    tau = orc_viscosity(ph, ph->gamma * pc / wc[0]) / pc; /* mu(T^c) / p^c */
    tn = tau + ph->c_press * jump * dt;
  } else {
    tn = ph->eps_inviscid * dt + ph->c_press * jump * dt;
    tau = tn;
  }
  double q[5];
  orc_time_integrals(dt, tau, tn, q);
  double Fi[5], Wi[5], Wd[5];
  double e_ = exp(-dt / tn);
  for (int a = 0; a < 5; ++a) {
    double Fc0 = orc_mom_term(&mc, 1, 0, 0, NULL, a);
    double Fc1 = orc_mom_term(&mc, 2, 0, 0, ac[0], a) + orc_mom_term(&mc, 1, 1, 0, ac[1], a) +
                 orc_mom_term(&mc, 1, 0, 1, ac[2], a);
    double Fc2 = orc_mom_term(&mc, 1, 0, 0, Ac, a);
    double Fl0 = orc_mom_term(&mlp, 1, 0, 0, NULL, a);
    double Fl1 = orc_mom_term(&mlp, 2, 0, 0, al[0], a) + orc_mom_term(&mlp, 1, 1, 0, al[1], a) +
                 orc_mom_term(&mlp, 1, 0, 1, al[2], a);
    double Fl2 = orc_mom_term(&mlp, 1, 0, 0, Al, a);
    double Fr0 = orc_mom_term(&mrn, 1, 0, 0, NULL, a);
    double Fr1 = orc_mom_term(&mrn, 2, 0, 0, ar[0], a) + orc_mom_term(&mrn, 1, 1, 0, ar[1], a) +
                 orc_mom_term(&mrn, 1, 0, 1, ar[2], a);
    double Fr2 = orc_mom_term(&mrn, 1, 0, 0, Ar, a);
    double Wc0 = orc_mom_term(&mc, 0, 0, 0, NULL, a);
    double Wc1 = orc_mom_term(&mc, 1, 0, 0, ac[0], a) + orc_mom_term(&mc, 0, 1, 0, ac[1], a) +
                 orc_mom_term(&mc, 0, 0, 1, ac[2], a);
    double Wc2 = orc_mom_term(&mc, 0, 0, 0, Ac, a);
    double Wl0 = orc_mom_term(&mlp, 0, 0, 0, NULL, a);
    double Wl1 = orc_mom_term(&mlp, 1, 0, 0, al[0], a) + orc_mom_term(&mlp, 0, 1, 0, al[1], a) +
                 orc_mom_term(&mlp, 0, 0, 1, al[2], a);
    double Wl2 = orc_mom_term(&mlp, 0, 0, 0, Al, a);
    double Wr0 = orc_mom_term(&mrn, 0, 0, 0, NULL, a);
    double Wr1 = orc_mom_term(&mrn, 1, 0, 0, ar[0], a) + orc_mom_term(&mrn, 0, 1, 0, ar[1], a) +
                 orc_mom_term(&mrn, 0, 0, 1, ar[2], a);
    double Wr2 = orc_mom_term(&mrn, 0, 0, 0, Ar, a);
    Fi[a] = q[0] * Fc0 + q[1] * Fc1 + q[2] * Fc2 + q[3] * (Fl0 + Fr0) - q[4] * (Fl1 + Fr1) -
            tau * q[3] * (Fl2 + Fr2);
    Wi[a] = q[0] * Wc0 + q[1] * Wc1 + q[2] * Wc2 + q[3] * (Wl0 + Wr0) - q[4] * (Wl1 + Wr1) -
            tau * q[3] * (Wl2 + Wr2);
    Wd[a] = (1.0 - e_) * Wc0 + ((dt + tau) * e_ - tau) * Wc1 + (dt - tau + tau * e_) * Wc2 +
            e_ * (Wl0 + Wr0) - e_ * (tau + dt) * (Wl1 + Wr1) - e_ * tau * (Wl2 + Wr2);
  }
  if (ph->viscous && ph->prandtl != 1.0) {
    double Ub[3] = {gc.U, gc.V, gc.W};
    double U2 = Ub[0] * Ub[0] + Ub[1] * Ub[1] + Ub[2] * Ub[2];
    double qn = Fi[4] - (Ub[0] * Fi[1] + Ub[1] * Fi[2] + Ub[2] * Fi[3]) + 0.5 * U2 * Fi[0] -
                Ub[0] * (Wi[4] - (Ub[0] * Wi[1] + Ub[1] * Wi[2] + Ub[2] * Wi[3]) + 0.5 * U2 * Wi[0]);
    Fi[4] += (1.0 / ph->prandtl - 1.0) * qn;
  }
  double Fl[5];
  for (int a = 0; a < 5; ++a) Fl[a] = Fi[a] / dt;
  rotate_out(Fl, n, t1, t2, F);
  rotate_out(Wd, n, t1, t2, Wt);
  return 0;
}

int orc_kfvs_point(const orc_phys* ph, const double WL[5], const double WR[5], const double n[3], double F[5]) {
  double t1[3], t2[3], wl[5], wr[5], Fl[5];
  orc_frame(n, t1, t2);
  rotate_in(WL, n, t1, t2, wl);
  rotate_in(WR, n, t1, t2, wr);
  orc_maxw gl, gr;
  if (orc_prim_from_cons(wl, ph->gamma, &gl) || orc_prim_from_cons(wr, ph->gamma, &gr)) return -1;
  orc_mom mlp, mrn;
  orc_moments(&gl, ph->K, +1, &mlp);
  orc_moments(&gr, ph->K, -1, &mrn);
  for (int a = 0; a < 5; ++a) Fl[a] = orc_mom_term(&mlp, 1, 0, 0, NULL, a) + orc_mom_term(&mrn, 1, 0, 0, NULL, a);
  rotate_out(Fl, n, t1, t2, F);
  return 0;
}

/* compression factor at one Gauss point (Sec. 3.3) */
double orc_cf_alpha(const orc_phys* ph, const double WL[5], const double WR[5], const double n[3]) {
  double t1[3], t2[3], wl[5], wr[5];
  orc_frame(n, t1, t2);
  rotate_in(WL, n, t1, t2, wl);
  rotate_in(WR, n, t1, t2, wr);
  orc_maxw gl, gr;
  if (orc_prim_from_cons(wl, ph->gamma, &gl) || orc_prim_from_cons(wr, ph->gamma, &gr)) return 0.0;
  double pl = gl.rho / (2.0 * gl.lam), pr = gr.rho / (2.0 * gr.lam);
  double cl = sqrt(ph->gamma * pl / gl.rho), cr = sqrt(ph->gamma * pr / gr.rho);
  double dp = fabs(pl - pr);
  double dn = gl.U / cl - gr.U / cr, d1 = gl.V / cl - gr.V / cr, d2 = gl.W / cl - gr.W / cr;
  double A = dp / pl + dp / pr + dn * dn + (d1 * d1 + d2 * d2);
  return 1.0 / (1.0 + A * A);
}

/* ghost state (and gradient) of a boundary face with outward unit normal n */
int orc_bc_ghost(const orc_phys* ph, int tag, const double n[3], const double W[5], const double G[15],
                 double Wg[5], double Gg[15]) {
  const double g = ph->gamma;
  double R[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) R[i][j] = (i == j ? 1.0 : 0.0) - 2.0 * n[i] * n[j];
  if (tag == 1 || tag == 2) {
    double mn = W[1] * n[0] + W[2] * n[1] + W[3] * n[2];
    Wg[0] = W[0];
    Wg[4] = W[4];
    for (int d = 0; d < 3; ++d) Wg[1 + d] = tag == 1 ? W[1 + d] - 2.0 * mn * n[d] : -W[1 + d];
    if (Gg) {
      for (int q = 0; q < 5; q += 4)
        for (int d = 0; d < 3; ++d) {
          double s = 0.0;
          for (int e = 0; e < 3; ++e) s += R[d][e] * G[3 * q + e];
          Gg[3 * q + d] = s;
        }
      for (int i = 0; i < 3; ++i)
        for (int d = 0; d < 3; ++d) {
          double s = 0.0;
          if (tag == 1) {
            for (int j = 0; j < 3; ++j)
              for (int e = 0; e < 3; ++e) s += R[i][j] * G[3 * (1 + j) + e] * R[e][d];
          } else {
            for (int e = 0; e < 3; ++e) s -= G[3 * (1 + i) + e] * R[e][d];
          }
          Gg[3 * (1 + i) + d] = s;
        }
    }
    return 0;
  }
  if (tag == 5) {
    memcpy(Wg, W, 5 * sizeof(double));
    if (Gg) memcpy(Gg, G, 15 * sizeof(double));
    return 0;
  }
  if (Gg) memset(Gg, 0, 15 * sizeof(double));
  if (tag == 4) {
    memcpy(Wg, ph->Winf, 5 * sizeof(double));
    return 0;
  }
  if (tag == 3) { /* 1D Riemann invariants normal to the face */
    double rho = W[0], u[3] = {W[1] / rho, W[2] / rho, W[3] / rho};
    double p = (g - 1.0) * (W[4] - 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
    const double* Wi = ph->Winf;
    double ri = Wi[0], ui[3] = {Wi[1] / ri, Wi[2] / ri, Wi[3] / ri};
    double pi_ = (g - 1.0) * (Wi[4] - 0.5 * ri * (ui[0] * ui[0] + ui[1] * ui[1] + ui[2] * ui[2]));
    if (!(rho > 0.0) || !(p > 0.0)) return -1;
    double c = sqrt(g * p / rho), ci = sqrt(g * pi_ / ri);
    double un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
    double uni = ui[0] * n[0] + ui[1] * n[1] + ui[2] * n[2];
    if (un >= c) {
      memcpy(Wg, W, 5 * sizeof(double));
      return 0;
    }
    if (un <= -c) {
      memcpy(Wg, Wi, 5 * sizeof(double));
      return 0;
    }
    double Rp = un + 2.0 * c / (g - 1.0), Rm = uni - 2.0 * ci / (g - 1.0);
    double unb = 0.5 * (Rp + Rm), cb = 0.25 * (g - 1.0) * (Rp - Rm);
    double s, ut[3];
    if (unb > 0.0) {
      s = p / pow(rho, g);
      for (int d = 0; d < 3; ++d) ut[d] = u[d] - un * n[d];
    } else {
      s = pi_ / pow(ri, g);
      for (int d = 0; d < 3; ++d) ut[d] = ui[d] - uni * n[d];
    }
    double rb = pow(cb * cb / (g * s), 1.0 / (g - 1.0));
    double pb = rb * cb * cb / g;
    double ub[3], u2 = 0.0;
    for (int d = 0; d < 3; ++d) {
      ub[d] = ut[d] + unb * n[d];
      u2 += ub[d] * ub[d];
    }
    Wg[0] = rb;
    for (int d = 0; d < 3; ++d) Wg[1 + d] = rb * ub[d];
    Wg[4] = pb / (g - 1.0) + 0.5 * rb * u2;
    return 0;
  }
  return -1;
}
