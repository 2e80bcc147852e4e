// Device functions of the gas-kinetic model shared by the fine (CGKS) and coarse (KFVS) kernels:
// primitive variables, the local face frame, half-space Maxwellian moments, the KFVS flux and the
// boundary ghost states.
#pragma once
#include <cuda_runtime.h>

#include "internal.cuh"

template <typename T>
struct Prim {
  T rho, U, V, W, lam;  // density, velocity in the face frame, lambda = rho / (2 p)
};

template <typename T>
HD T tsqrt(T x);
template <>
HD double tsqrt<double>(double x) { return sqrt(x); }
template <>
HD float tsqrt<float>(float x) { return sqrtf(x); }
template <typename T>
HD T texp(T x);
template <>
HD double texp<double>(double x) { return exp(x); }
template <>
HD float texp<float>(float x) { return expf(x); }
template <typename T>
HD T terfc(T x);
template <>
HD double terfc<double>(double x) { return erfc(x); }
template <>
HD float terfc<float>(float x) { return erfcf(x); }
// x^y for an exponent y that is a constant of the model (gamma, 1/(gamma - 1))
template <typename T>
HD T tpow(T x, T y);
template <>
HD double tpow<double>(double x, double y) { return pow(x, y); }
template <>
HD float tpow<float>(float x, float y) { return powf(x, y); }

// Forward-mode derivative: value v and directional derivative d of every quantity, so that one
// evaluation of a model function on Dual inputs (W, dW) yields f(W) and J(W) dW.  Comparisons act
// on values; constants (normals, gamma, the free stream) carry d = 0.
template <typename S>
struct Dual {
  S v, d;
  Dual() = default;
  HD Dual(S v_, S d_) : v(v_), d(d_) {}
  HD Dual(double c) : v(S(c)), d(S(0)) {}
  HD Dual(float c) : v(S(c)), d(S(0)) {}
  HD Dual(int c) : v(S(c)), d(S(0)) {}
};
template <typename S>
HD Dual<S> operator+(Dual<S> a, Dual<S> b) { return {a.v + b.v, a.d + b.d}; }
template <typename S>
HD Dual<S> operator-(Dual<S> a, Dual<S> b) { return {a.v - b.v, a.d - b.d}; }
template <typename S>
HD Dual<S> operator-(Dual<S> a) { return {-a.v, -a.d}; }
template <typename S>
HD Dual<S> operator*(Dual<S> a, Dual<S> b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
template <typename S>
HD Dual<S> operator/(Dual<S> a, Dual<S> b) {
  const S q = a.v / b.v;
  return {q, (a.d - q * b.d) / b.v};
}
template <typename S>
HD Dual<S>& operator+=(Dual<S>& a, Dual<S> b) { return a = a + b; }
template <typename S>
HD bool operator<(Dual<S> a, Dual<S> b) { return a.v < b.v; }
template <typename S>
HD bool operator>(Dual<S> a, Dual<S> b) { return a.v > b.v; }
template <typename S>
HD bool operator<=(Dual<S> a, Dual<S> b) { return a.v <= b.v; }
template <typename S>
HD bool operator>=(Dual<S> a, Dual<S> b) { return a.v >= b.v; }
template <>
HD Dual<float> tsqrt<Dual<float>>(Dual<float> x) {
  const float r = sqrtf(x.v);
  return {r, 0.5f * x.d / r};
}
template <>
HD Dual<float> texp<Dual<float>>(Dual<float> x) {
  const float e = expf(x.v);
  return {e, e * x.d};
}
template <>
HD Dual<float> terfc<Dual<float>>(Dual<float> x) {  // erfc'(x) = -2/sqrt(pi) exp(-x^2)
  return {erfcf(x.v), -1.1283791670955126f * expf(-x.v * x.v) * x.d};
}
template <>
HD Dual<float> tpow<Dual<float>>(Dual<float> x, Dual<float> y) {  // y constant
  const float p = powf(x.v, y.v);
  return {p, y.v * p / x.v * x.d};
}

// Dual<double>: the forward-mode linearisation of the FP64 residual.  Mixed operations with
// double constants, comparisons on values, and the elementary functions the residual calls (the
// derivative of each from its closed form: erfc' = -2/sqrt(pi) exp(-x^2)).  At the kinks the
// residual meets exactly (|x| at x = 0, fmin at equal arguments: a velocity component that is zero
// in a uniform stream, equal indicators in uniform regions) the derivative is the mean of the two
// one-sided ones, which is what a central difference measures: |x|' = 0 at 0, fmin' = the mean.
using DualD = Dual<double>;
HD DualD operator+(DualD a, double b) { return {a.v + b, a.d}; }
HD DualD operator+(double a, DualD b) { return {a + b.v, b.d}; }
HD DualD operator-(DualD a, double b) { return {a.v - b, a.d}; }
HD DualD operator-(double a, DualD b) { return {a - b.v, -b.d}; }
HD DualD operator*(DualD a, double b) { return {a.v * b, a.d * b}; }
HD DualD operator*(double a, DualD b) { return {a * b.v, a * b.d}; }
HD DualD operator/(DualD a, double b) { return {a.v / b, a.d / b}; }
HD DualD operator/(double a, DualD b) {
  const double q = a / b.v;
  return {q, -q * b.d / b.v};
}
HD DualD& operator+=(DualD& a, double b) { return a = a + b; }
HD DualD& operator-=(DualD& a, DualD b) { return a = a - b; }
HD DualD& operator*=(DualD& a, DualD b) { return a = a * b; }
HD DualD& operator*=(DualD& a, double b) { return a = a * b; }
HD bool operator>(DualD a, double b) { return a.v > b; }
HD bool operator<(DualD a, double b) { return a.v < b; }
HD bool operator>=(DualD a, double b) { return a.v >= b; }
HD bool operator<=(DualD a, double b) { return a.v <= b; }
HD bool operator!=(DualD a, double b) { return a.v != b; }
HD DualD sqrt(DualD x) {
  const double r = sqrt(x.v);
  return {r, 0.5 * x.d / r};
}
HD DualD exp(DualD x) {
  const double e = exp(x.v);
  return {e, e * x.d};
}
HD DualD erfc(DualD x) { return {erfc(x.v), -1.1283791670955125739 * exp(-x.v * x.v) * x.d}; }
HD DualD fabs(DualD x) { return {fabs(x.v), x.v < 0.0 ? -x.d : (x.v > 0.0 ? x.d : 0.0)}; }
HD DualD fmin(DualD a, DualD b) {
  if (a.v == b.v) return {a.v, 0.5 * (a.d + b.d)};
  return b.v < a.v ? b : a;
}
HD DualD pow(DualD x, double y) {
  const double p = pow(x.v, y);
  return {p, y * p / x.v * x.d};
}
HD bool isfinite(DualD x) { return isfinite(x.v); }
template <>
HD DualD tsqrt<DualD>(DualD x) { return sqrt(x); }
template <>
HD DualD texp<DualD>(DualD x) { return exp(x); }
template <>
HD DualD terfc<DualD>(DualD x) { return erfc(x); }
template <>
HD DualD tpow<DualD>(DualD x, DualD y) { return pow(x, y.v); }  // y constant

// branchless orthonormal basis (t1, t2) completing the unit normal n (Duff et al., JCGT 6(1), 2017)
template <typename T>
HD void face_frame(const T n[3], T t1[3], T t2[3]) {
  const T sign = n[2] >= T(0) ? T(1) : T(-1);
  const T a = T(-1) / (sign + n[2]);
  const T b = n[0] * n[1] * a;
  t1[0] = T(1) + sign * n[0] * n[0] * a;
  t1[1] = sign * b;
  t1[2] = -sign * n[0];
  t2[0] = b;
  t2[1] = sign + n[1] * n[1] * a;
  t2[2] = -n[1];
}

// conservative state in the face frame -> primitive; false when rho <= 0 or p <= 0
template <typename T>
HD bool prim_local(const T w[5], T gm1, Prim<T>& g) {
  const T r = T(1) / w[0];
  g.rho = w[0];
  g.U = w[1] * r;
  g.V = w[2] * r;
  g.W = w[3] * r;
  const T p = gm1 * (w[4] - T(0.5) * (w[1] * g.U + w[2] * g.V + w[3] * g.W));
  g.lam = T(0.5) * w[0] / p;
  return w[0] > T(0) && p > T(0);
}

template <typename T>
HD void rotate_in(const T W[5], const T n[3], const T t1[3], const T t2[3], T w[5]) {
  w[0] = W[0];
  w[1] = W[1] * n[0] + W[2] * n[1] + W[3] * n[2];
  w[2] = W[1] * t1[0] + W[2] * t1[1] + W[3] * t1[2];
  w[3] = W[1] * t2[0] + W[2] * t2[1] + W[3] * t2[2];
  w[4] = W[4];
}

template <typename T>
HD void rotate_out(const T f[5], const T n[3], const T t1[3], const T t2[3], T F[5]) {
  F[0] = f[0];
  F[1] = f[1] * n[0] + f[2] * t1[0] + f[3] * t2[0];
  F[2] = f[1] * n[1] + f[2] * t1[1] + f[3] * t2[1];
  F[3] = f[1] * n[2] + f[2] * t1[2] + f[3] * t2[2];
  F[4] = f[4];
}

// u-moments <u^0..u^N> over u > 0 (side = +1), u < 0 (side = -1) or all u (side = 0),
// normalised by rho: <u^(n+2)> = U <u^(n+1)> + (n+1)/(2 lam) <u^n>
template <typename T, int N>
HD void u_moments(T U, T lam, int side, T m[N + 1]) {
  if (side == 0) {
    m[0] = T(1);
    m[1] = U;
  } else {
    const T sl = tsqrt(lam);
    const T s = T(side);
    m[0] = T(0.5) * terfc(-s * sl * U);
    m[1] = U * m[0] + s * T(0.5) * texp(-lam * U * U) / (sl * T(1.7724538509055160273));
  }
  const T h = T(0.5) / lam;
#pragma unroll
  for (int n = 0; n + 2 <= N; ++n) m[n + 2] = U * m[n + 1] + T(n + 1) * h * m[n];
}

// KFVS flux through the face in the local frame: int_{u>0} u psi g^l + int_{u<0} u psi g^r
template <typename T>
HD void kfvs_local(const Prim<T>& gl, const Prim<T>& gr, T K, T f[5]) {
  const Prim<T>* gs[2] = {&gl, &gr};
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const Prim<T>& g = *gs[s];
    T m[4];
    u_moments<T, 3>(g.U, g.lam, s == 0 ? 1 : -1, m);
    const T h = T(0.5) / g.lam;
    const T q = g.V * g.V + g.W * g.W + (T(2) + K) * h;  // <v^2> + <w^2> + <xi^2>
    const T r = g.rho;
    f[0] = (s ? f[0] : T(0)) + r * m[1];
    f[1] = (s ? f[1] : T(0)) + r * m[2];
    f[2] = (s ? f[2] : T(0)) + r * g.V * m[1];
    f[3] = (s ? f[3] : T(0)) + r * g.W * m[1];
    f[4] = (s ? f[4] : T(0)) + T(0.5) * r * (m[3] + m[1] * q);
  }
}

// ghost state (and gradient when G != nullptr) of a boundary face with outward unit normal n.
// tag 1 slip wall (mirror), 2 no-slip adiabatic wall (mirror, velocity reversed), 3 farfield by 1D
// Riemann invariants, 4 supersonic inflow (free stream), 5 supersonic outflow (copy).
template <typename T>
HD bool bc_ghost(int tag, const T n[3], const T W[5], const T* G, T Wg[5], T* Gg,
                                         T gamma, const double* Winf) {
  if (tag == 1 || tag == 2) {
    const T mn = W[1] * n[0] + W[2] * n[1] + W[3] * n[2];
    Wg[0] = W[0];
    Wg[4] = W[4];
#pragma unroll
    for (int d = 0; d < 3; ++d) Wg[1 + d] = tag == 1 ? W[1 + d] - T(2) * mn * n[d] : -W[1 + d];
    if (Gg) {
      // scalars: R grad; momentum: R G R (slip) or -G R (no-slip), R = I - 2 n n^T
#pragma unroll
      for (int q = 0; q < 5; q += 4) {
        const T gn = G[3 * q] * n[0] + G[3 * q + 1] * n[1] + G[3 * q + 2] * n[2];
#pragma unroll
        for (int d = 0; d < 3; ++d) Gg[3 * q + d] = G[3 * q + d] - T(2) * gn * n[d];
      }
      T GR[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const T* g = G + 3 * (1 + i);
        const T gn = g[0] * n[0] + g[1] * n[1] + g[2] * n[2];
#pragma unroll
        for (int d = 0; d < 3; ++d) GR[i][d] = g[d] - T(2) * gn * n[d];
      }
      if (tag == 1) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const T cn = GR[0][d] * n[0] + GR[1][d] * n[1] + GR[2][d] * n[2];
#pragma unroll
          for (int i = 0; i < 3; ++i) Gg[3 * (1 + i) + d] = GR[i][d] - T(2) * n[i] * cn;
        }
      } else {
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int d = 0; d < 3; ++d) Gg[3 * (1 + i) + d] = -GR[i][d];
      }
    }
    return true;
  }
  if (tag == 5) {
#pragma unroll
    for (int q = 0; q < 5; ++q) Wg[q] = W[q];
    if (Gg)
#pragma unroll
      for (int j = 0; j < 15; ++j) Gg[j] = G[j];
    return true;
  }
  if (Gg)
#pragma unroll
    for (int j = 0; j < 15; ++j) Gg[j] = T(0);
  if (tag == 4) {
#pragma unroll
    for (int q = 0; q < 5; ++q) Wg[q] = T(Winf[q]);
    return true;
  }
  if (tag == 3) {
    const T gm1 = gamma - T(1);
    const T rho = W[0];
    const T u[3] = {W[1] / rho, W[2] / rho, W[3] / rho};
    const T p = gm1 * (W[4] - T(0.5) * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
    const T ri = T(Winf[0]);
    const T ui[3] = {T(Winf[1]) / ri, T(Winf[2]) / ri, T(Winf[3]) / ri};
    const T pi = gm1 * (T(Winf[4]) - T(0.5) * ri * (ui[0] * ui[0] + ui[1] * ui[1] + ui[2] * ui[2]));
    if (!(rho > T(0)) || !(p > T(0))) return false;
    const T c = tsqrt(gamma * p / rho), ci = tsqrt(gamma * pi / ri);
    const T un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
    const T uni = ui[0] * n[0] + ui[1] * n[1] + ui[2] * n[2];
    if (un >= c) {
#pragma unroll
      for (int q = 0; q < 5; ++q) Wg[q] = W[q];
      return true;
    }
    if (un <= -c) {
#pragma unroll
      for (int q = 0; q < 5; ++q) Wg[q] = T(Winf[q]);
      return true;
    }
    const T Rp = un + T(2) * c / gm1, Rm = uni - T(2) * ci / gm1;
    const T unb = T(0.5) * (Rp + Rm), cb = T(0.25) * gm1 * (Rp - Rm);
    T s, ut[3];
    if (unb > T(0)) {
      s = p / tpow(rho, gamma);
#pragma unroll
      for (int d = 0; d < 3; ++d) ut[d] = u[d] - un * n[d];
    } else {
      s = pi / tpow(ri, gamma);
#pragma unroll
      for (int d = 0; d < 3; ++d) ut[d] = ui[d] - uni * n[d];
    }
    const T rb = tpow(cb * cb / (gamma * s), T(1) / gm1);
    const T pb = rb * cb * cb / gamma;
    T ub[3], u2 = T(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      ub[d] = ut[d] + unb * n[d];
      u2 += ub[d] * ub[d];
    }
    Wg[0] = rb;
#pragma unroll
    for (int d = 0; d < 3; ++d) Wg[1 + d] = rb * ub[d];
    Wg[4] = pb / gm1 + T(0.5) * rb * u2;
    return true;
  }
  return false;
}

// KFVS flux in the global frame through a face with unit normal n
template <typename T>
HD bool kfvs_flux(const T WL[5], const T WR[5], const T n[3], T K, T gm1, T F[5]) {
  T t1[3], t2[3], wl[5], wr[5], f[5];
  face_frame(n, t1, t2);
  rotate_in(WL, n, t1, t2, wl);
  rotate_in(WR, n, t1, t2, wr);
  Prim<T> gl, gr;
  const bool ok = prim_local(wl, gm1, gl) & prim_local(wr, gm1, gr);
  kfvs_local(gl, gr, K, f);
  rotate_out(f, n, t1, t2, F);
  return ok;
}
