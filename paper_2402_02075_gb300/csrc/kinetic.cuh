// Device functions of the gas-kinetic model shared by the fine (CGKS) and coarse (KFVS) kernels:
// primitive variables, the local face frame, half-space Maxwellian moments, the KFVS flux and the
// boundary ghost states.
#pragma once
#include <cuda_runtime.h>

#include "internal.cuh"


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
HD T trsqrt(T x);
template <>
HD double trsqrt<double>(double x) {
#ifdef __CUDA_ARCH__
  return rsqrt(x);
#else
  return 1.0 / sqrt(x);
#endif
}
template <>
HD float trsqrt<float>(float x) {
#ifdef __CUDA_ARCH__
  return rsqrtf(x);
#else
  return 1.0f / sqrtf(x);
#endif
}
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
HD Dual<float> trsqrt<Dual<float>>(Dual<float> x) {
  const float r = trsqrt<float>(x.v);
  return {r, -0.5f * r * r * r * x.d};
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
template <>
HD DualD trsqrt<DualD>(DualD x) {
  const double r = trsqrt<double>(x.v);
  return {r, -0.5 * r * r * r * x.d};
}

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

// one side's half of the KFVS flux, int_{s u_n > 0} u_n psi g (s = +1 for the left state, -1 for the
// right), added into F in the global frame.  With U = u . n, h = p / rho = 1/(2 lambda) and the
// half-space moments m_k = <u_n^k> / rho: mass rho m1; momentum rho (m1 u + (m2 - U m1) n), since the
// tangential velocity is carried with the normal flux; energy rho (m3 + m1 (|u|^2 - U^2 + (K+2) h))/2.
// One division (1/rho) and one reciprocal square root (sqrt(lambda) = 1/sqrt(2 h)) per side.
template <typename T>
HD bool kfvs_side(const T w[5], const T n[3], T K, T gm1, T s, T F[5]) {
  const T r = T(1) / w[0];
  const T u[3] = {w[1] * r, w[2] * r, w[3] * r};
  const T u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const T p = gm1 * (w[4] - T(0.5) * (w[1] * u[0] + w[2] * u[1] + w[3] * u[2]));
  const T h = p * r;
  const T sl = trsqrt(T(2) * h);  // sqrt(lambda)
  const T U = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
  const T x = sl * U;
  T m[4];
  m[0] = T(0.5) * terfc(-s * x);
  // U m0 + s exp(-lambda U^2) / (2 sqrt(pi lambda)), 1/sqrt(lambda) = 2 h sqrt(lambda)
  m[1] = U * m[0] + s * T(0.56418958354775628695) * texp(-x * x) * (h * sl);
  m[2] = U * m[1] + h * m[0];
  m[3] = U * m[2] + T(2) * h * m[1];
  const T rho = w[0];
  const T rm1 = rho * m[1], rn = rho * (m[2] - U * m[1]);
  F[0] += rm1;
#pragma unroll
  for (int d = 0; d < 3; ++d) F[1 + d] += rm1 * u[d] + rn * n[d];
  F[4] += T(0.5) * rho * (m[3] + m[1] * (u2 - U * U + (T(2) + K) * h));
  return w[0] > T(0) && p > T(0);
}

// KFVS flux (int_{u_n > 0} u_n psi g^l + int_{u_n < 0} u_n psi g^r) in the global frame through a
// face with unit normal n
template <typename T>
HD bool kfvs_flux(const T WL[5], const T WR[5], const T n[3], T K, T gm1, T F[5]) {
#pragma unroll
  for (int q = 0; q < 5; ++q) F[q] = T(0);
  const bool okl = kfvs_side<T>(WL, n, K, gm1, T(1), F);
  const bool okr = kfvs_side<T>(WR, n, K, gm1, T(-1), F);
  return okl && okr;
}
