"""Exact source-level operation count of the gas-kinetic flux per Gauss point, from the kernel's own
point body instantiated on a counting scalar type (host).  Additions, subtractions and
multiplications count one FLOP each; divisions, square roots and transcendental functions are
counted apart (each is several FP64 instructions on the device).  The counts explain the FP64
instruction count that ncu reports for the kernel; they are asserted to stay in the range they
were measured at, so that an accidental change of the flux's arithmetic shows up."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2402_02075_gb300", "csrc")

HARNESS = r'''
#include "fine.cuh"

// the counters exist in the host pass only (the device pass compiles the same code without them)
#ifdef __CUDA_ARCH__
#define CNT(c)
#else
#define CNT(c) ++c
#endif
#define CD __host__ __device__ inline
struct Cnt {
  double v;
  Cnt() = default;
  CD Cnt(double x) : v(x) {}
};
static long g_flop = 0, g_div = 0, g_sqrt = 0, g_trans = 0;
CD Cnt F1(double x) { CNT(g_flop); return Cnt(x); }
CD Cnt operator+(Cnt a, Cnt b) { return F1(a.v + b.v); }
CD Cnt operator-(Cnt a, Cnt b) { return F1(a.v - b.v); }
CD Cnt operator*(Cnt a, Cnt b) { return F1(a.v * b.v); }
CD Cnt operator/(Cnt a, Cnt b) { CNT(g_div); return Cnt(a.v / b.v); }
CD Cnt operator-(Cnt a) { return Cnt(-a.v); }
CD Cnt operator+(Cnt a, double b) { return F1(a.v + b); }
CD Cnt operator+(double a, Cnt b) { return F1(a + b.v); }
CD Cnt operator-(Cnt a, double b) { return F1(a.v - b); }
CD Cnt operator-(double a, Cnt b) { return F1(a - b.v); }
CD Cnt operator*(Cnt a, double b) { return F1(a.v * b); }
CD Cnt operator*(double a, Cnt b) { return F1(a * b.v); }
CD Cnt operator/(Cnt a, double b) { CNT(g_div); return Cnt(a.v / b); }
CD Cnt operator/(double a, Cnt b) { CNT(g_div); return Cnt(a / b.v); }
CD Cnt& operator+=(Cnt& a, Cnt b) { return a = a + b; }
CD Cnt& operator+=(Cnt& a, double b) { return a = a + b; }
CD Cnt& operator-=(Cnt& a, Cnt b) { return a = a - b; }
CD Cnt& operator*=(Cnt& a, Cnt b) { return a = a * b; }
CD Cnt& operator*=(Cnt& a, double b) { return a = a * b; }
CD bool operator<(Cnt a, Cnt b) { return a.v < b.v; }
CD bool operator>(Cnt a, Cnt b) { return a.v > b.v; }
CD bool operator<=(Cnt a, Cnt b) { return a.v <= b.v; }
CD bool operator>=(Cnt a, Cnt b) { return a.v >= b.v; }
CD bool operator<(Cnt a, double b) { return a.v < b; }
CD bool operator>(Cnt a, double b) { return a.v > b; }
CD bool operator<=(Cnt a, double b) { return a.v <= b; }
CD bool operator>=(Cnt a, double b) { return a.v >= b; }
CD bool operator!=(Cnt a, double b) { return a.v != b; }
CD Cnt sqrt(Cnt x) { CNT(g_sqrt); return Cnt(sqrt(x.v)); }
CD Cnt rsqrt_hd(Cnt x) { CNT(g_sqrt); return Cnt(1.0 / sqrt(x.v)); }
CD Cnt exp(Cnt x) { CNT(g_trans); return Cnt(exp(x.v)); }
CD Cnt erfc(Cnt x) { CNT(g_trans); return Cnt(erfc(x.v)); }
CD Cnt fabs(Cnt x) { return Cnt(fabs(x.v)); }
CD Cnt fmin(Cnt a, Cnt b) { return b.v < a.v ? b : a; }
template <> CD Cnt tsqrt<Cnt>(Cnt x) { return sqrt(x); }
template <> CD Cnt texp<Cnt>(Cnt x) { return exp(x); }
template <> CD Cnt terfc<Cnt>(Cnt x) { return erfc(x); }
template <> CD Cnt tpow<Cnt>(Cnt x, Cnt y) { CNT(g_trans); return Cnt(pow(x.v, y.v)); }

// operation counts of one interior Gauss point: out = (flop, div, sqrt, transcendental)
extern "C" void count_point(int viscous, double prandtl, const double* WL, const double* GL, const double* WR,
                            const double* GR, const double* n, double dt, long* out) {
  Phys ph{};
  ph.gamma = 1.4;
  ph.K = 2.0;
  ph.mu = viscous ? 1e-3 : 0.0;
  ph.prandtl = prandtl;
  ph.eps_inviscid = 0.01;
  ph.c_press = 1.0;
  ph.viscous = viscous;
  ph.cf = 1;
  Cnt wl[5], gl[15], wr[5], gr[15], F[5], Wt[5], al;
  for (int q = 0; q < 5; ++q) { wl[q] = WL[q]; wr[q] = WR[q]; }
  for (int j = 0; j < 15; ++j) { gl[j] = GL[j]; gr[j] = GR[j]; }
  DevErr err{};
  g_flop = g_div = g_sqrt = g_trans = 0;
  point_flux<Cnt>(n, 1.0, false, 0, wl, gl, wr, gr, Cnt(dt), ph, F, Wt, al, &err, 0);
  out[0] = g_flop; out[1] = g_div; out[2] = g_sqrt; out[3] = g_trans;
}
'''


@pytest.fixture(scope="module")
def counter(tmp_path_factory):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("op_count")
    (d / "count.cu").write_text(HARNESS)
    lib = d / "count.so"
    subprocess.run([nvcc, "-std=c++17", "-O1", "-Xcompiler", "-fPIC", "-shared", "--expt-relaxed-constexpr",
                    "-I" + os.path.join(ROOT, "include"), "-I" + CSRC, "-o", str(lib), str(d / "count.cu")], check=True)
    L = C.CDLL(str(lib))
    L.count_point.argtypes = [C.c_int, C.c_double] + [C.c_void_p] * 5 + [C.c_double, C.c_void_p]
    return L


def _p(a):
    return np.ascontiguousarray(a, dtype=np.float64).ctypes.data_as(C.c_void_p)


@pytest.mark.parametrize("viscous,prandtl", [(0, 1.0), (1, 0.72)])
def test_flux_operation_count_per_gauss_point(counter, viscous, prandtl):
    rng = np.random.default_rng(51)
    WL = np.array([1.0, 0.5, 0.1, 0.0, 2.0])
    WR = np.array([1.1, 0.4, 0.0, 0.1, 2.1])
    GL, GR = rng.normal(size=15) * 0.1, rng.normal(size=15) * 0.1
    n = np.array([0.6, 0.8, 0.0])
    out = np.zeros(4, np.int64)
    counter.count_point(viscous, prandtl, _p(WL), _p(GL), _p(WR), _p(GR), _p(n), 0.01, out.ctypes.data_as(C.c_void_p))
    flop, div, sq, trans = (int(x) for x in out)
    print(f"viscous={viscous} Pr={prandtl}: {flop} add/sub/mul, {div} div, {sq} sqrt/rsqrt, {trans} exp/erfc/pow")
    # measured: 2,574 (inviscid) and 2,604 (viscous, Pr 0.72: the Prandtl correction) add/sub/mul,
    # 11 divisions, 4 square roots, 5 exp/erfc (2,989 and 3,019 before the slope solve, the Euler-flux
    # derivative and the moment products shared their per-Maxwellian coefficients); the ncu count of
    # the kernel adds the device expansions of the 20 special operations
    assert 2400 <= flop <= 2800 and div <= 12 and sq <= 4 and trans <= 5, (flop, div, sq, trans)
