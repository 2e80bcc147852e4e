"""The library's gas-kinetic point flux, compiled for the host, against the oracle's independent
point flux; and its forward-mode linearisation (the code the adjoint stores) against central
differences of the oracle.  The kernel bodies are host+device functions, so this runs without a
GPU: it checks the CUDA path's arithmetic, not the device.  Tolerances as in the GPU parity tests
(1e-11 of the terms' scale for values; 1e-8 for derivatives against Richardson-extrapolated
differences)."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2402_02075_gb300", "csrc")

HARNESS = r'''
#include <vector>

#include "adjoint.cuh"
#include "recon_ops.cuh"

static Phys phys(const double* p) {
  Phys ph{};
  ph.gamma = p[0];
  ph.K = (5.0 - 3.0 * p[0]) / (p[0] - 1.0);
  ph.mu = p[1];
  ph.prandtl = p[2];
  ph.eps_inviscid = p[3];
  ph.c_press = p[4];
  ph.viscous = p[1] > 0.0;
  ph.cf = 0;
  return ph;
}

extern "C" int host_point_flux(const double* p, const double* WL, const double* GL, const double* WR, const double* GR,
                               const double* n, double dt, double* F, double* Wt) {
  const Phys ph = phys(p);
  DevErr err{};
  double al;
  point_flux<double>(n, 1.0, false, 0, WL, GL, WR, GR, dt, ph, F, Wt, al, &err, 0);
  return err.code;
}

extern "C" void host_kfvs(double gamma, const double* WL, const double* WR, const double* n, double* F) {
  kfvs_flux<double>(WL, WR, n, (5.0 - 3.0 * gamma) / (gamma - 1.0), gamma - 1.0, F);
}

extern "C" int host_ghost(int tag, double gamma, const double* Winf, const double* n, const double* W, const double* G,
                          double* Wg, double* Gg) {
  return bc_ghost<double>(tag, n, W, G, Wg, Gg, gamma, Winf) ? 0 : 1;
}

extern "C" void host_kfvs_jvp32(double gamma, const double* WL, const double* WR, const double* dL, const double* dR,
                                const double* n, double* dF) {
  Dual<float> wl[5], wr[5], nn[3], F[5];
  for (int q = 0; q < 5; ++q) {
    wl[q] = Dual<float>((float)WL[q], (float)dL[q]);
    wr[q] = Dual<float>((float)WR[q], (float)dR[q]);
  }
  for (int d = 0; d < 3; ++d) nn[d] = Dual<float>((float)n[d], 0.0f);
  const float K = (float)((5.0 - 3.0 * gamma) / (gamma - 1.0));
  kfvs_flux<Dual<float>>(wl, wr, nn, Dual<float>(K, 0.0f), Dual<float>((float)(gamma - 1.0), 0.0f), F);
  for (int q = 0; q < 5; ++q) dF[q] = F[q].d;
}

// the reconstruction operators of every cell from its geometry, then the WENO reconstruction and the
// local time step of every cell; p = (gamma, mu, prandtl, weno_eps, cfl, Winf[5])
extern "C" int host_reconstruct(int64_t nc, int64_t nf, const int8_t* ctype, const int32_t* cf, const int8_t* cside,
                                const int32_t* fL, const int32_t* fR, const int32_t* ftag, const double* vol,
                                const double* ctr, const double* m2, const double* Sn, const double* area,
                                const double* fshift, const double* fctr, const double* fnrm, const double* W,
                                const double* G, const double* alpha, const double* p, double* rc, double* dt) {
  std::vector<double> Kop(216 * nc), ggw(18 * nc), lsw(18 * nc), aux(8 * nc), dtw(24 * nc);
  DevErr err{};
  ROArgs ro{nc, nf, ctype, cf, cside, fL, fR, vol, ctr, m2, Sn, area, fshift, fctr, fnrm,
            Kop.data(), ggw.data(), lsw.data(), aux.data(), dtw.data(), &err};
  for (int64_t i = 0; i < nc; ++i) recon_ops_body(i, ro);
  if (err.code) return 100 + err.code;
  Phys ph{};
  ph.gamma = p[0];
  ph.K = (5.0 - 3.0 * p[0]) / (p[0] - 1.0);
  ph.mu = p[1];
  ph.prandtl = p[2];
  ph.weno_eps = p[3];
  ph.cfl_fine = p[4];
  ph.viscous = p[1] > 0.0;
  for (int q = 0; q < 5; ++q) ph.Winf[q] = p[5 + q];
  ReconArgs ra{nc, nf, ctype, cf, fL, fR, ftag, cside, fnrm, Kop.data(), ggw.data(), lsw.data(), aux.data(),
               dtw.data(), vol, W, G, alpha, rc, dt, ph, &err};
  for (int64_t i = 0; i < nc; ++i) reconstruct_body(i, ra);
  return err.code;
}

// the whole fine residual (Res, Gnew, alpha) of the CUDA path on the host; when res_flux != NULL,
// the residual again by the flux-only point body and the residual-only gather (into fresh records);
// and, when rbar != NULL, the adjoint's transposed product (stored Jacobians and the four
// transposed-product bodies)
extern "C" int host_fine(int64_t nc, int64_t nf, int64_t ngp, const int8_t* ctype, const int32_t* cf,
                         const int8_t* cside, const int32_t* fL, const int32_t* fR, const int32_t* ftag,
                         const int32_t* gp_ptr, const int32_t* gp_face, const double* gp_x, const double* gp_A,
                         const double* vol, const double* ctr, const double* m2, const double* Sn, const double* area,
                         const double* fshift, const double* fctr, const double* fnrm, const double* W, const double* G,
                         const double* alpha, const double* p, int cf_on, double* res, double* Gout, double* aout,
                         const double* rbar, const double* gbar, double* out, int recompute, double* res_flux) {
  std::vector<double> Kop(216 * nc), ggw(18 * nc), lsw(18 * nc), aux(8 * nc), dtw(24 * nc);
  DevErr err{};
  ROArgs ro{nc, nf, ctype, cf, cside, fL, fR, vol, ctr, m2, Sn, area, fshift, fctr, fnrm,
            Kop.data(), ggw.data(), lsw.data(), aux.data(), dtw.data(), &err};
  for (int64_t i = 0; i < nc; ++i) recon_ops_body(i, ro);
  if (err.code) return 100 + err.code;
  Phys ph{};
  ph.gamma = p[0];
  ph.K = (5.0 - 3.0 * p[0]) / (p[0] - 1.0);
  ph.mu = p[1];
  ph.prandtl = p[2];
  ph.weno_eps = p[3];
  ph.cfl_fine = p[4];
  ph.eps_inviscid = 0.01;
  ph.c_press = 1.0;
  ph.viscous = p[1] > 0.0;
  ph.cf = cf_on;
  for (int q = 0; q < 5; ++q) ph.Winf[q] = p[5 + q];
  std::vector<double> rc(50 * nc + 2), dt(nc), gpr(CGKS_GPR * ngp + 2);
  double* rca = rc.data() + ((reinterpret_cast<uintptr_t>(rc.data()) & 15) ? 1 : 0);  // 16-byte aligned
  ReconArgs ra{nc, nf, ctype, cf, fL, fR, ftag, cside, fnrm, Kop.data(), ggw.data(), lsw.data(), aux.data(),
               dtw.data(), vol, W, G, alpha, rca, dt.data(), ph, &err};
  for (int64_t i = 0; i < nc; ++i) reconstruct_body(i, ra);
  double* gpra = gpr.data() + ((reinterpret_cast<uintptr_t>(gpr.data()) & 15) ? 1 : 0);  // 16-byte aligned
  PointArgs pa{ngp, nf, nc, gp_face, fL, fR, ftag, gp_x, gp_A, fshift, ctr, rca, dt.data(), gpra, ph, &err};
  for (int64_t g = 0; g < ngp; ++g) gks_point_body(g, pa);
  GatherArgs ga{nc, ngp, ctype, cside, cf, gp_ptr, gpra, vol, dt.data(), W,
                nullptr, res, Gout, aout, 0, ph.gamma, &err};
  for (int64_t i = 0; i < nc; ++i) gather_body(i, ga);
  if (res_flux) {
    std::vector<double> gpr2(CGKS_GPR * ngp + 2, 0.0);
    double* g2 = gpr2.data() + ((reinterpret_cast<uintptr_t>(gpr2.data()) & 15) ? 1 : 0);
    PointArgs pf = pa;
    pf.gpr = g2;
    for (int64_t g = 0; g < ngp; ++g) gks_point_body<false>(g, pf);
    GatherArgs gf{nc, ngp, ctype, cside, cf, gp_ptr, g2, vol, dt.data(), W,
                  nullptr, res_flux, nullptr, nullptr, 0, ph.gamma, &err};
    for (int64_t i = 0; i < nc; ++i) gather_body(i, gf);
  }
  if (err.code || !rbar) return err.code;
  std::vector<double> Jr(recompute ? 1 : (size_t)CGKS_RJ_ROWS * nc), Jp((size_t)CGKS_PJ_IN * CGKS_PJ_OUT * ngp);
  if (!recompute)
    for (int64_t i = 0; i < nc; ++i) recon_jacobian_body(i, ra, Jr.data());
  for (int64_t g = 0; g < ngp; ++g) point_jacobian_body(g, pa, Jp.data());
  std::vector<double> pbar(CGKS_PB * ngp + 2), self(20 * nc), rec(40 * nf + 2), cbuf(CGKS_RJ_OUT * nc);
  double* pb = pbar.data() + ((reinterpret_cast<uintptr_t>(pbar.data()) & 15) ? 1 : 0);
  double* rr = rec.data() + ((reinterpret_cast<uintptr_t>(rec.data()) & 15) ? 1 : 0);
  VjpArgs va{nc, nf, ngp, ctype, cside, cf, fL, fR, gp_face, gp_ptr, gp_x, gp_A, fshift, ctr, vol, dt.data(),
             Jp.data(), Jr.data(), rbar, gbar, pb, self.data(), rr, cbuf.data(), out};
  for (int64_t g = 0; g < ngp; ++g) vjp_point_body(g, va);
  for (int64_t i = 0; i < nc; ++i) vjp_coef_body(i, va);
  if (recompute) {
    for (int64_t i = 0; i < nc; ++i) vjp_recon_body(i, ra, va, cbuf.data() + i, nc);
  } else {
    for (int64_t i = 0; i < nc; ++i)
      for (int k = 0; k < 50; ++k) vjp_slot_body(i, k, va, cbuf.data() + i, (int)nc);
  }
  for (int64_t i = 0; i < nc; ++i) vjp_cell_body(i, va);
  return err.code;
}

extern "C" int host_point_jvp(const double* p, const double* WL, const double* GL, const double* WR, const double* GR,
                              const double* n, double dt, const double* d, double* dF, double* dWt) {
  const Phys ph = phys(p);
  DevErr err{};
  DualD wl[5], gl[15], wr[5], gr[15], F[5], Wt[5], al;
  for (int q = 0; q < 5; ++q) {
    wl[q] = DualD(WL[q], d[q]);
    wr[q] = DualD(WR[q], d[20 + q]);
  }
  for (int j = 0; j < 15; ++j) {
    gl[j] = DualD(GL[j], d[5 + j]);
    gr[j] = DualD(GR[j], d[25 + j]);
  }
  point_flux<DualD>(n, 1.0, false, 0, wl, gl, wr, gr, DualD(dt, d[40]), ph, F, Wt, al, &err, 0);
  for (int q = 0; q < 5; ++q) {
    dF[q] = F[q].d;
    dWt[q] = Wt[q].d;
  }
  return err.code;
}
'''


@pytest.fixture(scope="module")
def host(tmp_path_factory):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("host_bodies")
    src, lib = d / "harness.cu", d / "harness.so"
    src.write_text(HARNESS)
    subprocess.run([nvcc, "-std=c++17", "-O2", "-Xcompiler", "-fPIC", "-shared", "--expt-relaxed-constexpr",
                    "-I" + os.path.join(ROOT, "include"), "-I" + CSRC, "-o", str(lib), str(src)], check=True)
    L = C.CDLL(str(lib))
    d_ = C.c_void_p
    L.host_point_flux.argtypes = [d_] * 6 + [C.c_double, d_, d_]
    L.host_point_jvp.argtypes = [d_] * 6 + [C.c_double, d_, d_, d_]
    L.host_kfvs.argtypes = [C.c_double, d_, d_, d_, d_]
    L.host_ghost.argtypes = [C.c_int, C.c_double] + [d_] * 6
    L.host_kfvs_jvp32.argtypes = [C.c_double] + [d_] * 6
    L.host_reconstruct.argtypes = [C.c_int64, C.c_int64] + [d_] * 20
    L.host_fine.argtypes = [C.c_int64] * 3 + [d_] * 22 + [C.c_int] + [d_] * 6 + [C.c_int, d_]
    return L


def _p(a):
    return np.ascontiguousarray(a, dtype=np.float64).ctypes.data_as(C.c_void_p)


def _cases(rng, n_cases=6):
    def state():
        rho, u, p = 0.8 + 0.4 * rng.random(), rng.normal(size=3) * 0.5, 0.6 + 0.3 * rng.random()
        return np.array([rho, *(rho * u), p / 0.4 + 0.5 * rho * u @ u])
    for _ in range(n_cases):
        n = rng.normal(size=3)
        yield state(), rng.normal(size=15) * 0.2, state(), rng.normal(size=15) * 0.2, n / np.linalg.norm(n)


PHYS = [dict(mach=0.5), dict(mach=0.5, viscous=1, reynolds=500.0, prandtl=0.72),
        dict(mach=0.5, viscous=1, reynolds=500.0, prandtl=1.0)]


def _host_params(prm):
    mu = prm.get("mach", 0.2) / prm["reynolds"] if prm.get("viscous") else 0.0
    return np.array([1.4, mu, prm.get("prandtl", 1.0), 0.01, 1.0])


@pytest.mark.parametrize("prm", PHYS)
def test_point_flux_body_matches_the_oracle(orc, host, prm):
    op, hp = orc.params(**prm), _host_params(prm)
    rng = np.random.default_rng(31)
    dt = 0.01
    for WL, GL, WR, GR, n in _cases(rng):
        F, Wt = np.zeros(5), np.zeros(5)
        assert host.host_point_flux(_p(hp), _p(WL), _p(GL), _p(WR), _p(GR), _p(n), dt, _p(F), _p(Wt)) == 0
        Fo, Wto = orc.gks_point(op, WL, GL, WR, GR, n, dt)
        assert np.abs(F - Fo).max() <= 1e-11 * np.abs(Fo).max(), (F, Fo)
        assert np.abs(Wt - Wto).max() <= 1e-11 * np.abs(Wto).max(), (Wt, Wto)


@pytest.mark.parametrize("prm", PHYS)
def test_point_linearisation_matches_oracle_differences(orc, host, prm):
    """The directional derivative that the adjoint's stored Jacobian holds, against Richardson-
    extrapolated central differences of the oracle's point flux in the same direction (inputs: both
    sides' states and gradients and the time step)."""
    op, hp = orc.params(**prm), _host_params(prm)
    rng = np.random.default_rng(32)
    dt = 0.01
    for WL, GL, WR, GR, n in _cases(rng, 4):
        x = np.concatenate([WL, GL, WR, GR, [dt]])
        d = rng.normal(size=41) * np.concatenate([np.abs(WL), np.full(15, 0.2), np.abs(WR), np.full(15, 0.2), [dt]])
        dF, dWt = np.zeros(5), np.zeros(5)
        assert host.host_point_jvp(_p(hp), _p(WL), _p(GL), _p(WR), _p(GR), _p(n), dt, _p(d), _p(dF), _p(dWt)) == 0

        def f(y):
            F, Wt = orc.gks_point(op, y[:5], y[5:20], y[20:25], y[25:40], n, y[40])
            return np.concatenate([F, Wt])

        def cd(h):
            return (f(x + h * d) - f(x - h * d)) / (2 * h)

        ref = (4.0 * cd(0.5e-6) - cd(1e-6)) / 3.0
        got = np.concatenate([dF, dWt])
        assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max(), (got, ref)


def test_kfvs_body_matches_the_oracle(orc, host):
    """The coarse-level first-order flux (KFVS) of the CUDA path against the oracle's."""
    op = orc.params()
    rng = np.random.default_rng(33)
    for WL, _, WR, _, n in _cases(rng, 8):
        F = np.zeros(5)
        host.host_kfvs(1.4, _p(WL), _p(WR), _p(n), _p(F))
        Fo = orc.kfvs_point(op, WL, WR, n)
        assert np.abs(F - Fo).max() <= 1e-13 * np.abs(Fo).max(), (F, Fo)


def _prim_state(rho, u, p, gamma=1.4):
    u = np.asarray(u, dtype=np.float64)
    return np.array([rho, *(rho * u), p / (gamma - 1.0) + 0.5 * rho * u @ u])


@pytest.mark.parametrize("name,WL,WR,n", [
    # one-sided fluxes: supersonic along +n and along -n (the half-space erfc tails vanish)
    ("supersonic +n", _prim_state(1.0, [3.0, 0.2, -0.1], 1 / 1.4), _prim_state(1.2, [2.9, 0.1, 0.0], 0.8), [1.0, 0.0, 0.0]),
    ("hypersonic -n", _prim_state(0.9, [0.0, 0.0, 8.0], 0.7), _prim_state(1.0, [0.1, 0.0, 8.2], 0.72), [0.0, 0.0, -1.0]),
    # flow tangential to the face: U = 0, the energy flux carries |u|^2 - U^2 = |u_t|^2
    ("tangential", _prim_state(1.0, [0.0, 0.9, 0.4], 0.7), _prim_state(1.1, [0.0, 0.8, 0.5], 0.75), [1.0, 0.0, 0.0]),
    # strong jumps across an oblique face
    ("strong jump", _prim_state(5.0, [0.3, -0.2, 0.1], 4.0), _prim_state(0.2, [-0.4, 0.3, 0.0], 0.1),
     [0.48, -0.6, 0.64]),
])
def test_kfvs_body_one_sided_tangential_and_jumps(orc, host, name, WL, WR, n):
    """The coarse KFVS flux in the global frame at the states the random cases do not reach, against
    the oracle's face-frame KFVS (1e-13 of the flux scale)."""
    op = orc.params()
    n = np.asarray(n, dtype=np.float64)
    n = n / np.linalg.norm(n)
    F = np.zeros(5)
    host.host_kfvs(1.4, _p(WL), _p(WR), _p(n), _p(F))
    Fo = orc.kfvs_point(op, WL, WR, n)
    assert np.abs(F - Fo).max() <= 1e-13 * np.abs(Fo).max(), (name, F, Fo)


@pytest.mark.parametrize("tag", [1, 2, 3, 4, 5])
def test_ghost_states_match_the_oracle(orc, host, tag):
    """Ghost states and gradients of the five boundary kinds (slip wall, no-slip wall, farfield by
    Riemann invariants, supersonic inflow, supersonic outflow), subsonic and supersonic normal
    velocities, against the oracle's."""
    for mach in (0.5, 3.0):
        op = orc.params(mach=mach)
        u = np.array([mach, 0.0, 0.0])
        Winf = np.array([1.0, *u, 1.0 / 1.4 / 0.4 + 0.5 * u @ u])
        rng = np.random.default_rng(34 + tag)
        for WL, GL, _, _, n in _cases(rng, 6):
            Wg, Gg = np.zeros(5), np.zeros(15)
            assert host.host_ghost(tag, 1.4, _p(Winf), _p(n), _p(WL), _p(GL), _p(Wg), _p(Gg)) == 0
            Wo, Go = orc.bc_ghost(op, tag, n, WL, GL)
            assert np.abs(Wg - Wo).max() <= 1e-13 * np.abs(Wo).max(), (tag, Wg, Wo)
            assert np.abs(Gg - Go).max() <= 1e-13 * max(np.abs(Go).max(), 1e-300) or np.abs(Gg - Go).max() == 0.0, (tag, Gg, Go)


def test_fp32_kfvs_linearisation_matches_oracle_differences(orc, host):
    """The FP32 forward-mode KFVS derivative of the mixed-precision coarse levels against central
    differences of the oracle's FP64 KFVS flux: FP32 accuracy (1e-5 of the derivative's scale)."""
    op = orc.params()
    rng = np.random.default_rng(35)
    for WL, _, WR, _, n in _cases(rng, 8):
        dL, dR = rng.normal(size=5) * np.abs(WL) * 1e-2, rng.normal(size=5) * np.abs(WR) * 1e-2
        dF = np.zeros(5)
        host.host_kfvs_jvp32(1.4, _p(WL), _p(WR), _p(dL), _p(dR), _p(n), _p(dF))
        h = 1e-4
        ref = (orc.kfvs_point(op, WL + h * dL, WR + h * dR, n) - orc.kfvs_point(op, WL - h * dL, WR - h * dR, n)) / (2 * h)
        assert np.abs(dF - ref).max() <= 1e-5 * np.abs(ref).max(), (dF, ref)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32).ctypes.data_as(C.c_void_p)


def _i8(a):
    return np.ascontiguousarray(a, dtype=np.int8).ctypes.data_as(C.c_void_p)


RECON_CASES = {
    "mixed periodic": (lambda mg: mg.periodic_box(6), dict(mach=0.5)),
    "wall box": (lambda mg: mg.wall_box(8, 4, 8, n_prism=3), dict(mach=0.5, viscous=1, reynolds=1e3, prandtl=0.72)),
    "ramp": (lambda mg: mg.ramp_box(8, 4, 2, n_prism=1), dict(mach=3.0)),
    "pyramids": (lambda mg: mg.pyramid_box(6, periodic=False), dict(mach=0.5)),
}


@pytest.mark.parametrize("name", list(RECON_CASES))
def test_reconstruction_body_matches_the_oracle(orc, host, name):
    """The CUDA path's reconstruction-operator precompute and WENO reconstruction (Sec. 3), run on the
    host from the oracle's cell and face geometry, against the oracle's reconstruction (which solves
    the constrained least-squares problem per call) and its local time steps."""
    import meshgen as mg
    mk, prm = RECON_CASES[name]
    mesh = mk(mg)
    om = orc.Mesh(mesh)
    nc, nf = om.nc, om.nf
    vol, ctr, m2 = om.cells()
    F = om.faces()
    ngp = F["ngp"]
    mask = (np.arange(4)[None, :] < ngp[:, None])[:, :, None]
    gA, gx = np.where(mask, F["gA"], 0.0), np.where(mask, F["gx"], 0.0)
    Sn = gA.sum(1)
    w = np.linalg.norm(gA, axis=2)
    area = w.sum(1)
    fctr = (w[:, :, None] * gx).sum(1) / area[:, None]
    fnrm = Sn / np.linalg.norm(Sn, axis=1)[:, None]
    rng = np.random.default_rng(41)
    mach = prm["mach"]
    W, G = mg.uniform_state(nc, mach=mach)
    amp = 0.003 if mach > 1 else 0.02
    W = W * (1.0 + amp * rng.standard_normal(W.shape))
    G = 2.5 * amp * rng.standard_normal(G.shape)
    alpha = 1.0 - 0.1 * rng.random(nc)
    op = orc.params(n_levels=1, **prm)
    u = np.array([mach, 0.0, 0.0])
    p = np.array([1.4, mach / prm["reynolds"] if prm.get("viscous") else 0.0, prm.get("prandtl", 1.0), 1e-5, 0.5,
                  1.0, *u, 1.0 / 1.4 / 0.4 + 0.5 * u @ u])
    rc = np.zeros((nc, 50))
    dt = np.zeros(nc)
    T = np.ascontiguousarray
    code = host.host_reconstruct(nc, nf, _i8(mesh["cell_type"]), _i32(F["cf"].T), _i8(F["cside"].T), _i32(F["fL"]),
                                 _i32(F["fR"]), _i32(F["tag"]), _p(vol), _p(T(ctr.T)), _p(T(m2.T)), _p(T(Sn.T)),
                                 _p(area), _p(T(F["shift"].T)), _p(T(fctr.T)), _p(T(fnrm.T)), _p(W), _p(G), _p(alpha),
                                 _p(p), _p(rc), _p(dt))
    assert code == 0
    os_ = orc.Solver(om, op)
    os_.set_state(W, G, alpha)
    ref = os_.reconstruct(0).reshape(nc, 50)
    for q in range(5):
        blk, rblk = rc[:, 10 * q:10 * q + 10], ref[:, 10 * q:10 * q + 10]
        err = np.linalg.norm(blk - rblk) / np.linalg.norm(rblk)
        assert err <= 1e-10, (name, q, err)
    dto = os_.residual()["dt"]
    assert np.abs(dt - dto).max() <= 1e-13 * np.abs(dto).max()


def _fine_inputs(orc, mesh):
    om = orc.Mesh(mesh)
    nc, nf = om.nc, om.nf
    vol, ctr, m2 = om.cells()
    F = om.faces()
    ngpf = F["ngp"]
    mask = (np.arange(4)[None, :] < ngpf[:, None])[:, :, None]
    gA, gx = np.where(mask, F["gA"], 0.0), np.where(mask, F["gx"], 0.0)
    Sn = gA.sum(1)
    w = np.linalg.norm(gA, axis=2)
    area = w.sum(1)
    fctr = (w[:, :, None] * gx).sum(1) / area[:, None]
    fnrm = Sn / np.linalg.norm(Sn, axis=1)[:, None]
    gp_ptr = np.concatenate([[0], np.cumsum(ngpf)]).astype(np.int32)
    sel = mask[:, :, 0].ravel()
    gp_x = np.ascontiguousarray(gx.reshape(-1, 3)[sel].T)
    gp_A = np.ascontiguousarray(gA.reshape(-1, 3)[sel].T)
    gp_face = np.repeat(np.arange(nf, dtype=np.int32), ngpf)
    T = np.ascontiguousarray
    arrays = [_i8(mesh["cell_type"]), _i32(F["cf"].T), _i8(F["cside"].T), _i32(F["fL"]), _i32(F["fR"]), _i32(F["tag"]),
              _i32(gp_ptr), _i32(gp_face), _p(gp_x), _p(gp_A), _p(vol), _p(T(ctr.T)), _p(T(m2.T)), _p(T(Sn.T)),
              _p(area), _p(T(F["shift"].T)), _p(T(fctr.T)), _p(T(fnrm.T))]
    keep = (gp_ptr, gp_face, gp_x, gp_A, vol, ctr, m2, Sn, area, fctr, fnrm, F)  # alive while the arrays are used
    return om, nc, nf, int(gp_ptr[-1]), arrays, keep


def _phys_vector(prm):
    mach = prm["mach"]
    u = np.array([mach, 0.0, 0.0])
    return np.array([1.4, mach / prm["reynolds"] if prm.get("viscous") else 0.0, prm.get("prandtl", 1.0), 1e-5, 0.5,
                     1.0, *u, 1.0 / 1.4 / 0.4 + 0.5 * u @ u])


FINE_CASES = {
    "mixed periodic": (lambda mg: mg.periodic_box(6), dict(mach=0.5)),
    "wall box": (lambda mg: mg.wall_box(8, 4, 8, n_prism=3), dict(mach=0.5, viscous=1, reynolds=1e3, prandtl=0.72)),
    "ramp": (lambda mg: mg.ramp_box(8, 4, 2, n_prism=1), dict(mach=3.0)),
    "pyramids": (lambda mg: mg.pyramid_box(6, periodic=False), dict(mach=0.5, viscous=1, reynolds=1e3, prandtl=0.72)),
}


def _state(mg, nc, mach, seed):
    rng = np.random.default_rng(seed)
    W, G = mg.uniform_state(nc, mach=mach)
    amp = 0.003 if mach > 1 else 0.02
    return W * (1.0 + amp * rng.standard_normal(W.shape)), 2.5 * amp * rng.standard_normal(G.shape), rng


@pytest.mark.parametrize("cf_on", [1, 0])
@pytest.mark.parametrize("name", list(FINE_CASES))
def test_fine_residual_on_the_host_matches_the_oracle(orc, host, name, cf_on):
    """The whole fine CGKS residual of the CUDA path (operators, reconstruction, point flux, gather),
    run on the host, against the oracle's residual, Gauss-Green gradients and compression factors,
    with the tolerances of the GPU parity tests."""
    import meshgen as mg
    from parity import assert_normwise, grad_scale
    mk, prm = FINE_CASES[name]
    mesh = mk(mg)
    om, nc, nf, ngp, arrays, keep = _fine_inputs(orc, mesh)
    W, G, rng = _state(mg, nc, prm["mach"], 43)
    alpha = 1.0 - 0.1 * rng.random(nc)
    res, Gout, aout, res_flux = np.zeros((5, nc)), np.zeros((15, nc)), np.zeros(nc), np.full((5, nc), np.nan)
    code = host.host_fine(nc, nf, ngp, *arrays, _p(W), _p(G), _p(alpha), _p(_phys_vector(prm)), cf_on, _p(res),
                          _p(Gout), _p(aout), None, None, None, 0, _p(res_flux))
    assert code == 0
    # the V-cycle's defect (flux-only points, residual-only gather) is the same residual, bit for bit
    assert np.array_equal(res_flux, res)
    os_ = orc.Solver(om, orc.params(n_levels=1, compression_factor=cf_on, **prm))
    os_.set_state(W, G, alpha)
    ro = os_.residual()
    assert_normwise(res, ro["res"], 1e-11, "residual", scale=ro["fscale"])
    assert_normwise(Gout, ro["grad"], 1e-11, "Gauss-Green gradients", scale=grad_scale(ro["gscale"]))
    assert_normwise(aout[None], ro["alpha"][None], 1e-11, "compression factor")


@pytest.mark.parametrize("name", list(FINE_CASES))
def test_adjoint_product_on_the_host_matches_oracle_differences(orc, host, name):
    """The adjoint's whole transposed product (forward-mode Jacobians of the reconstruction and the
    point flux, then the four transposed-product bodies), run on the host: w . (J v) = (J^T w) . v
    with J v a Richardson-extrapolated central difference of the oracle's (Res, Gnew).  Both ways of
    taking the reconstruction's part: from its stored forward-mode linearisation, and recomputed by
    the reverse-mode body (adjoint_recompute 1); the two products agree to round-off."""
    import meshgen as mg
    mk, prm = FINE_CASES[name]
    mesh = mk(mg)
    om, nc, nf, ngp, arrays, keep = _fine_inputs(orc, mesh)
    W, G, rng = _state(mg, nc, prm["mach"], 44)
    ones = np.ones(nc)
    os_ = orc.Solver(om, orc.params(n_levels=1, compression_factor=0, **prm))

    def Fo(x):
        os_.set_state(x[:5 * nc].reshape(5, nc), x[5 * nc:].reshape(15, nc), ones)
        r = os_.residual()
        return np.concatenate([r["res"].ravel(), r["grad"].ravel()])

    u = np.concatenate([W.ravel(), G.ravel()])
    scale = np.concatenate([np.abs(W).ravel(), (np.abs(G) + 0.1).ravel()])
    for _ in range(2):
        v = scale * rng.standard_normal(u.size)
        w = rng.standard_normal(u.size)
        outs = []
        for recompute in (0, 1):
            out = np.zeros((20, nc))
            res, Gout, aout = np.zeros((5, nc)), np.zeros((15, nc)), np.zeros(nc)
            code = host.host_fine(nc, nf, ngp, *arrays, _p(W), _p(G), _p(ones), _p(_phys_vector(prm)), 0, _p(res),
                                  _p(Gout), _p(aout), _p(w[:5 * nc]), _p(w[5 * nc:]), _p(out), recompute, None)
            assert code == 0
            outs.append(out)
        from parity import assert_normwise
        assert_normwise(outs[1].ravel()[None], outs[0].ravel()[None], 1e-12, "recomputed vs stored J^T w")

        def jv(h):
            return (Fo(u + h * v) - Fo(u - h * v)) / (2 * h)

        Jv = (4.0 * jv(0.5e-7) - jv(1e-7)) / 3.0
        for out in outs:
            lhs, rhs = float(w @ Jv), float(out.ravel() @ v)
            assert abs(lhs - rhs) <= 1e-6 * float(np.abs(w) @ np.abs(Jv)), (name, lhs, rhs)
