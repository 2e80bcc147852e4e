"""CPU oracle of the multigrid compact gas-kinetic scheme (arXiv 2402.02075).

TEST INFRASTRUCTURE ONLY: a plain, slow FP64 C implementation written from the paper, used by the
tests, the smoke check and the benchmark's CPU-baseline leg to check and time the CUDA library.  The
product library never imports, links or calls it, and it shares no code with the CUDA path.

Functions without an independent pin ("parity unpinned" in the design notes): the Prandtl-number
correction of the energy flux beyond its Pr = 1 reduction, the choice of the kinetic-weighted
interface gradient of the equilibrium state (its half-space moment terms are pinned by quadrature;
the paper prints no number for the reading), and the skewness limit value (the paper gives none).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = ["orc_linalg.c", "orc_mesh.c", "orc_gks.c", "orc_solver.c", "orc_agglo.c", "orc_lusgs.c", "orc_api.c"]
_LIB = os.path.join(_HERE, "liborc.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -ffp-contract=off, no fast-math) into oracle/liborc.so."""
    srcs = [os.path.join(_HERE, s) for s in _SRCS]
    newest = max(os.path.getmtime(s) for s in srcs + [os.path.join(_HERE, "orc.h")])
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-D_DEFAULT_SOURCE",
               "-fPIC", "-shared", "-fopenmp", "-o", tmp] + srcs + ["-lm"]
        subprocess.run(cmd, check=True, cwd=_HERE)
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("mach", C.c_double), ("reynolds", C.c_double),
                ("prandtl", C.c_double), ("aoa", C.c_double * 2), ("cfl_fine", C.c_double),
                ("cfl_coarse", C.c_double), ("eps_inviscid", C.c_double), ("c_press", C.c_double),
                ("weno_eps", C.c_double), ("skew_min", C.c_double), ("sutherland", C.c_double), ("correction_relax", C.c_double),
                ("n_levels", C.c_int32), ("pre", C.c_int32), ("post", C.c_int32),
                ("coarse_steps", C.c_int32), ("passes_per_level", C.c_int32), ("viscous", C.c_int32),
                ("dt_mode", C.c_int32), ("precision", C.c_int32), ("coarse_smoother", C.c_int32), ("compression_factor", C.c_int32), ("prolongation", C.c_int32),
                ("agglo_seed", C.c_uint64)]


def params(**kw) -> Params:
    """Defaults are the readings of the paper's free constants (eps = 0.01, C = 1, WENO eps = 1e-5,
    3 levels, 1 pre- and 0 post-smoothing steps, 2 coarse forward-Euler steps at CFL 0.9, 2 passes per
    level)."""
    d = dict(gamma=1.4, mach=0.2, reynolds=1e4, prandtl=1.0, aoa=(0.0, 0.0), cfl_fine=0.5,
             cfl_coarse=0.9, eps_inviscid=0.01, c_press=1.0, weno_eps=1e-5, skew_min=0.2, sutherland=0.0, correction_relax=1.0,
             n_levels=3, pre=1, post=0, coarse_steps=2, passes_per_level=2, viscous=0,
             dt_mode=0, precision=0, coarse_smoother=0, compression_factor=1, prolongation=0, agglo_seed=0)
    d.update(kw)
    p = Params()
    for k, v in d.items():
        if k == "aoa":
            p.aoa[0], p.aoa[1] = v
        else:
            setattr(p, k, v)
    return p


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.c_void_p
        d = C.POINTER(C.c_double)
        i32 = C.POINTER(C.c_int32)
        i64 = C.POINTER(C.c_int64)
        _lib.orc_mesh_new.restype = P
        _lib.orc_mesh_new.argtypes = [C.c_int64, d, C.c_int64, C.POINTER(C.c_int8), i64, i32, C.c_int64,
                                      i64, i32, i32, C.c_int64, i32, C.c_char_p]
        _lib.orc_mesh_delete.argtypes = [P]
        _lib.orc_mesh_counts.argtypes = [P, i64]
        _lib.orc_mesh_cells.argtypes = [P, d, d, d]
        _lib.orc_mesh_coarsening_geometry.argtypes = [P, d, d, d, d]
        _lib.orc_mesh_faces.argtypes = [P, i32, i32, i32, i32, d, d, d, i32, C.POINTER(C.c_int8)]
        _lib.orc_mesh_qpoints.argtypes = [P, C.POINTER(C.c_int8), i64, i32, d, C.c_int, d, d]
        _lib.orc_new.restype = P
        _lib.orc_new.argtypes = [P, C.POINTER(Params), C.c_char_p]
        _lib.orc_delete.argtypes = [P]
        _lib.orc_set_state.argtypes = [P, d, d, d]
        _lib.orc_get_state.argtypes = [P, d, d, d]
        _lib.orc_residual.argtypes = [P, d, d, d, d, d]
        _lib.orc_run.argtypes = [P, C.c_int, C.c_int, d]
        _lib.orc_skipped.restype = C.c_int64
        _lib.orc_skipped.argtypes = [P]
        _lib.orc_reconstruct.argtypes = [P, d, C.c_int]
        _lib.orc_level_counts.argtypes = [P, C.c_int, i64]
        _lib.orc_level_data.argtypes = [P, C.c_int, i32, d, d, i32, i32, i32, d, d]
        _lib.orc_kfvs_residual.argtypes = [P, C.c_int, d, d]
        _lib.orc_level_dt.argtypes = [P, C.c_int, d, d]
        _lib.orc_colors.argtypes = [P, C.c_int, C.POINTER(C.c_int32)]
        _lib.orc_lusgs.argtypes = [P, C.c_int, d, d, d, d, C.POINTER(C.c_int64)]
        _lib.orc_pt_moments.argtypes = [d, C.c_double, C.c_int, d]
        _lib.orc_pt_slope.argtypes = [d, C.c_double, d, d]
        _lib.orc_pt_mom_term.restype = C.c_double
        _lib.orc_pt_mom_term.argtypes = [d, C.c_double, C.c_int, C.c_int, C.c_int, C.c_int, d, C.c_int]
        _lib.orc_pt_time.argtypes = [C.c_double, C.c_double, C.c_double, d]
        _lib.orc_pt_gks.argtypes = [C.POINTER(Params), d, d, d, d, d, C.c_double, d, d]
        _lib.orc_pt_kfvs.argtypes = [C.POINTER(Params), d, d, d, d]
        _lib.orc_pt_cf.restype = C.c_double
        _lib.orc_pt_cf.argtypes = [C.POINTER(Params), d, d, d]
        _lib.orc_pt_ghost.argtypes = [C.POINTER(Params), C.c_int, d, d, d, d, d]
        _lib.orc_pt_frame.argtypes = [d, d, d]
        _lib.orc_pt_hash.restype = C.c_uint64
        _lib.orc_pt_hash.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64]
        _lib.orc_term_scales.argtypes = [P, d, d]
        _lib.orc_pt_splitmix64.restype = C.c_uint64
        _lib.orc_pt_splitmix64.argtypes = [C.c_uint64]
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Mesh:
    """Fine mesh: topology, face Gauss points and cell volume moments."""

    def __init__(self, m):
        L = lib()
        self._src = {k: np.ascontiguousarray(v) for k, v in m.items() if isinstance(v, np.ndarray)}
        s = self._src
        err = C.create_string_buffer(256)
        pairs = s["periodic_pairs"].astype(np.int32).reshape(-1)
        self.h = L.orc_mesh_new(len(s["xyz"]), _p(_f64(s["xyz"]), C.c_double), len(s["cell_type"]),
                                _p(s["cell_type"].astype(np.int8), C.c_int8), _p(s["cell_ptr"].astype(np.int64), C.c_int64),
                                _p(s["cell_nodes"].astype(np.int32), C.c_int32), len(s["bface_tag"]),
                                _p(s["bface_ptr"].astype(np.int64), C.c_int64), _p(s["bface_nodes"].astype(np.int32), C.c_int32),
                                _p(s["bface_tag"].astype(np.int32), C.c_int32), len(pairs) // 2,
                                _p(pairs, C.c_int32), err)
        if not self.h:
            raise ValueError("oracle mesh: " + err.value.decode())
        cnt = np.zeros(5, np.int64)
        L.orc_mesh_counts(self.h, _p(cnt, C.c_int64))
        self.nc, self.nf, self.n_int, self.n_per, self.n_bnd = (int(x) for x in cnt)

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_mesh_delete(self.h)
            self.h = None

    def cells(self):
        vol, ctr, m2 = np.zeros(self.nc), np.zeros((self.nc, 3)), np.zeros((self.nc, 6))
        lib().orc_mesh_cells(self.h, _p(vol, C.c_double), _p(ctr, C.c_double), _p(m2, C.c_double))
        return vol, ctr, m2

    def coarsening_geometry(self):
        """(vol, ctr [nc][3], Sn [nf][3], area) of the fine level as the coarsening sees it: node-mean
        centres, area vectors from the diagonals, divergence-theorem volumes."""
        vol, ctr = np.zeros(self.nc), np.zeros((self.nc, 3))
        Sn, area = np.zeros((self.nf, 3)), np.zeros(self.nf)
        lib().orc_mesh_coarsening_geometry(self.h, _p(vol, C.c_double), _p(ctr, C.c_double), _p(Sn, C.c_double),
                                           _p(area, C.c_double))
        return vol, ctr, Sn, area

    def faces(self):
        nf, nc = self.nf, self.nc
        fL, fR, tag, ngp = (np.zeros(nf, np.int32) for _ in range(4))
        gx, gA, sh = np.zeros((nf, 4, 3)), np.zeros((nf, 4, 3)), np.zeros((nf, 3))
        cf, cs = np.zeros((nc, 6), np.int32), np.zeros((nc, 6), np.int8)
        lib().orc_mesh_faces(self.h, _p(fL, C.c_int32), _p(fR, C.c_int32), _p(tag, C.c_int32), _p(ngp, C.c_int32),
                             _p(gx, C.c_double), _p(gA, C.c_double), _p(sh, C.c_double), _p(cf, C.c_int32),
                             _p(cs, C.c_int8))
        return dict(fL=fL, fR=fR, tag=tag, ngp=ngp, gx=gx, gA=gA, shift=sh, cf=cf, cside=cs)

    def qpoints(self, n1d=5):
        s = self._src
        nq = n1d ** 3
        pts, w = np.zeros((self.nc, nq, 3)), np.zeros((self.nc, nq))
        rc = lib().orc_mesh_qpoints(self.h, _p(s["cell_type"].astype(np.int8), C.c_int8),
                                    _p(s["cell_ptr"].astype(np.int64), C.c_int64),
                                    _p(s["cell_nodes"].astype(np.int32), C.c_int32), _p(_f64(s["xyz"]), C.c_double),
                                    n1d, _p(pts, C.c_double), _p(w, C.c_double))
        assert rc == 0
        return pts, w


class Solver:
    """Oracle solver state (W, gradW, compression factor) on a mesh with its coarse levels."""

    def __init__(self, mesh: Mesh, prm: Params):
        self.mesh = mesh
        self.prm = prm
        err = C.create_string_buffer(256)
        self.h = lib().orc_new(mesh.h, C.byref(prm), err)
        if not self.h:
            raise ValueError("oracle solver: " + err.value.decode())

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_delete(self.h)
            self.h = None

    def set_state(self, W, G=None, alpha=None):
        W = _f64(W)
        G = None if G is None else _f64(G)
        a = None if alpha is None else _f64(alpha)
        lib().orc_set_state(self.h, _p(W, C.c_double), None if G is None else _p(G, C.c_double),
                            None if a is None else _p(a, C.c_double))

    def state(self):
        n = self.mesh.nc
        W, G, a = np.zeros((5, n)), np.zeros((15, n)), np.zeros(n)
        lib().orc_get_state(self.h, _p(W, C.c_double), _p(G, C.c_double), _p(a, C.c_double))
        return W, G, a

    def residual(self):
        n = self.mesh.nc
        R, G, a, dt, nm = np.zeros((5, n)), np.zeros((15, n)), np.zeros(n), np.zeros(n), np.zeros(1)
        rc = lib().orc_residual(self.h, _p(R, C.c_double), _p(G, C.c_double), _p(a, C.c_double),
                                _p(dt, C.c_double), _p(nm, C.c_double))
        if rc:
            raise RuntimeError(f"oracle residual failed ({rc})")
        fs, gs = np.zeros((5, n)), np.zeros((5, n))
        lib().orc_term_scales(self.h, _p(fs, C.c_double), _p(gs, C.c_double))
        # fscale: per cell and component, sum over its Gauss points of |weight x flux| (the terms the
        # residual adds up); gscale: the same for |weight x interface state| / |Omega| (gradients)
        return dict(res=R, grad=G, alpha=a, dt=dt, norm=float(nm[0]), fscale=fs, gscale=gs)

    def run(self, n, multigrid=False):
        h = np.zeros(max(n, 1))
        rc = lib().orc_run(self.h, int(bool(multigrid)), int(n), _p(h, C.c_double))
        if rc:
            raise RuntimeError(f"oracle run failed ({rc})")
        return h[:n]

    def skipped(self):
        return int(lib().orc_skipped(self.h))

    def reconstruct(self, mode=0):
        """[nc][5][10] coefficients in the basis 1,X,Y,Z,X^2,Y^2,Z^2,XY,YZ,XZ about each centroid;
        mode 0: the WENO combination R, 1: p^2 alone, 2: p^1 alone."""
        rc = np.zeros((self.mesh.nc, 5, 10))
        if lib().orc_reconstruct(self.h, _p(rc, C.c_double), int(mode)):
            raise RuntimeError("oracle reconstruction failed")
        return rc

    def level(self, lev):
        cnt = np.zeros(4, np.int64)
        if lib().orc_level_counts(self.h, lev, _p(cnt, C.c_int64)):
            raise IndexError(lev)
        nc, nf = int(cnt[0]), int(cnt[1])
        nfiner = self.level(lev - 1)["nc"] if lev > 0 else 0
        m = np.zeros(nfiner, np.int32)
        vol, ctr = np.zeros(nc), np.zeros((nc, 3))
        fL, fR, tag = (np.zeros(nf, np.int32) for _ in range(3))
        Sn, area = np.zeros((nf, 3)), np.zeros(nf)
        lib().orc_level_data(self.h, lev, _p(m, C.c_int32) if nfiner else None, _p(vol, C.c_double),
                             _p(ctr, C.c_double), _p(fL, C.c_int32), _p(fR, C.c_int32), _p(tag, C.c_int32),
                             _p(Sn, C.c_double), _p(area, C.c_double))
        return dict(nc=nc, nf=nf, n_int=int(cnt[2]), n_per=int(cnt[3]), map=m, vol=vol, ctr=ctr,
                    fL=fL, fR=fR, tag=tag, Sn=Sn, area=area)

    def kfvs_residual(self, lev, W):
        W = _f64(W)
        R = np.zeros_like(W)
        if lib().orc_kfvs_residual(self.h, lev, _p(W, C.c_double), _p(R, C.c_double)):
            raise RuntimeError("oracle kfvs residual failed")
        return R

    def colors(self, lev):
        """(colour per cell, number of colours) of the LU-SGS ordering of level lev."""
        n = self.level(lev)["nc"]
        col = np.zeros(n, np.int32)
        k = lib().orc_colors(self.h, lev, _p(col, C.c_int32))
        if k < 0:
            raise IndexError(lev)
        return col, k

    def lusgs(self, lev, W, rhs, dt):
        """One LU-SGS step (Sec. 4.3) on level lev: (W + dU, cells skipped by positivity)."""
        W, rhs, dt = _f64(W), _f64(rhs), _f64(dt)
        out = np.zeros_like(W)
        sk = C.c_int64()
        if lib().orc_lusgs(self.h, lev, _p(W, C.c_double), _p(rhs, C.c_double), _p(dt, C.c_double),
                           _p(out, C.c_double), C.byref(sk)):
            raise RuntimeError("oracle LU-SGS step failed")
        return out, sk.value

    def level_dt(self, lev, W):
        W = _f64(W)
        dt = np.zeros(W.shape[1])
        lib().orc_level_dt(self.h, lev, _p(W, C.c_double), _p(dt, C.c_double))
        return dt


# ---- point-wise functions ------------------------------------------------------------------

def moments(rho, U, V, W, lam, K, space):
    out = np.zeros(26)
    g = _f64([rho, U, V, W, lam])
    lib().orc_pt_moments(_p(g, C.c_double), K, space, _p(out, C.c_double))
    return dict(u=out[:9], v=out[9:16], w=out[16:23], xi=out[23:26])


def slope(rho, U, V, W, lam, K, dW):
    g = _f64([rho, U, V, W, lam])
    dW = _f64(dW)
    s = np.zeros(5)
    rc = lib().orc_pt_slope(_p(g, C.c_double), K, _p(dW, C.c_double), _p(s, C.c_double))
    assert rc == 0
    return s


def mom_term(rho, U, V, W, lam, K, space, ku, kv, kw, s, alpha):
    """int u^ku v^kv w^kw (s . psi) psi_alpha g over the full (0) or half (+1, -1) space; s None
    for s . psi = 1."""
    g = _f64([rho, U, V, W, lam])
    sp = None if s is None else _f64(s)
    return float(lib().orc_pt_mom_term(_p(g, C.c_double), K, space, ku, kv, kw,
                                       None if sp is None else _p(sp, C.c_double), alpha))


def time_integrals(dt, tau, tau_n):
    q = np.zeros(5)
    lib().orc_pt_time(dt, tau, tau_n, _p(q, C.c_double))
    return q


def gks_point(prm, WL, GL, WR, GR, n, dt):
    F, Wt = np.zeros(5), np.zeros(5)
    a = [_f64(x) for x in (WL, GL, WR, GR, n)]
    rc = lib().orc_pt_gks(C.byref(prm), *[_p(x, C.c_double) for x in a], dt, _p(F, C.c_double), _p(Wt, C.c_double))
    if rc:
        raise RuntimeError(f"gks_point failed ({rc})")
    return F, Wt


def kfvs_point(prm, WL, WR, n):
    F = np.zeros(5)
    a = [_f64(x) for x in (WL, WR, n)]
    rc = lib().orc_pt_kfvs(C.byref(prm), *[_p(x, C.c_double) for x in a], _p(F, C.c_double))
    assert rc == 0
    return F


def cf_alpha(prm, WL, WR, n):
    a = [_f64(x) for x in (WL, WR, n)]
    return float(lib().orc_pt_cf(C.byref(prm), *[_p(x, C.c_double) for x in a]))


def bc_ghost(prm, tag, n, W, G):
    Wg, Gg = np.zeros(5), np.zeros(15)
    a = [_f64(x) for x in (n, W, G)]
    rc = lib().orc_pt_ghost(C.byref(prm), tag, *[_p(x, C.c_double) for x in a], _p(Wg, C.c_double), _p(Gg, C.c_double))
    assert rc == 0
    return Wg, Gg


def frame(n):
    n = _f64(n)
    t1, t2 = np.zeros(3), np.zeros(3)
    lib().orc_pt_frame(_p(n, C.c_double), _p(t1, C.c_double), _p(t2, C.c_double))
    return t1, t2


def face_hash(nl, nr, nf):
    return int(lib().orc_pt_hash(nl, nr, nf))


def splitmix64(x):
    return int(lib().orc_pt_splitmix64(x))
