"""Python binding of libcgks (include/cgks.h): multigrid compact gas-kinetic scheme on GB300.

Argument marshalling only: every step of the method runs in the CUDA kernels of libcgks.so.
Device arrays are torch CUDA tensors (float64, component-major [5][N] / [15][N]); PyTorch provides
device memory and streams.  The functions named cgks_* mirror the C entry points one to one;
`Context` is a convenience wrapper over them.  Importing this module does not need a GPU; calling
into the library does, and it fails loudly when libcgks.so has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcgks.so")
_lib = None

STATUS = {0: "CGKS_OK", 1: "CGKS_EINVAL", 2: "CGKS_ENOMEM", 3: "CGKS_ECUDA", 4: "CGKS_EMESH", 5: "CGKS_ENAN",
          6: "CGKS_ENOTCONV", 7: "CGKS_ETIMEOUT", 8: "CGKS_EUNSUPPORTED"}

# every entry point declared in include/cgks.h
EXPORTS = ["cgks_default_params", "cgks_create", "cgks_destroy", "cgks_set_params", "cgks_mesh_upload",
           "cgks_level_info", "cgks_coarse_map", "cgks_level_geometry", "cgks_fine_moments", "cgks_state_init",
           "cgks_state_get", "cgks_residual", "cgks_kfvs_residual", "cgks_kfvs_jvp", "cgks_step", "cgks_vcycle", "cgks_steady_solve",
           "cgks_coarse_colors", "cgks_skipped_updates", "cgks_linearize", "cgks_residual_vjp",
           "cgks_wall_force", "cgks_adjoint_solve", "cgks_adjoint", "cgks_fp64_peak", "cgks_profile", "cgks_kernel_stats", "cgks_density_norm_noalloc",
           "cgks_last_error"]


class CgksError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("mach", C.c_double), ("reynolds", C.c_double), ("prandtl", C.c_double),
                ("aoa", C.c_double * 2), ("cfl_fine", C.c_double), ("cfl_coarse", C.c_double),
                ("eps_inviscid", C.c_double), ("c_press", C.c_double), ("weno_eps", C.c_double),
                ("skew_min", C.c_double), ("sutherland", C.c_double), ("correction_relax", C.c_double), ("n_levels", C.c_int32), ("pre", C.c_int32), ("post", C.c_int32),
                ("coarse_steps", C.c_int32), ("passes_per_level", C.c_int32), ("viscous", C.c_int32),
                ("dt_mode", C.c_int32), ("precision", C.c_int32), ("coarse_smoother", C.c_int32), ("compression_factor", C.c_int32), ("prolongation", C.c_int32),
                ("adjoint_recompute", C.c_int32), ("agglo_seed", C.c_uint64)]


def load(path: str = LIB_PATH):
    """Load libcgks.so (raises when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with paper_2402_02075_gb300.build.build()")
        L = C.CDLL(path)
        P, d, i32, i64 = C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p
        sig = {
            "cgks_default_params": [C.POINTER(Params)],
            "cgks_create": [C.POINTER(Params), P, C.POINTER(C.c_void_p)],
            "cgks_destroy": [P],
            "cgks_set_params": [P, C.POINTER(Params)],
            "cgks_mesh_upload": [P, C.c_int64, d, C.c_int64, P, i64, i32, C.c_int64, i64, i32, i32, i32, C.c_int64],
            "cgks_level_info": [P, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64)],
            "cgks_coarse_map": [P, C.c_int, i32],
            "cgks_level_geometry": [P, C.c_int, d, d, i32, i32, i32, d],
            "cgks_fine_moments": [P, d],
            "cgks_state_init": [P, d, d, d],
            "cgks_state_get": [P, d, d, d],
            "cgks_residual": [P, C.c_int, d, d, d, d, C.POINTER(C.c_double)],
            "cgks_kfvs_residual": [P, C.c_int, d, d],
            "cgks_kfvs_jvp": [P, C.c_int, d, d, d],
            "cgks_step": [P, C.c_int, C.POINTER(C.c_double)],
            "cgks_vcycle": [P, C.c_int, C.POINTER(C.c_double)],
            "cgks_steady_solve": [P, C.c_int, C.c_double, C.c_int64, C.POINTER(C.c_int64), C.POINTER(C.c_double),
                                  C.POINTER(C.c_double)],
            "cgks_coarse_colors": [P, C.c_int, i32, C.POINTER(C.c_int32)],
            "cgks_skipped_updates": [P, C.POINTER(C.c_int64)],
            "cgks_linearize": [P],
            "cgks_residual_vjp": [P, d, d, d, d],
            "cgks_wall_force": [P, C.c_int, C.POINTER(C.c_double), d],
            "cgks_adjoint_solve": [P, d, C.c_int, C.c_int64, C.c_double, d, C.POINTER(C.c_int64),
                                   C.POINTER(C.c_double)],
            "cgks_adjoint": [P, C.c_int, d, C.c_int, C.c_double, C.c_double, C.c_int, C.c_int64, C.c_double, d,
                             C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_double)],
            "cgks_fp64_peak": [C.POINTER(C.c_double)],
            "cgks_profile": [P, C.c_int],
            "cgks_kernel_stats": [P, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_double),
                                  C.POINTER(C.c_double)],
            "cgks_density_norm_noalloc": [d, d, C.c_int64, P, d],
            "cgks_last_error": [P],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = C.c_char_p if name == "cgks_last_error" else C.c_int
        _lib = L
    return _lib


def _check(status, ctx=None):
    if status != 0:
        msg = load().cgks_last_error(ctx)
        raise CgksError(status, msg.decode() if msg else "")


def default_params(**kw) -> Params:
    p = Params()
    _check(load().cgks_default_params(C.byref(p)))
    for k, v in kw.items():
        if k == "aoa":
            p.aoa[0], p.aoa[1] = v
        else:
            setattr(p, k, v)
    return p


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _host(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _hp(a):
    return a.ctypes.data_as(C.c_void_p)


# ---- the C entry points under their own names ----------------------------------------------

def cgks_fp64_peak() -> float:
    v = C.c_double()
    _check(load().cgks_fp64_peak(C.byref(v)))
    return v.value


class Context:
    """One libcgks context bound to the current torch CUDA stream."""

    def __init__(self, params: Params | None = None, stream=None):
        import torch
        self.torch = torch
        self.params = params or default_params()
        self.stream = stream or torch.cuda.current_stream()
        h = C.c_void_p()
        _check(load().cgks_create(C.byref(self.params), C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self.h = h
        self.nc = 0

    def close(self):
        if getattr(self, "h", None):
            load().cgks_destroy(self.h)
            self.h = None

    __del__ = close

    def set_params(self, params: Params):
        _check(load().cgks_set_params(self.h, C.byref(params)), self.h)
        self.params = params

    def mesh_upload(self, m):
        xyz = _host(m["xyz"], np.float64)
        ct = _host(m["cell_type"], np.int8)
        cp = _host(m["cell_ptr"], np.int64)
        cn = _host(m["cell_nodes"], np.int32)
        bp = _host(m["bface_ptr"], np.int64)
        bn = _host(m["bface_nodes"], np.int32)
        bt = _host(m["bface_tag"], np.int32)
        pp = _host(m["periodic_pairs"], np.int32).reshape(-1)
        _check(load().cgks_mesh_upload(self.h, len(xyz), _hp(xyz), len(ct), _hp(ct), _hp(cp), _hp(cn), len(bt), _hp(bp),
                                       _hp(bn), _hp(bt), _hp(pp) if len(pp) else None, len(pp) // 2), self.h)
        self.nc = len(ct)

    def level_info(self, level):
        nc, nf = C.c_int64(), C.c_int64()
        _check(load().cgks_level_info(self.h, level, C.byref(nc), C.byref(nf)), self.h)
        return nc.value, nf.value

    def _empty(self, *shape, dtype=None):
        t = self.torch
        return t.empty(*shape, dtype=dtype or t.float64, device="cuda")

    def coarse_map(self, level):
        n_finer = self.level_info(level - 1)[0]
        out = self._empty(n_finer, dtype=self.torch.int32)
        _check(load().cgks_coarse_map(self.h, level, _ptr(out)), self.h)
        return out

    def level_geometry(self, level):
        nc, nf = self.level_info(level)
        t = self.torch
        vol, ctr = self._empty(nc), self._empty(3, nc)
        fL, fR, tag = (self._empty(nf, dtype=t.int32) for _ in range(3))
        Sn = self._empty(3, nf)
        _check(load().cgks_level_geometry(self.h, level, _ptr(vol), _ptr(ctr), _ptr(fL), _ptr(fR), _ptr(tag), _ptr(Sn)),
               self.h)
        return dict(vol=vol, ctr=ctr, fL=fL, fR=fR, tag=tag, Sn=Sn)

    def fine_moments(self):
        m2 = self._empty(6, self.nc)
        _check(load().cgks_fine_moments(self.h, _ptr(m2)), self.h)
        return m2

    def state_init(self, W, G=None, alpha=None):
        """W, G, alpha: float64 contiguous tensors on the GPU or in pinned host memory."""
        for x in (W, G, alpha):
            assert x is None or ((x.is_cuda or x.is_pinned()) and x.dtype == self.torch.float64 and x.is_contiguous())
        _check(load().cgks_state_init(self.h, _ptr(W), _ptr(G), _ptr(alpha)), self.h)

    def state_get(self):
        W, G, a = self._empty(5, self.nc), self._empty(15, self.nc), self._empty(self.nc)
        _check(load().cgks_state_get(self.h, _ptr(W), _ptr(G), _ptr(a)), self.h)
        return W, G, a

    def residual(self, order=3, grads=True):
        res, dt = self._empty(5, self.nc), self._empty(self.nc)
        G = self._empty(15, self.nc) if (grads and order == 3) else None
        a = self._empty(self.nc) if (grads and order == 3) else None
        nm = C.c_double()
        _check(load().cgks_residual(self.h, order, _ptr(res), _ptr(G), _ptr(a), _ptr(dt), C.byref(nm)), self.h)
        return dict(res=res, grad=G, alpha=a, dt=dt, norm=nm.value)

    def kfvs_residual(self, level, W):
        res = self.torch.empty_like(W)
        _check(load().cgks_kfvs_residual(self.h, level, _ptr(W), _ptr(res)), self.h)
        return res

    def kfvs_jvp(self, level, W0, dW):
        """J(W0) dW of the level's KFVS residual (FP32 forward mode, FP64 sums)."""
        out = self.torch.empty_like(W0)
        _check(load().cgks_kfvs_jvp(self.h, level, _ptr(W0), _ptr(dW), _ptr(out)), self.h)
        return out

    def step(self, n=1, history=True):
        h = np.zeros(max(n, 1))
        _check(load().cgks_step(self.h, n, h.ctypes.data_as(C.POINTER(C.c_double)) if history else None), self.h)
        return h[:n]

    def vcycle(self, n=1, history=True):
        h = np.zeros(max(n, 1))
        _check(load().cgks_vcycle(self.h, n, h.ctypes.data_as(C.POINTER(C.c_double)) if history else None), self.h)
        return h[:n]

    def coarse_colors(self, level):
        """(colour per cell, number of colours) of the LU-SGS sweep order of a coarse level."""
        n = self.level_info(level)[0]
        col = self._empty(n, dtype=self.torch.int32)
        k = C.c_int32()
        _check(load().cgks_coarse_colors(self.h, level, _ptr(col), C.byref(k)), self.h)
        return col, k.value

    def skipped_updates(self):
        """Cell updates skipped by the positivity rule since the last state_init."""
        n = C.c_int64()
        _check(load().cgks_skipped_updates(self.h, C.byref(n)), self.h)
        return n.value

    def profile(self, enable=True):
        _check(load().cgks_profile(self.h, int(bool(enable))), self.h)

    KERNELS = ("k_gks_points", "k_reconstruct", "k_gather", "k_kfvs_faces", "k_kfvs_gather", "k_coarse_dt",
               "k_forcing", "k_fe_update", "k_restrict", "k_prolong", "k_kfvs_jvp_faces", "k_norm",
               "k_gks_points_flux", "k_gather_res")

    def kernel_stats(self, which):
        """(total device ms, launches, units, algorithmic bytes) of kernel `which` (an index or a name
        of KERNELS) since profiling was enabled."""
        if isinstance(which, str):
            which = self.KERNELS.index(which)
        ms, n, u, b = C.c_double(), C.c_int64(), C.c_double(), C.c_double()
        _check(load().cgks_kernel_stats(self.h, which, C.byref(ms), C.byref(n), C.byref(u), C.byref(b)), self.h)
        return ms.value, n.value, u.value, b.value

    # ---- adjoint of the steady problem (compression_factor 0) ----
    def linearize(self):
        _check(load().cgks_linearize(self.h), self.h)

    def residual_vjp(self, res_bar, grad_bar):
        """(W_bar, G_bar) = J^T (res_bar, grad_bar) with the stored linearisation of (Res, Gnew)."""
        Wb, Gb = self._empty(5, self.nc), self._empty(15, self.nc)
        _check(load().cgks_residual_vjp(self.h, _ptr(res_bar), _ptr(grad_bar), _ptr(Wb), _ptr(Gb)), self.h)
        return Wb, Gb

    def wall_force(self, component=1, grad=False):
        J = C.c_double()
        dJ = self.torch.zeros(5, self.nc, dtype=self.torch.float64, device="cuda") if grad else None
        _check(load().cgks_wall_force(self.h, component, C.byref(J), _ptr(dJ)), self.h)
        return (J.value, dJ) if grad else J.value

    def adjoint_solve(self, dJ_du, max_iters=100000, tol=1e-10, method=0):
        """lambda of (dF/du)^T lambda = -dJ_du; method 0 transposed pseudo-time (the default: it
        converges where the explicit scheme does), 1 restarted GMRES(30) (fewer products on small
        cases, but it can stagnate)."""
        lam = self._empty(20, self.nc)
        it, rr = C.c_int64(), C.c_double()
        _check(load().cgks_adjoint_solve(self.h, _ptr(dJ_du), method, max_iters, tol, _ptr(lam), C.byref(it),
                                         C.byref(rr)), self.h)
        return lam, it.value, rr.value

    def adjoint(self, component=1, modes=None, h_mode=1e-6, h_mach=1e-6, max_iters=100000, tol=1e-10, method=0):
        """dJ/dMach and dJ/d(mode amplitudes) of the wall force at the current steady state; modes:
        host float64 [n_modes][n_nodes][3] or None."""
        n = 0 if modes is None else len(modes)
        md = None if modes is None else np.ascontiguousarray(modes, dtype=np.float64)
        out = np.zeros(max(n, 1))
        dm, it, rr = C.c_double(), C.c_int64(), C.c_double()
        _check(load().cgks_adjoint(self.h, component, None if md is None else md.ctypes.data_as(C.c_void_p), n, h_mode,
                                   h_mach, method, max_iters, tol, out.ctypes.data_as(C.c_void_p), C.byref(dm),
                                   C.byref(it), C.byref(rr)), self.h)
        return dict(dJ_dmach=dm.value, dJ_dmodes=out[:n], iters=it.value, rel_res=rr.value)

    def steady_solve(self, multigrid=True, drop=1e-10, max_iters=100000, raise_on_notconv=True):
        it, fd, sec = C.c_int64(), C.c_double(), C.c_double()
        s = load().cgks_steady_solve(self.h, int(bool(multigrid)), drop, max_iters, C.byref(it), C.byref(fd), C.byref(sec))
        if s != 6 or raise_on_notconv:
            _check(s, self.h)
        return dict(iters=it.value, drop=fd.value, seconds=sec.value, converged=s == 0)


def upload_mesh(mesh, params=None):
    """Convenience: a Context with `mesh` (a meshgen-style dict of host arrays) uploaded."""
    ctx = Context(params)
    ctx.mesh_upload(mesh)
    return ctx


def _settle(ctx, tol=1e-10, chunk=200, max_steps=200000):
    """Single-grid steps (cgks_step) until the density-residual norm is below `tol` and has stopped
    falling (its chunk minimum no more than 10 % under the previous chunk's); returns the steps."""
    steps, last = 0, float("inf")
    while steps < max_steps:
        h = ctx.step(chunk)
        steps += chunk
        if h[-1] < tol and h.min() > 0.9 * last:
            return steps
        last = min(last, float(h.min()))
    raise CgksError(6, f"no steady state within {max_steps} steps (residual {h[-1]:.3e})")


def wall_force_function(ctx: Context, mesh, modes=None, component=1, steady_tol=1e-10, max_steps=200000,
                        **adjoint_kw):
    """The wall force J(mach, amps) of the steady state as a torch function: forward sets the free-stream
    Mach number, moves the nodes of `mesh` (a meshgen-style dict) by sum_k amps_k modes_k (re-uploading
    it when the amplitudes change), runs single-grid steps from the context's current state to a steady
    state (density-residual norm below steady_tol and no longer falling) and returns cgks_wall_force;
    backward runs the discrete adjoint at that state (cgks_adjoint: dJ/dMach and dJ/d(mode amplitude)).
    `ctx` holds `mesh` (or a displaced copy) and a state; compression_factor 0, local time steps."""
    import torch
    modes_np = None if modes is None else np.ascontiguousarray(modes, dtype=np.float64)
    n_modes = 0 if modes_np is None else len(modes_np)
    current = {"amps": np.zeros(n_modes)}

    def place(amps):
        if np.array_equal(amps, current["amps"]):
            return
        W, G, a = ctx.state_get()
        moved = dict(mesh)
        moved["xyz"] = np.ascontiguousarray(mesh["xyz"] + np.tensordot(amps, modes_np, axes=1))
        ctx.mesh_upload(moved)
        ctx.state_init(W, G, a)
        current["amps"] = amps.copy()

    class _WallForce(torch.autograd.Function):
        @staticmethod
        def forward(fctx, mach, amps):
            a = amps.detach().cpu().numpy().astype(np.float64).reshape(-1)
            if a.size != n_modes:
                raise ValueError(f"expected {n_modes} mode amplitudes, got {a.size}")
            prm = ctx.params
            prm.mach = float(mach)
            ctx.set_params(prm)
            place(a)
            _settle(ctx, steady_tol, max_steps=max_steps)
            return torch.tensor(ctx.wall_force(component), dtype=torch.float64)

        @staticmethod
        def backward(fctx, gout):
            g = ctx.adjoint(component, modes_np, **adjoint_kw)
            s = float(gout)
            return (torch.tensor(s * g["dJ_dmach"], dtype=torch.float64),
                    torch.as_tensor(s * g["dJ_dmodes"], dtype=torch.float64))

    return _WallForce.apply
