"""cgks_density_norm_noalloc: the residual norm for callers that cannot let the library allocate GPU
memory (a fixed, accounted memory budget; no device-wide synchronisation from allocations).  It keeps
its partial sums in a fixed array inside the loaded module, so this test checks, through the C ABI,
that two calls in a row (a larger mesh, then a smaller one, so the second call reuses scratch the first
left behind) each reproduce the norm that cgks_residual computes with its own work arrays."""
import ctypes

import numpy as np
import pytest

import meshgen as mg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

RTOL = 1e-11


def _residual_and_norm(cg, mesh):
    W, G = mg.density_wave_state(mesh)
    ctx = cg.upload_mesh(mesh, cg.default_params(mach=0.2))
    ctx.state_init(torch.from_numpy(W).cuda(), torch.from_numpy(G).cuda())
    r = ctx.residual(order=3)
    vol = ctx.level_geometry(0)["vol"]
    return ctx, r["res"][0].contiguous(), vol, r["norm"]


def test_norm_without_allocation_matches_residual_norm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_02075_gb300 as cg
    from paper_2402_02075_gb300 import build
    build.build()
    lib = cg.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    keep = []
    for mesh in (mg.periodic_box(12), mg.periodic_box(6)):
        ctx, res_rho, vol, ref = _residual_and_norm(cg, mesh)
        keep.append(ctx)
        out.fill_(float("nan"))
        status = lib.cgks_density_norm_noalloc(ctypes.c_void_p(res_rho.data_ptr()), ctypes.c_void_p(vol.data_ptr()),
                                               res_rho.numel(), stream, ctypes.c_void_p(out.data_ptr()))
        assert status == 0, lib.cgks_last_error(None)
        torch.cuda.synchronize()
        got = out.item()
        assert np.isfinite(got) and abs(got - ref) <= RTOL * ref, (got, ref)
    # more cells than the module's scratch covers: rejected with a message, nothing launched
    status = lib.cgks_density_norm_noalloc(ctypes.c_void_p(res_rho.data_ptr()), ctypes.c_void_p(vol.data_ptr()),
                                           65536 * 1024 + 1, stream, ctypes.c_void_p(out.data_ptr()))
    assert status == 1 and b"exceeds" in lib.cgks_last_error(None)
    for ctx in keep:
        ctx.close()
