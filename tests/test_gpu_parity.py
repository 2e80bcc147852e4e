"""CUDA library (through the C ABI) against the oracle on the same seeded inputs.

Tolerances: integer outputs (faces, coarse maps) bit-exact; FP64 quantities within 1e-11
normwise relative (the kernels and the oracle round differently: FMA contraction, other summation
orders, closed-form instead of eliminated 5x5 systems)."""
import numpy as np
import pytest

import meshgen as mg
from parity import assert_normwise, grad_scale

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

RTOL = 1e-11


@pytest.fixture(scope="module")
def cg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_02075_gb300 as cg
    from paper_2402_02075_gb300 import build
    build.build()
    return cg


def _pair(cg, orc, mesh, **prm):
    ctx = cg.upload_mesh(mesh, cg.default_params(**prm))
    om = orc.Mesh(mesh)
    os_ = orc.Solver(om, orc.params(**prm))
    return ctx, om, os_


MESHES = {
    "periodic6": lambda: mg.periodic_box(6),
    "periodic16": lambda: mg.periodic_box(16),
    "wall": lambda: mg.wall_box(12, 8, 12, n_prism=5),
    "ramp": lambda: mg.ramp_box(16, 8, 8, n_prism=3),
    "scale8": lambda: mg.scale_box(8),
    "pyramid6": lambda: mg.pyramid_box(6),
    "pyramid6-farfield": lambda: mg.pyramid_box(6, periodic=False),
}


@pytest.mark.parametrize("name", list(MESHES))
def test_geometry_and_faces(cg, orc, name):
    mesh = MESHES[name]()
    ctx, om, _ = _pair(cg, orc, mesh, n_levels=1)
    g = ctx.level_geometry(0)
    vol, ctr, m2 = om.cells()
    F = om.faces()
    assert np.array_equal(g["fL"].cpu().numpy(), F["fL"])
    assert np.array_equal(g["fR"].cpu().numpy(), F["fR"])
    assert np.array_equal(g["tag"].cpu().numpy(), F["tag"])
    assert_normwise(g["vol"].cpu().numpy()[None], vol[None], 1e-13, "volumes")
    assert_normwise(g["ctr"].cpu().numpy(), ctr.T, 1e-14, "centroids")
    assert_normwise(ctx.fine_moments().cpu().numpy(), m2.T, 1e-12, "second moments",
                    scale=np.full((6, 1), np.abs(m2).max()))
    Sn = np.stack([F["gA"][f, :F["ngp"][f]].sum(0) for f in range(om.nf)]).T
    assert_normwise(g["Sn"].cpu().numpy(), Sn, 1e-13, "area vectors")


def _state(mesh, nc, kind, mach=0.5):
    """density wave, or a free stream with random cell-to-cell perturbations (small enough at high
    Mach number that every reconstructed Gauss-point state stays physical)."""
    if kind == "wave":
        return mg.density_wave_state(mesh)
    rng = np.random.default_rng(5)
    amp = 0.02 if mach < 1.0 else 0.003
    W, G = mg.uniform_state(nc, mach=mach)
    W = W * (1.0 + amp * rng.standard_normal(W.shape))
    G = 2.5 * amp * rng.standard_normal(G.shape)
    return W, G


@pytest.mark.parametrize("name,kind,prm", [
    ("periodic6", "wave", dict(mach=0.2)),
    ("periodic16", "wave", dict(mach=0.2)),
    ("periodic6", "noise", dict(mach=0.5, viscous=1, reynolds=200.0, prandtl=0.72)),
    ("wall", "noise", dict(mach=0.5, viscous=1, reynolds=1e4, prandtl=0.72)),
    ("wall", "noise", dict(mach=0.5, viscous=1, reynolds=1e4, prandtl=0.72, sutherland=110.4 / 288.15)),
    ("wall", "noise", dict(mach=0.5, viscous=1, reynolds=1e4, prandtl=0.72, compression_factor=0)),
    ("ramp", "noise", dict(mach=3.0)),
    ("scale8", "noise", dict(mach=0.8, viscous=1, reynolds=1e5, prandtl=0.72)),
    ("pyramid6", "wave", dict(mach=0.2)),
    ("pyramid6-farfield", "noise", dict(mach=0.5, viscous=1, reynolds=1e3, prandtl=0.72)),
])
def test_cgks_residual(cg, orc, name, kind, prm):
    mesh = MESHES[name]()
    ctx, om, os_ = _pair(cg, orc, mesh, n_levels=1, **prm)
    W, G = _state(mesh, om.nc, kind, prm["mach"])
    rng = np.random.default_rng(1)
    alpha = 1.0 - 0.1 * rng.random(om.nc)
    ctx.state_init(torch.from_numpy(W).cuda(), torch.from_numpy(G).cuda(), torch.from_numpy(alpha).cuda())
    os_.set_state(W, G, alpha)
    r = ctx.residual(order=3)
    ro = os_.residual()
    assert_normwise(r["dt"].cpu().numpy()[None], ro["dt"][None], 1e-13, "time steps")
    assert_normwise(r["res"].cpu().numpy(), ro["res"], RTOL, "residual", scale=ro["fscale"])
    assert_normwise(r["grad"].cpu().numpy(), ro["grad"], RTOL, "Gauss-Green gradients", scale=grad_scale(ro["gscale"]))
    assert_normwise(r["alpha"].cpu().numpy()[None], ro["alpha"][None], RTOL, "compression factor")
    # the density-residual norm against the norm of the oracle residual, bounded by the same scale
    vol = om.cells()[0]
    bound = RTOL * np.sqrt(np.mean((ro["fscale"][0] / vol) ** 2))
    assert abs(r["norm"] - ro["norm"]) <= bound


@pytest.mark.parametrize("name", ["periodic6", "wall", "ramp", "pyramid6-farfield"])
def test_kfvs_residual_fine_level(cg, orc, name):
    mesh = MESHES[name]()
    ctx, om, os_ = _pair(cg, orc, mesh, n_levels=1, mach=0.5)
    W, G = _state(mesh, om.nc, "noise")
    Wt = torch.from_numpy(W).cuda()
    got = ctx.kfvs_residual(0, Wt).cpu().numpy()
    ref = os_.kfvs_residual(0, W)
    assert_normwise(got, ref, RTOL, "KFVS residual")
