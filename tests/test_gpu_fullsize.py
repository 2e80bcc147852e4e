"""Parity at the full size of the benchmark workload, in the configuration bench.py times: the
96x64x64 boundary-layer box (1,327,104 cells, 3 levels, M 0.5, Re 1e4, Pr 0.72).  The oracle runs
the same computations over the whole mesh (tens of seconds on the host cores), so every output is
compared, not a sample.  Tolerances as in the small parity tests: integer outputs bit-exact, FP64
residuals within 1e-11 of the magnitude of the terms they sum, states after a V-cycle within 1e-11."""
import numpy as np
import pytest

import meshgen as mg
from parity import assert_normwise, grad_scale

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PRM = dict(mach=0.5, reynolds=1e4, prandtl=0.72, gamma=1.4, viscous=1, n_levels=3, cfl_fine=0.5,
           cfl_coarse=0.9, coarse_steps=2, agglo_seed=0)


@pytest.fixture(scope="module")
def cg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_02075_gb300 as cg
    from paper_2402_02075_gb300 import build
    build.build()
    return cg


@pytest.fixture(scope="module")
def pair(cg, orc):
    mesh = mg.wall_box(96, 64, 64)
    ctx = cg.upload_mesh(mesh, cg.default_params(**PRM))
    os_ = orc.Solver(orc.Mesh(mesh), orc.params(**PRM))
    # a free stream with cell-to-cell perturbations of 2 % and random gradients (seeded)
    rng = np.random.default_rng(11)
    W, G = mg.uniform_state(ctx.nc, mach=0.5)
    W = W * (1.0 + 0.02 * rng.standard_normal(W.shape))
    G = 0.05 * rng.standard_normal(G.shape)
    yield ctx, os_, W, G
    ctx.close()


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_hierarchy_is_bit_exact(pair):
    ctx, os_, _, _ = pair
    assert ctx.nc == 1_327_104
    for lev in (1, 2):
        ref = os_.level(lev)
        assert np.array_equal(ctx.coarse_map(lev).cpu().numpy(), ref["map"])
        g = ctx.level_geometry(lev)
        assert np.array_equal(g["fL"].cpu().numpy(), ref["fL"])
        assert np.array_equal(g["fR"].cpu().numpy(), ref["fR"])
        # the coarsening's geometry is one formula with a fixed order of correctly rounded operations
        assert np.array_equal(g["vol"].cpu().numpy(), ref["vol"])
        assert np.array_equal(g["Sn"].cpu().numpy(), ref["Sn"].T)


def test_cgks_residual_full_size(pair):
    ctx, os_, W, G = pair
    ctx.state_init(_t(W), _t(G))
    os_.set_state(W, G)
    r = ctx.residual(order=3)
    ro = os_.residual()
    assert_normwise(r["dt"].cpu().numpy()[None], ro["dt"][None], 1e-13, "time steps")
    assert_normwise(r["res"].cpu().numpy(), ro["res"], 1e-11, "residual", scale=ro["fscale"])
    assert_normwise(r["grad"].cpu().numpy(), ro["grad"], 1e-11, "Gauss-Green gradients",
                    scale=grad_scale(ro["gscale"]))
    assert_normwise(r["alpha"].cpu().numpy()[None], ro["alpha"][None], 1e-11, "compression factor")


def test_coarse_kfvs_full_size(pair):
    ctx, os_, _, _ = pair
    rng = np.random.default_rng(12)
    for lev in (1, 2):
        n = ctx.level_info(lev)[0]
        Wl, _ = mg.uniform_state(n, mach=0.5)
        Wl = Wl * (1.0 + 0.02 * rng.standard_normal(Wl.shape))
        assert_normwise(ctx.kfvs_residual(lev, _t(Wl)).cpu().numpy(), os_.kfvs_residual(lev, Wl), 1e-12,
                        f"KFVS residual level {lev}")


def test_vcycle_full_size(pair):
    """One V-cycle of the bench configuration from the perturbed state."""
    ctx, os_, W, G = pair
    ctx.state_init(_t(W), _t(G))
    os_.set_state(W, G)
    hg = ctx.vcycle(1)
    ho = os_.run(1, multigrid=True)
    np.testing.assert_allclose(hg, ho, rtol=1e-11)
    Wg = ctx.state_get()[0].cpu().numpy()
    Wo = os_.state()[0]
    assert np.abs(Wg - Wo).max() <= 1e-11 * np.abs(Wo).max(), np.abs(Wg - Wo).max()
    assert ctx.skipped_updates() == os_.skipped()
