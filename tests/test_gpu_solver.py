"""Explicit steps, coarsening, coarse levels and V-cycles of the CUDA library against the oracle,
plus determinism and the error paths of the C ABI."""
import numpy as np
import pytest

import meshgen as mg
from parity import assert_normwise

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_02075_gb300 as cg
    from paper_2402_02075_gb300 import build
    build.build()
    return cg


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _pair(cg, orc, mesh, W, G, **prm):
    ctx = cg.upload_mesh(mesh, cg.default_params(**prm))
    ctx.state_init(_t(W), _t(G))
    om = orc.Mesh(mesh)
    os_ = orc.Solver(om, orc.params(**prm))
    os_.set_state(W, G)
    return ctx, om, os_


def _gg_amplification(om):
    """per cell: the sum over its faces of the Gauss points' |area vector|, over its volume: the
    factor by which the Gauss-Green gradient (alpha/|Omega|) sum_p W_p A_p (Sec. 3) scales a
    difference in the interface states W_p"""
    vol = om.cells()[0]
    F = om.faces()
    used = (np.arange(4)[None, :] < F["ngp"][:, None])
    fa = np.where(used, np.linalg.norm(F["gA"], axis=2), 0.0).sum(1)
    ct = om._src["cell_type"]
    mask = np.arange(6)[None, :] < np.where(ct == 7, 5, ct)[:, None]  # pyramids (type 7) have 5 faces
    return np.where(mask, fa[np.where(mask, F["cf"], 0)], 0.0).sum(1) / vol


def _compare_states(ctx, os_, atol_w=1e-11, rtol_g=1e-10, atol_a=1e-10):
    """States after iterations: each step adds dt/|Omega| x residual, and the residuals agree to
    1e-11 of the summed flux magnitudes, so W agrees to 1e-11 of its scale.  The gradients inherit
    that difference through the Gauss-Green sum, scaled by each cell's surface over volume (large in
    the thin cells at a no-slip wall), and the compression factor (a non-smooth function of the
    reconstructed jumps) inherits it too: a gradient may differ by 1e-11 of the state's scale times
    that ratio, on top of rtol_g of its own scale."""
    Wg, Gg, ag = (x.cpu().numpy() for x in ctx.state_get())
    Wo, Go, ao = os_.state()
    assert np.abs(Wg - Wo).max() <= atol_w * np.abs(Wo).max(), np.abs(Wg - Wo).max()
    bound = atol_w * np.abs(Wo).max() * _gg_amplification(os_.mesh)[None, :] + rtol_g * np.abs(Go).max()
    dG = np.abs(Gg - Go)
    assert (dG <= bound).all(), (dG.max(), (dG / bound).max())
    assert np.abs(ag - ao).max() <= atol_a, np.abs(ag - ao).max()


def test_config1_hundred_steps(cg, orc):
    """The 16^3 mixed periodic density wave (6,912 cells), global time step, CFL 0.5, 100 steps."""
    mesh = mg.periodic_box(16)
    W, G = mg.density_wave_state(mesh)
    ctx, om, os_ = _pair(cg, orc, mesh, W, G, mach=0.2, dt_mode=1, cfl_fine=0.5, n_levels=1)
    hg = ctx.step(100)
    ho = os_.run(100)
    np.testing.assert_allclose(hg, ho, rtol=1e-9)
    _compare_states(ctx, os_)


@pytest.mark.parametrize("name,mk,seed", [
    ("periodic8", lambda: mg.periodic_box(8), 0),
    ("periodic8-s3", lambda: mg.periodic_box(8), 3),
    ("wall", lambda: mg.wall_box(16, 8, 16, n_prism=6), 0),
    ("ramp", lambda: mg.ramp_box(24, 12, 8, n_prism=3), 0),
    ("scale10", lambda: mg.scale_box(10), 1),
    ("pyramid8", lambda: mg.pyramid_box(8), 0),
])
def test_coarsening_is_bit_exact(cg, orc, name, mk, seed):
    mesh = mk()
    prm = dict(n_levels=3, agglo_seed=seed)
    ctx = cg.upload_mesh(mesh, cg.default_params(**prm))
    om = orc.Mesh(mesh)
    os_ = orc.Solver(om, orc.params(**prm))
    for lev in (1, 2):
        Lo = os_.level(lev)
        nc, nf = ctx.level_info(lev)
        assert (nc, nf) == (Lo["nc"], Lo["nf"])
        assert np.array_equal(ctx.coarse_map(lev).cpu().numpy(), Lo["map"])
        g = ctx.level_geometry(lev)
        assert np.array_equal(g["fL"].cpu().numpy(), Lo["fL"])
        assert np.array_equal(g["fR"].cpu().numpy(), Lo["fR"])
        assert np.array_equal(g["tag"].cpu().numpy(), Lo["tag"])
        assert_normwise(g["vol"].cpu().numpy()[None], Lo["vol"][None], 1e-13, "coarse volumes")
        assert_normwise(g["ctr"].cpu().numpy(), Lo["ctr"].T, 1e-13, "coarse centroids")
        assert_normwise(g["Sn"].cpu().numpy(), Lo["Sn"].T, 1e-12, "coarse area vectors",
                        scale=np.full((3, 1), np.abs(Lo["Sn"]).max()))


@pytest.mark.parametrize("mk", [lambda: mg.periodic_box(8), lambda: mg.wall_box(16, 8, 16, n_prism=6),
                                lambda: mg.ramp_box(24, 12, 8, n_prism=3), lambda: mg.prism_slab()])
def test_coarse_kfvs_residuals(cg, orc, mk):
    mesh = mk()
    prm = dict(n_levels=3, mach=0.6)
    ctx = cg.upload_mesh(mesh, cg.default_params(**prm))
    om = orc.Mesh(mesh)
    os_ = orc.Solver(om, orc.params(**prm))
    rng = np.random.default_rng(3)
    for lev in (0, 1, 2):
        n = ctx.level_info(lev)[0]
        W, _ = mg.uniform_state(n, mach=0.6)
        W = W * (1 + 0.03 * rng.standard_normal(W.shape))
        got = ctx.kfvs_residual(lev, _t(W)).cpu().numpy()
        ref = os_.kfvs_residual(lev, W)
        assert_normwise(got, ref, 1e-12, f"KFVS residual level {lev}")


@pytest.mark.parametrize("case", ["wave", "wall", "ramp", "slab", "pyramid"])
def test_vcycles(cg, orc, case):
    rng = np.random.default_rng(11)
    if case == "wave":
        mesh = mg.periodic_box(8)
        W, G = mg.density_wave_state(mesh)
        prm = dict(mach=0.2)
        n = 4
    elif case == "wall":
        mesh = mg.wall_box(16, 8, 16, n_prism=6)
        W, G = mg.uniform_state(len(mesh["cell_type"]), mach=0.5)
        prm = dict(mach=0.5, viscous=1, reynolds=1e4, prandtl=0.72)
        n = 3
    elif case == "ramp":
        mesh = mg.ramp_box(24, 12, 8, n_prism=3)
        W, G = mg.uniform_state(len(mesh["cell_type"]), mach=3.0)
        prm = dict(mach=3.0)
        n = 3
    elif case == "pyramid":  # hexahedra around a block of pyramids, farfield on every side
        mesh = mg.pyramid_box(8, periodic=False)
        W, G = mg.uniform_state(len(mesh["cell_type"]), mach=0.5)
        W = W * (1 + 0.01 * rng.standard_normal(W.shape))
        prm = dict(mach=0.5, viscous=1, reynolds=1e3, prandtl=0.72)
        n = 3
    else:  # a level-2 coarse face of zero net area
        mesh = mg.prism_slab()
        W, G = mg.uniform_state(len(mesh["cell_type"]), mach=0.5)
        prm = dict(mach=0.5, viscous=1, reynolds=1e4, prandtl=0.72)
        n = 3
    ctx, om, os_ = _pair(cg, orc, mesh, W, G, n_levels=3, **prm)
    hg = ctx.vcycle(n)
    ho = os_.run(n, multigrid=True)
    np.testing.assert_allclose(hg, ho, rtol=1e-9)
    _compare_states(ctx, os_)
    assert ctx.skipped_updates() == os_.skipped()


def test_runs_are_bitwise_reproducible(cg):
    mesh = mg.periodic_box(8)
    W, G = mg.density_wave_state(mesh)
    outs = []
    for _ in range(2):
        ctx = cg.upload_mesh(mesh, cg.default_params(mach=0.2))
        ctx.state_init(_t(W), _t(G))
        h = ctx.vcycle(3)
        outs.append((h, [x.cpu().numpy() for x in ctx.state_get()]))
        ctx.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    for a, b in zip(outs[0][1], outs[1][1]):
        assert np.array_equal(a, b)


def test_error_paths(cg):
    with pytest.raises(cg.CgksError) as e:
        cg.Context(cg.default_params(gamma=0.9))
    assert e.value.status == 1
    with pytest.raises(cg.CgksError) as e:
        cg.Context(cg.default_params(precision=2))
    assert e.value.status == 1
    mesh = mg.periodic_box(4)
    ctx = cg.Context(cg.default_params())
    with pytest.raises(cg.CgksError) as e:
        ctx.step(1)
    assert e.value.status == 1  # no mesh
    broken = dict(mesh)
    broken["bface_tag"] = mesh["bface_tag"][:-2].copy()
    broken["bface_ptr"] = mesh["bface_ptr"][:-2].copy()
    broken["periodic_pairs"] = mesh["periodic_pairs"][:-1].copy()
    with pytest.raises(cg.CgksError) as e:
        ctx.mesh_upload(broken)
    assert e.value.status in (1, 4)
    ctx.mesh_upload(mesh)
    with pytest.raises(cg.CgksError) as e:
        ctx.residual()
    assert e.value.status == 1  # no state
    W, G = mg.uniform_state(ctx.nc)
    W[0, 5] = -1.0
    ctx.state_init(_t(W), _t(G))
    with pytest.raises(cg.CgksError) as e:
        ctx.step(1)
    assert e.value.status == 5 and "index" in str(e.value)
    # the adjoint needs the compression factor off (it is on by default)
    with pytest.raises(cg.CgksError) as e:
        ctx.linearize()
    assert e.value.status == 8
    with pytest.raises(cg.CgksError) as e:
        ctx.adjoint(1)
    assert e.value.status == 8
    ctx.close()


@pytest.mark.parametrize("mk", [lambda: mg.periodic_box(8), lambda: mg.wall_box(16, 8, 16, n_prism=6),
                                lambda: mg.prism_slab()])
def test_lusgs_colours_are_bit_exact(cg, orc, mk):
    mesh = mk()
    ctx = cg.upload_mesh(mesh, cg.default_params(n_levels=3, coarse_smoother=1))
    S = orc.Solver(orc.Mesh(mesh), orc.params(n_levels=3, coarse_smoother=1))
    for lev in (1, 2):
        col, k = ctx.coarse_colors(lev)
        ref, kr = S.colors(lev)
        assert k == kr
        assert np.array_equal(col.cpu().numpy(), ref)
    ctx.close()


@pytest.mark.parametrize("case", ["wave", "wall", "ramp"])
def test_vcycles_with_lusgs_coarse_smoother(cg, orc, case):
    """V-cycles whose coarse levels relax with LU-SGS (Sec. 4.3) against the oracle: the colour-major
    parallel sweep equals the oracle's sequential sweep in (colour, id) order."""
    if case == "wave":
        mesh = mg.periodic_box(8)
        W, G = mg.density_wave_state(mesh)
        prm = dict(mach=0.2)
    elif case == "wall":
        mesh = mg.wall_box(16, 8, 16, n_prism=6)
        W, G = mg.uniform_state(len(mesh["cell_type"]), mach=0.5)
        prm = dict(mach=0.5, viscous=1, reynolds=1e4, prandtl=0.72)
    else:
        mesh = mg.ramp_box(24, 12, 8, n_prism=3)
        W, G = mg.uniform_state(len(mesh["cell_type"]), mach=3.0)
        prm = dict(mach=3.0)
    ctx, om, os_ = _pair(cg, orc, mesh, W, G, n_levels=3, coarse_smoother=1, **prm)
    hg = ctx.vcycle(3)
    ho = os_.run(3, multigrid=True)
    np.testing.assert_allclose(hg, ho, rtol=1e-9)
    _compare_states(ctx, os_)
    assert ctx.skipped_updates() == os_.skipped()


@pytest.mark.parametrize("extra", [dict(correction_relax=0.5), dict(prolongation=1),
                                   dict(prolongation=1, correction_relax=0.7), dict(compression_factor=0)])
def test_vcycles_with_relaxed_or_smoothed_correction(cg, orc, extra):
    """correction_relax r < 1 scales the injected coarse correction and prolongation 1 averages it
    over face neighbours, on every level, the same way in the oracle."""
    mesh = mg.wall_box(16, 8, 16, n_prism=6)
    W, G = mg.uniform_state(len(mesh["cell_type"]), mach=0.5)
    prm = dict(mach=0.5, viscous=1, reynolds=1e4, prandtl=0.72, **extra)
    ctx, om, os_ = _pair(cg, orc, mesh, W, G, n_levels=3, **prm)
    hg = ctx.vcycle(3)
    ho = os_.run(3, multigrid=True)
    np.testing.assert_allclose(hg, ho, rtol=1e-9)
    _compare_states(ctx, os_)


@pytest.mark.parametrize("extra", [dict(coarse_steps=1, cfl_coarse=0.5), dict(coarse_steps=3),
                                   dict(coarse_steps=2, post=1)])
def test_vcycles_with_other_coarse_smoothing(cg, orc, extra):
    """Other numbers of coarse forward-Euler steps, coarse CFL numbers and post-smoothing steps
    (the paper fixes none of them) follow the oracle's V-cycle the same way."""
    mesh = mg.wall_box(16, 8, 16, n_prism=6)
    W, G = mg.uniform_state(len(mesh["cell_type"]), mach=0.5)
    prm = dict(mach=0.5, viscous=1, reynolds=1e4, prandtl=0.72, **extra)
    ctx, om, os_ = _pair(cg, orc, mesh, W, G, n_levels=3, **prm)
    hg = ctx.vcycle(3)
    ho = os_.run(3, multigrid=True)
    np.testing.assert_allclose(hg, ho, rtol=1e-9)
    _compare_states(ctx, os_)


@pytest.mark.parametrize("multigrid,extra", [(False, {}), (True, {}), (True, dict(precision=1)),
                                             (True, dict(coarse_smoother=1))],
                         ids=["single grid", "V-cycle", "mixed V-cycle", "LU-SGS V-cycle"])
def test_graph_replayed_steady_solve_equals_eager_iterations(cg, multigrid, extra):
    """cgks_steady_solve replays its chunks of 10 iterations as a captured CUDA graph after the first
    chunk: 50 iterations of it leave bit for bit the state, gradients and compression factors of 50
    eagerly launched iterations (cgks_step / cgks_vcycle), with the same residual norms."""
    mesh = mg.wall_box(12, 4, 12, first=2e-3, ratio=1.3, outflow=mg.BC_SUPER_OUT)
    prm = dict(mach=0.5, viscous=1, reynolds=1e4, prandtl=0.72, n_levels=3, **extra)
    out = []
    for graphs in (True, False):
        ctx = cg.upload_mesh(mesh, cg.default_params(**prm))
        W, G = mg.uniform_state(ctx.nc, mach=0.5)
        ctx.state_init(_t(W), _t(G))
        if graphs:
            r = ctx.steady_solve(multigrid=multigrid, drop=1e-300, max_iters=50, raise_on_notconv=False)
            assert r["iters"] == 50 and not r["converged"]
            last = r["drop"]
        else:
            h = ctx.vcycle(50) if multigrid else ctx.step(50)
            last = h[-1] / h[0]
        out.append(([x.cpu().numpy() for x in ctx.state_get()], last))
        ctx.close()
    for a, b in zip(out[0][0], out[1][0]):
        assert np.array_equal(a, b)
    assert out[0][1] == out[1][1]
