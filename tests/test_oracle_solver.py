"""Pins of the oracle's residual, explicit step and V-cycle (Sec. 2.2, 2.4, 4.2 of the paper):
free-stream preservation, discrete conservation, the 1-level V-cycle, determinism and design
order on a smooth travelling density wave."""
import numpy as np

import meshgen as mg


def _uniform(orc, mesh, **kw):
    M = orc.Mesh(mesh)
    S = orc.Solver(M, orc.params(**kw))
    W, G = mg.uniform_state(M.nc, mach=kw.get("mach", 0.2), aoa=kw.get("aoa", (0.0, 0.0)))
    S.set_state(W, G)
    return M, S, W


def test_free_stream_preserved_on_jittered_mixed_mesh(orc):
    M, S, W = _uniform(orc, mg.periodic_box(6), mach=0.3, aoa=(20.0, 10.0))
    vol, _, _ = M.cells()
    r = S.residual()
    flux_scale = np.abs(W).max() * vol.max() ** (2.0 / 3.0)
    assert np.abs(r["res"]).max() < 1e-13 * flux_scale
    assert np.abs(r["grad"]).max() < 1e-12
    np.testing.assert_allclose(r["alpha"], 1.0, atol=1e-15)
    S.run(2, multigrid=True)
    Wn, Gn, _ = S.state()
    np.testing.assert_allclose(Wn, W, rtol=0, atol=1e-13)


def test_free_stream_preserved_with_slip_walls_and_farfield(orc):
    """A uniform flow parallel to slip walls, with farfield (Riemann-invariant) in/outflow."""
    mesh = mg.box_mesh(5, 4, 4, mg.quadrant_split(3, 3), periodic=(False, False, True), jitter=0.05,
                       bc=dict(xmin=3, xmax=3, ymin=1, ymax=1))
    M, S, W = _uniform(orc, mesh, mach=0.4)
    vol, _, _ = M.cells()
    r = S.residual()
    assert np.abs(r["res"]).max() < 1e-13 * np.abs(W).max() * vol.max() ** (2.0 / 3.0)
    S.run(2, multigrid=True)
    Wn, _, _ = S.state()
    np.testing.assert_allclose(Wn, W, rtol=0, atol=1e-13)


def _wave(orc, n=6, **kw):
    mesh = mg.periodic_box(n)
    M = orc.Mesh(mesh)
    S = orc.Solver(M, orc.params(mach=0.2, **kw))
    W, G = mg.density_wave_state(mesh)
    S.set_state(W, G)
    return M, S, W, G


def test_fluxes_telescope_on_periodic_mesh(orc):
    M, S, W, _ = _wave(orc)
    r = S.residual()
    tot = r["res"].sum(axis=1)
    assert np.all(np.abs(tot) < 1e-14 * np.abs(r["res"]).sum(axis=1).max())


def test_vcycle_conserves_total_mass_momentum_energy(orc):
    """With one global time step per level, sum |Omega| W is conserved by the fine step, and the
    coarse corrections add sum_c dt (Res_c + F_c) = 0 because every residual telescopes."""
    M, S, W, _ = _wave(orc, dt_mode=1)
    vol, _, _ = M.cells()
    before = W @ vol
    S.run(3, multigrid=True)
    Wn, _, _ = S.state()
    np.testing.assert_allclose(Wn @ vol, before, rtol=1e-14, atol=1e-15)


def test_one_level_vcycle_is_the_single_grid_step(orc):
    _, S1, _, _ = _wave(orc, n_levels=1)
    _, S2, _, _ = _wave(orc, n_levels=3)
    h1 = S1.run(3, multigrid=True)
    h2 = S2.run(3, multigrid=False)
    assert np.array_equal(h1, h2)
    for a, b in zip(S1.state(), S2.state()):
        assert np.array_equal(a, b)


def test_runs_are_bitwise_reproducible(orc):
    _, S1, _, _ = _wave(orc)
    _, S2, _, _ = _wave(orc)
    assert np.array_equal(S1.run(2, multigrid=True), S2.run(2, multigrid=True))
    for a, b in zip(S1.state(), S2.state()):
        assert np.array_equal(a, b)


def test_kfvs_levels_free_stream_and_telescoping(orc):
    M, S, W = _uniform(orc, mg.periodic_box(8), mach=0.3, aoa=(10.0, 0.0))
    for lev in (1, 2):
        L = S.level(lev)
        Wl = np.repeat(W[:, :1], L["nc"], axis=1)
        R = S.kfvs_residual(lev, Wl)
        assert np.abs(R).max() < 1e-13 * L["area"].max()
        rng = np.random.default_rng(lev)
        Wp = Wl * (1.0 + 0.01 * rng.normal(size=Wl.shape))
        R = S.kfvs_residual(lev, Wp)
        assert np.all(np.abs(R.sum(axis=1)) < 1e-14 * np.abs(R).sum(axis=1).max())


def _wave_error(orc, n, cfl, T=0.1, mixed=False):
    """L1 density error of a travelling density wave rho = 1 + 0.01 sin(2 pi (x - U t)) after time T,
    on n x 4 x 4 periodic cubes of side 1/n in y and z (hexahedra, or the quadrant layout of
    hexahedra, both prism orientations and Kuhn tetrahedra with 5 % jitter), global time step."""
    h = 1.0 / n
    if mixed:
        mesh = mg.box_mesh(n, 4, 4, mg.quadrant_split(3 * n // 4, 3), ys=np.arange(5) * h, zs=np.arange(5) * h,
                           periodic=(True, True, True), jitter=0.05)
    else:
        mesh = mg.box_mesh(n, 4, 4, lambda i, j, k: np.zeros(np.shape(i), int), periodic=(True, True, True))
    M = orc.Mesh(mesh)
    pts, w = M.qpoints(4)
    vol = w.sum(1)
    U, g = 0.2, 1.4

    def avg(t):
        ph = 2 * np.pi * (pts[..., 0] - U * t)
        rho, drho = 1 + 0.01 * np.sin(ph), 0.02 * np.pi * np.cos(ph)
        R, D = (w * rho).sum(1) / vol, (w * drho).sum(1) / vol
        Wv = np.stack([R, U * R, 0 * R, 0 * R, 1 / g / (g - 1) + 0.5 * U * U * R])
        G = np.zeros((15, M.nc))
        G[0], G[3], G[12] = D, U * D, 0.5 * U * U * D
        return Wv, G

    def solver(c):
        return orc.Solver(M, orc.params(mach=U, dt_mode=1, n_levels=1, cfl_fine=c))

    S = solver(cfl)
    S.set_state(*avg(0.0))
    t = 0.0
    while t < T - 1e-14:
        dt = S.residual()["dt"][0]
        if t + dt > T:
            last = solver(cfl * (T - t) / dt)
            last.set_state(*S.state())
            last.run(1)
            S, t = last, T
            break
        S.run(1)
        t += dt
    We, _ = avg(T)
    Wn, _, _ = S.state()
    return np.sum(vol * np.abs(Wn[0] - We[0])) / vol.sum()


def test_design_order_on_smooth_density_wave(orc):
    """Third-order reconstruction with second-order time accuracy: on hexahedra at CFL 0.2 the
    error of a travelling density wave falls at a rate of at least 2.2 per grid halving."""
    e1 = _wave_error(orc, 16, 0.2)
    e2 = _wave_error(orc, 32, 0.2)
    assert e1 < 2e-5
    assert np.log2(e1 / e2) > 2.2


def test_design_order_on_jittered_mixed_elements(orc):
    """The same wave on the jittered quadrant layout (hexahedra, prisms of both orientations, Kuhn
    tetrahedra) at CFL 0.05, where the time error is small: over 8, 16 and 32 cells per wavelength
    the error falls at a rate of at least 2.5 per halving (third order in space)."""
    e = [_wave_error(orc, n, 0.05, T=0.05, mixed=True) for n in (8, 16, 32)]
    rates = [np.log2(e[i] / e[i + 1]) for i in range(2)]
    assert e[0] < 1e-4
    assert min(rates) >= 2.5, (e, rates)


def test_zero_area_coarse_face_carries_no_flux(orc):
    """A coarse face with zero net area vector contributes nothing (it has no normal); the KFVS
    residual stays finite, keeps the free stream and telescopes, and V-cycles conserve mass, momentum
    and energy on that hierarchy."""
    M, S, W = _uniform(orc, mg.prism_slab(periodic=True), mach=0.5, n_levels=3, dt_mode=1)
    L = S.level(2)
    area = np.linalg.norm(L["Sn"], axis=1)
    assert (area == 0.0).sum() == 1
    Wl = np.repeat(W[:, :1], L["nc"], axis=1)
    assert np.abs(S.kfvs_residual(2, Wl)).max() < 1e-13 * area.max()
    rng = np.random.default_rng(2)
    Wp = Wl * (1.0 + 0.01 * rng.normal(size=Wl.shape))
    R = S.kfvs_residual(2, Wp)
    assert np.isfinite(R).all()
    assert np.all(np.abs(R.sum(axis=1)) < 1e-14 * np.abs(R).sum(axis=1).max())
    # a perturbed fine state through two V-cycles: totals conserved (dt_mode 1, periodic)
    vol, _, _ = M.cells()
    Wf = W * (1.0 + 0.01 * rng.normal(size=W.shape))
    S.set_state(Wf, np.zeros((15, M.nc)))
    before = Wf @ vol
    S.run(2, multigrid=True)
    np.testing.assert_allclose(S.state()[0] @ vol, before, rtol=1e-13, atol=1e-15)


def test_compression_factor_off_gives_alpha_one(orc):
    """compression_factor = 0: every Gauss-point factor, hence every cell's alpha, is exactly 1."""
    M = orc.Mesh(mg.periodic_box(6))
    S = orc.Solver(M, orc.params(mach=0.5, compression_factor=0))
    rng = np.random.default_rng(3)
    W, G = mg.uniform_state(M.nc, mach=0.5)
    S.set_state(W * (1 + 0.05 * rng.standard_normal(W.shape)), 0.1 * rng.standard_normal(G.shape))
    assert np.all(S.residual()["alpha"] == 1.0)
    S1 = orc.Solver(M, orc.params(mach=0.5))
    S1.set_state(*S.state()[:2])
    assert np.any(S1.residual()["alpha"] < 1.0)


def test_free_stream_preserved_with_pyramids(orc):
    M, S, W = _uniform(orc, mg.pyramid_box(6), mach=0.3, aoa=(15.0, 5.0), viscous=1, reynolds=100.0)
    vol, _, _ = M.cells()
    r = S.residual()
    assert np.abs(r["res"] / vol).max() < 1e-11
    S.run(2, multigrid=True)
    np.testing.assert_allclose(S.state()[0], W, rtol=0, atol=1e-13)
