"""Pins of the oracle's dense discrete adjoint (the steady problem of Sec. 2.4 and 4 with the
compression factor off) against central differences of the converged wall-force functional: the
adjoint gradient needs only the linearisation at one steady state, the difference needs two more
steady solves, so the two share nothing but the residual itself.  Tolerance 1e-5 relative (the
accuracy asked of the adjoint gradients)."""
import numpy as np
import pytest

import meshgen as mg


@pytest.fixture(scope="module")
def ramp(orc):
    from oracle import adjoint as adj
    mesh = mg.ramp_box(8, 4, 2, n_prism=1)
    W0, G0 = mg.uniform_state(len(mesh["cell_type"]), mach=3.0)
    prm = dict(mach=3.0)
    W, G, steps = adj.solve_steady(mesh, dict(prm, compression_factor=0), W0, G0)
    assert steps < 20000
    modes = mg.ramp_wall_modes(mesh, 4)
    res = adj.adjoint_gradient(mesh, prm, W, G, modes=modes[:1])
    return adj, mesh, prm, W, G, modes, res


def test_wall_force_derivative_is_its_difference_quotient(ramp):
    adj, mesh, prm, W, G, _, res = ramp
    import oracle as orc
    om = orc.Mesh(mesh)
    rng = np.random.default_rng(3)
    v = rng.standard_normal(W.shape) * W
    h = 1e-6
    fd = (adj.wall_force(om, W + h * v, 1.4) - adj.wall_force(om, W - h * v, 1.4)) / (2 * h)
    assert abs(res["dJdu"][:W.size] @ v.ravel() - fd) <= 1e-8 * abs(fd)


def test_adjoint_mach_gradient_matches_converged_difference(ramp):
    adj, mesh, prm, W, G, _, res = ramp
    fd = adj.fd_gradient(mesh, prm, W, G)
    assert abs(res["dJ_dmach"] - fd) <= 1e-5 * abs(fd), (res["dJ_dmach"], fd)


def test_adjoint_mode_gradient_matches_converged_difference(ramp):
    adj, mesh, prm, W, G, modes, res = ramp
    fd = adj.fd_gradient(mesh, prm, W, G, field=modes[0])
    assert abs(res["dJ_dmodes"][0] - fd) <= 1e-5 * abs(fd), (res["dJ_dmodes"][0], fd)


def test_adjoint_solves_the_transposed_system(ramp):
    _, _, _, W, G, _, res = ramp
    A, lam, g = res["A"], res["lam"], res["dJdu"]
    assert np.linalg.norm(A.T @ lam + g) <= 1e-10 * np.linalg.norm(g)
    # the steady problem is well posed: the linearisation is far from singular
    assert np.linalg.cond(A) < 1e10


def test_wall_force_of_a_uniform_pressure_is_pressure_times_projected_area(orc):
    """For a uniform pressure p the ramp's wall force in y is -p times the wall's projection on the
    x-z plane, 2 x L_z (x from -0.5 to 1.5; the area vectors point out of the fluid, into the wall)."""
    from oracle import adjoint as adj
    for nx, ny, nz in ((8, 4, 2), (12, 6, 4)):
        mesh = mg.ramp_box(nx, ny, nz, n_prism=1)
        om = orc.Mesh(mesh)
        W, _ = mg.uniform_state(om.nc, mach=3.0)
        p = 1.0 / 1.4
        Lz = nz * 2.0 / nx
        assert abs(adj.wall_force(om, W, 1.4) - (-p * 2.0 * Lz)) <= 1e-12 * p * 2.0 * Lz
        assert abs(adj.wall_force(om, W, 1.4, comp=2)) <= 1e-14


def test_ramp_wall_modes_keep_periodic_copies_together_and_cells_valid(orc):
    mesh = mg.ramp_box(16, 8, 4, n_prism=2)
    modes = mg.ramp_wall_modes(mesh, 8)
    xyz = mesh["xyz"]
    ptr, nodes = mesh["bface_ptr"], mesh["bface_nodes"]
    for a, b in np.asarray(mesh["periodic_pairs"]).reshape(-1, 2):
        na, nb = nodes[ptr[a]:ptr[a + 1]], nodes[ptr[b]:ptr[b + 1]]
        # each node of face a has a partner on face b at the same x, y
        for i in na:
            j = nb[np.argmin(np.abs(xyz[nb, 0] - xyz[i, 0]) + np.abs(xyz[nb, 1] - xyz[i, 1]))]
            assert np.array_equal(modes[:, i], modes[:, j])
    # amplitude 1e-3 (far above the differencing steps) leaves every cell with a positive volume
    for m in modes:
        vol = orc.Mesh(mg.displaced(mesh, m, 1e-3)).cells()[0]
        assert vol.min() > 0.0
