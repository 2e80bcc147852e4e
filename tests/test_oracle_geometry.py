"""Pins of the oracle's mesh geometry and reconstruction (Sec. 2.2 and 3 of the paper) against
closed forms, the divergence theorem and polynomial exactness."""
import numpy as np
import pytest

import meshgen as mg


def _box(split_kind, n=3, jitter=0.0, periodic=(False, False, False)):
    bc = dict(xmin=3, xmax=3, ymin=3, ymax=3, zmin=3, zmax=3)
    return mg.box_mesh(n, n, n, lambda i, j, k: np.full(np.shape(i), split_kind), periodic=periodic,
                       bc={k: v for k, v in bc.items()}, jitter=jitter)


def test_unjittered_cell_moments_closed_forms(orc):
    h = 1.0 / 3.0
    # hexahedra: volume h^3, centroid at the cell centre, central moments h^2/12 I
    M = orc.Mesh(_box(0))
    vol, ctr, m2 = M.cells()
    np.testing.assert_allclose(vol, h ** 3, rtol=1e-14)
    np.testing.assert_allclose(m2[:, :3], h * h / 12.0, rtol=1e-13)
    np.testing.assert_allclose(m2[:, 3:], 0.0, atol=1e-17)
    # right prisms: triangle moments (1/12) sum (v - c)(v - c)^T, uniform along the axis
    mesh = _box(1)
    M = orc.Mesh(mesh)
    vol, ctr, m2 = M.cells()
    np.testing.assert_allclose(vol, h ** 3 / 2.0, rtol=1e-13)
    X = mesh["xyz"][mesh["cell_nodes"].reshape(-1, 6)]
    tri = X[:, :3, :2]
    c = tri.mean(axis=1)
    d = tri - c[:, None, :]
    np.testing.assert_allclose(ctr[:, :2], c, atol=1e-15)
    np.testing.assert_allclose(m2[:, 0], (d[:, :, 0] ** 2).sum(1) / 12.0, rtol=1e-12)
    np.testing.assert_allclose(m2[:, 1], (d[:, :, 1] ** 2).sum(1) / 12.0, rtol=1e-12)
    np.testing.assert_allclose(m2[:, 3], (d[:, :, 0] * d[:, :, 1]).sum(1) / 12.0, rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose(m2[:, 2], h * h / 12.0, rtol=1e-12)
    # Kuhn tetrahedra: volume h^3/6
    M = orc.Mesh(_box(3))
    vol, _, _ = M.cells()
    np.testing.assert_allclose(vol, h ** 3 / 6.0, rtol=1e-13)


NFACES = {4: 4, 5: 5, 6: 6, 7: 5}


@pytest.mark.parametrize("kind", ["periodic", "farfield", "pyramids"])
def test_jittered_mixed_mesh_divergence_theorem(orc, kind):
    """Per cell: sum of outward area vectors = 0, |Omega| = (1/3) sum x.dA and
    int x_d dV = (1/2) sum x_d^2 dA_d (the face rules are exact for these integrands on bilinear
    faces), so the volume quadrature is pinned by the surface quadrature (pyramids included)."""
    if kind == "periodic":
        mesh = mg.periodic_box(6)
    elif kind == "farfield":
        mesh = mg.scale_box(6)
    else:
        mesh = mg.pyramid_box(6)
    M = orc.Mesh(mesh)
    vol, ctr, m2 = M.cells()
    F = M.faces()
    assert abs(vol.sum() - 1.0) < 1e-13
    S = np.zeros((M.nc, 3))
    V3 = np.zeros(M.nc)
    C2 = np.zeros((M.nc, 3))
    for i in range(M.nc):
        for m in range(NFACES[int(mesh["cell_type"][i])]):
            f, side = F["cf"][i, m], F["cside"][i, m]
            k = F["ngp"][f]
            dA = F["gA"][f, :k] * (-1.0 if side else 1.0)
            x = F["gx"][f, :k] - (F["shift"][f] if side else 0.0)
            S[i] += dA.sum(0)
            V3[i] += (x * dA).sum() / 3.0
            C2[i] += 0.5 * (x * x * dA).sum(0)
    assert np.abs(S).max() < 1e-15
    np.testing.assert_allclose(V3, vol, rtol=1e-12)
    np.testing.assert_allclose(C2 / vol[:, None], ctr, rtol=0, atol=1e-13)


def test_second_moments_against_higher_order_rule(orc):
    """The 3-point (or closed-form) second moments equal a 5-point tensor rule on every cell type."""
    mesh = mg.periodic_box(4)
    M = orc.Mesh(mesh)
    vol, ctr, m2 = M.cells()
    pts, w = M.qpoints(5)
    np.testing.assert_allclose(w.sum(1), vol, rtol=1e-13)
    d = pts - ctr[:, None, :]
    for q, (a, b) in enumerate([(0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (0, 2)]):
        got = (w * d[:, :, a] * d[:, :, b]).sum(1) / vol
        np.testing.assert_allclose(got, m2[:, q], rtol=1e-10, atol=1e-17)


def _interior_cells(M):
    F = M.faces()
    bad = np.zeros(M.nc, bool)
    for f in range(M.nf):
        if F["fR"][f] < 0 or F["tag"][f] >= 100:
            bad[F["fL"][f]] = True
            if F["fR"][f] >= 0:
                bad[F["fR"][f]] = True
    return ~bad


def _quadratic_data(M, coef):
    """Exact cell averages and averaged gradients of q(x) = a + b.x + x^T H x / 2."""
    vol, ctr, m2 = M.cells()
    a, b, H = coef
    val = a + ctr @ b + 0.5 * np.einsum("ni,ij,nj->n", ctr, H, ctr)
    val += 0.5 * (H[0, 0] * m2[:, 0] + H[1, 1] * m2[:, 1] + H[2, 2] * m2[:, 2]) + H[0, 1] * m2[:, 3] + H[1, 2] * m2[:, 4] + H[0, 2] * m2[:, 5]
    grad = b[None, :] + ctr @ H.T
    return val, grad


def _taylor_coeffs(ctr, coef):
    a, b, H = coef
    out = np.zeros((len(ctr), 10))
    out[:, 0] = a + ctr @ b + 0.5 * np.einsum("ni,ij,nj->n", ctr, H, ctr)
    out[:, 1:4] = b[None, :] + ctr @ H.T
    out[:, 4], out[:, 5], out[:, 6] = 0.5 * H[0, 0], 0.5 * H[1, 1], 0.5 * H[2, 2]
    out[:, 7], out[:, 8], out[:, 9] = H[0, 1], H[1, 2], H[0, 2]
    return out


def _state_from(fields):
    base = np.array([1.0, 0.2, 0.0, 0.0, 2.5])
    W = np.stack([base[q] + 0.05 * fields[q][0] for q in range(5)])
    G = np.zeros((15, W.shape[1]))
    for q in range(5):
        G[3 * q:3 * q + 3] = 0.05 * fields[q][1].T
    return W, G


@pytest.mark.parametrize("kind", ["mixed", "pyramids"])
def test_p2_reproduces_quadratic_fields(orc, kind):
    """The constrained least-squares p^2 (Sec. 3.1) is exact for quadratic data on the jittered
    mixed mesh and on a box with pyramids (cells whose stencil has no boundary face)."""
    mesh = mg.scale_box(7) if kind == "mixed" else mg.pyramid_box(7, periodic=False)
    M = orc.Mesh(mesh)
    S = orc.Solver(M, orc.params(mach=0.2, n_levels=1))
    rng = np.random.default_rng(0)
    coefs = []
    for _ in range(5):
        H = rng.normal(size=(3, 3))
        coefs.append((rng.normal(), rng.normal(size=3), 0.5 * (H + H.T)))
    fields = [_quadratic_data(M, c) for c in coefs]
    W, G = _state_from(fields)
    S.set_state(W, G)
    rc = S.reconstruct(mode=1)
    inner = _interior_cells(M)
    _, ctr, _ = M.cells()
    base = np.array([1.0, 0.2, 0.0, 0.0, 2.5])
    for q in range(5):
        expect = 0.05 * _taylor_coeffs(ctr, coefs[q])
        expect[:, 0] += base[q]
        np.testing.assert_allclose(rc[inner, q], expect[inner], rtol=0, atol=1e-11)


def test_green_gauss_and_weno_exact_for_linear_data_on_uniform_hexes(orc):
    """On an unjittered hexahedral grid the Green-Gauss p^1 (Sec. 3.2) is exact for linear data,
    both smoothness indicators agree, the WENO weights (Sec. 3.4) are the linear ones and R is the
    exact linear field."""
    mesh = _box(0, n=5)
    M = orc.Mesh(mesh)
    S = orc.Solver(M, orc.params(mach=0.2, n_levels=1))
    rng = np.random.default_rng(1)
    coefs = [(rng.normal(), rng.normal(size=3), np.zeros((3, 3))) for _ in range(5)]
    fields = [_quadratic_data(M, c) for c in coefs]
    W, G = _state_from(fields)
    S.set_state(W, G)
    inner = _interior_cells(M)
    _, ctr, _ = M.cells()
    base = np.array([1.0, 0.2, 0.0, 0.0, 2.5])
    for mode in (2, 0):
        rc = S.reconstruct(mode=mode)
        for q in range(5):
            expect = 0.05 * _taylor_coeffs(ctr, coefs[q])
            expect[:, 0] += base[q]
            np.testing.assert_allclose(rc[inner, q], expect[inner], rtol=0, atol=1e-12)


def test_weno_falls_back_towards_p1_at_a_discontinuity(orc):
    """At a density jump the non-linear weights move to the Green-Gauss sub-stencil, so the
    curvature of R (2 w_2 times that of p^2) is far below the curvature of p^2 next to the jump."""
    mesh = _box(0, n=6)
    M = orc.Mesh(mesh)
    S = orc.Solver(M, orc.params(mach=0.2, n_levels=1))
    _, ctr, _ = M.cells()
    rho = np.where(ctr[:, 0] < 0.5, 1.0, 2.0)
    W = np.stack([rho, 0.2 * rho, 0 * rho, 0 * rho, 2.5 + 0.02 * rho])
    S.set_state(W, np.zeros((15, M.nc)))
    r = S.reconstruct(mode=0)[:, 0, 4]
    p2 = S.reconstruct(mode=1)[:, 0, 4]
    near = np.abs(ctr[:, 0] - 0.5) < 0.1
    assert np.all(np.abs(p2[near]) > 10.0)
    assert np.all(np.abs(r[near]) < 0.3 * np.abs(p2[near]))


def test_coarsening_geometry(orc):
    """The coarsening's geometry: node-mean centres, face area vectors from the diagonals (exact for
    flat triangles and bilinear quadrilaterals), divergence-theorem volumes.  On an unjittered mixed
    box every face is flat, so volumes and area vectors equal the quadrature ones and the cells
    close; tetrahedron centres are centroids."""
    mesh = mg.periodic_box(6, jitter=0.0) if "jitter" in mg.periodic_box.__code__.co_varnames else None
    if mesh is None:
        pytest.skip("periodic_box without a jitter argument")
    M = orc.Mesh(mesh)
    vol, ctr, Sn, area = M.coarsening_geometry()
    rvol, rctr, _ = M.cells()
    np.testing.assert_allclose(vol, rvol, rtol=1e-13)
    np.testing.assert_allclose(area, np.linalg.norm(Sn, axis=1), rtol=1e-15)
    F = M.faces()
    qS = F["gA"].sum(axis=1)
    np.testing.assert_allclose(Sn, qS, rtol=0, atol=1e-15 * np.abs(qS).max())
    tets = np.asarray(mesh["cell_type"]) == 4
    np.testing.assert_allclose(ctr[tets], rctr[tets], rtol=0, atol=1e-15)
    nodes = mesh["xyz"][mesh["cell_nodes"]]
    owner = np.repeat(np.arange(len(mesh["cell_type"])), np.diff(mesh["cell_ptr"]))
    mean = np.zeros((len(mesh["cell_type"]), 3))
    np.add.at(mean, owner, nodes)
    mean /= np.diff(mesh["cell_ptr"])[:, None]
    np.testing.assert_allclose(ctr, mean, rtol=0, atol=1e-15)
    # closure of every cell: the outward canonical area vectors of its faces sum to zero
    clos = np.zeros((M.nc, 3))
    np.add.at(clos, F["fL"], Sn)
    inner = F["fR"] >= 0
    np.add.at(clos, F["fR"][inner], -Sn[inner])
    assert np.abs(clos).max() < 1e-15


def test_pyramid_closed_forms(orc):
    """Unjittered pyramids (six per grid cell of side h around its centre): volume h^3/6, centroid a
    quarter of the way from the base centre to the apex, and the canonical coarsening volume equal."""
    n = 6
    h = 1.0 / n
    mesh = mg.pyramid_box(n, jitter=0.0)
    M = orc.Mesh(mesh)
    vol, ctr, _ = M.cells()
    pyr = np.nonzero(np.asarray(mesh["cell_type"]) == 7)[0]
    assert len(pyr) == 6 * (n - 2 * (n // 3)) ** 3
    np.testing.assert_allclose(vol[pyr], h ** 3 / 6.0, rtol=1e-13)
    X = mesh["xyz"][mesh["cell_nodes"][mesh["cell_ptr"][pyr][:, None] + np.arange(5)]]
    base = X[:, :4].mean(axis=1)
    np.testing.assert_allclose(ctr[pyr], base + 0.25 * (X[:, 4] - base), rtol=0, atol=1e-15)
    cvol = M.coarsening_geometry()[0]
    np.testing.assert_allclose(cvol[pyr], h ** 3 / 6.0, rtol=1e-13)
