"""Pins of oracle parts whose only other checks were parity or invariants that a plausible mistake
would survive:

- the local time step (a free reading of the paper's local time stepping, Sec. 4.2 and 4.3):
  dt_i = CFL |Omega_i| / sum_p S_p (|U_i . n_p| + c_i + 2 nu_i S_p / |Omega_i|), nu = mu / rho, worked
  out here from node coordinates of single hand-built cells, and on the coarse KFVS levels from the
  grid lines of a graded Cartesian box and the coarse maps (each coarse face's summed area and the
  direction of its summed area vector);
- the skewness confirmation of the coarsening (Sec. 4.1, Eqs. virtual center and skewness factor,
  read as the cosine between d_f = face centre - C_c and the face normal over the faces of the merged
  cell that are not between its two halves, C_c the volume-weighted centre): a hand-built pair whose
  merge flips at the value computed here;
- the FAS V-cycle (Sec. 4.2): from a converged steady state one V-cycle changes nothing beyond
  round-off (the forcing F = Res* - Res_2h(W^0) cancels the coarse residual exactly when
  Res* = 0), and near a steady state the coarse correction speeds convergence up.
"""
import numpy as np
import pytest

import meshgen as mg

GAMMA = 1.4


def _affine(A, b):
    A = np.asarray(A, dtype=float)

    def f(x, y, z):
        p = np.stack([x, y, z])
        q = A @ p + np.asarray(b, dtype=float)[:, None]
        return q[0], q[1], q[2]
    return f


A_MAP = [[1.0, 0.35, 0.2], [0.1, 0.8, -0.15], [0.45, -0.15, 1.3]]


def _cell_nodes(mesh, i):
    return mesh["xyz"][mesh["cell_nodes"][mesh["cell_ptr"][i]:mesh["cell_ptr"][i + 1]]]


def _hex_faces(P):
    """area vectors and areas of a parallelepiped's six (planar) faces from its corner nodes"""
    quads = [(0, 3, 2, 1), (4, 5, 6, 7), (0, 1, 5, 4), (1, 2, 6, 5), (2, 3, 7, 6), (3, 0, 4, 7)]
    out = []
    for q in quads:
        a, b, c, d = (P[k] for k in q)
        out.append(0.5 * np.cross(c - a, d - b))
    return out


def _tet_faces(P):
    return [0.5 * np.cross(P[j] - P[i], P[k] - P[i]) for i, j, k in ((0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3))]


def _state(rho, u, p):
    u = np.asarray(u, dtype=float)
    return np.array([rho, *(rho * u), p / (GAMMA - 1.0) + 0.5 * rho * u @ u])


def _expected_dt(faces, vol, rho, u, p, cfl, mu):
    c = np.sqrt(GAMMA * p / rho)
    nu = mu / rho
    s = 0.0
    for Sv in faces:
        S = np.linalg.norm(Sv)
        s += S * (abs(np.dot(u, Sv)) / S + c + 2.0 * nu * S / vol)
    return cfl * vol / s


@pytest.mark.parametrize("viscous,reynolds,sutherland", [(0, 1e4, 0.0), (1, 20.0, 0.0), (1, 5.0, 0.4)])
def test_local_time_step_of_single_hex_and_tets(orc, viscous, reynolds, sutherland):
    """A parallelepiped hexahedron and the six Kuhn tetrahedra of another, each a mesh of its own with
    farfield boundaries: the oracle's local time step equals the closed form evaluated from the node
    coordinates.  rho != 1 separates nu from mu; the low Reynolds numbers make the viscous term a
    large part of the sum."""
    mach, cfl = 0.6, 0.37
    rho, u, p = 1.7, np.array([0.3, -0.25, 0.4]), 0.9
    T = GAMMA * p / rho  # free-stream temperature is 1 (rho = 1, p = 1/gamma)
    mu = mach / reynolds if viscous else 0.0
    if viscous and sutherland:
        mu *= T ** 1.5 * (1.0 + sutherland) / (T + sutherland)
    bc = {k: mg.BC_FARFIELD for k in ("xmin", "xmax", "ymin", "ymax", "zmin", "zmax")}
    cases = [(0, [0.0, 0.7], [0.0, 0.4], [0.0, 0.55]), (3, [0.0, 0.3], [0.0, 0.5], [0.0, 0.45])]
    for kind, xs, ys, zs in cases:
        mesh = mg.box_mesh(1, 1, 1, lambda i, j, k: np.full(np.shape(i), kind), xs=xs, ys=ys, zs=zs, bc=bc,
                           mapping=_affine(A_MAP, [0.2, -0.1, 0.05]))
        M = orc.Mesh(mesh)
        S = orc.Solver(M, orc.params(mach=mach, viscous=viscous, reynolds=reynolds, sutherland=sutherland,
                                     cfl_fine=cfl, n_levels=1))
        W = np.repeat(_state(rho, u, p)[:, None], M.nc, axis=1)
        S.set_state(W, np.zeros((15, M.nc)))
        dt = S.residual()["dt"]
        for i in range(M.nc):
            P = _cell_nodes(mesh, i)
            if kind == 0:
                faces = _hex_faces(P)
                vol = abs(np.linalg.det(np.stack([P[1] - P[0], P[3] - P[0], P[4] - P[0]])))
            else:
                faces = _tet_faces(P)
                vol = abs(np.linalg.det(np.stack([P[1] - P[0], P[2] - P[0], P[3] - P[0]]))) / 6.0
            ref = _expected_dt(faces, vol, rho, u, p, cfl, mu)
            assert abs(dt[i] - ref) <= 1e-13 * ref, (kind, i, dt[i], ref)
    # the global mode takes the smallest local step
    S1 = orc.Solver(M, orc.params(mach=mach, viscous=viscous, reynolds=reynolds, sutherland=sutherland,
                                  cfl_fine=cfl, n_levels=1, dt_mode=1))
    S1.set_state(W, np.zeros((15, M.nc)))
    assert np.all(S1.residual()["dt"] == dt.min())


def _skew_values(mesh):
    """min over the outer faces of the two-hexahedron mesh of |d . n|/(|d||n|) with C_c the
    volume-weighted node-mean centre, and the same value of the shared face and with the
    unweighted centre (what two plausible mistakes would use)."""
    P = [_cell_nodes(mesh, i) for i in range(2)]
    ctr = [q.mean(axis=0) for q in P]
    quads = [(0, 3, 2, 1), (4, 5, 6, 7), (0, 1, 5, 4), (1, 2, 6, 5), (2, 3, 7, 6), (3, 0, 4, 7)]
    faces = []  # (centre, area vector, cell)
    for c in range(2):
        for q in quads:
            a, b, cc, d = (P[c][k] for k in q)
            faces.append((np.mean([a, b, cc, d], axis=0), 0.5 * np.cross(cc - a, d - b), c))
    vols = []
    for c in range(2):
        v = 0.0
        for xc, Sv, cell in faces:
            if cell == c:
                sgn = 1.0 if np.dot(xc - ctr[c], Sv) > 0 else -1.0
                v += np.dot(xc, sgn * Sv) / 3.0
        vols.append(v)
    keys = [tuple(np.round(xc, 12)) for xc, _, _ in faces]
    shared = {k for k in keys if keys.count(k) == 2}

    def s_min(Cc, with_shared=False):
        vals = []
        for (xc, Sv, _), k in zip(faces, keys):
            if k in shared and not with_shared:
                continue
            d = xc - Cc
            vals.append(abs(np.dot(d, Sv)) / (np.linalg.norm(d) * np.linalg.norm(Sv)))
        return min(vals)
    Cw = (vols[0] * ctr[0] + vols[1] * ctr[1]) / (vols[0] + vols[1])
    return s_min(Cw), s_min(Cw, True), s_min(0.5 * (ctr[0] + ctr[1])), vols


def test_skewness_limit_flips_the_merge_of_a_hand_built_pair(orc):
    """Two hexahedra of unequal volume whose shared face (their only interior face, so the hash
    selects it) is shifted sideways, in a general affine frame.  The merge is confirmed when skew_min
    is just below the smallest face cosine worked out here and refused just above it; that flip
    point is neither the value with the shared face included nor the one with an unweighted centre."""
    bc = {k: mg.BC_FARFIELD for k in ("xmin", "xmax", "ymin", "ymax", "zmin", "zmax")}
    frame = _affine([[1.0, 0.03, 0.02], [0.02, 1.0, -0.02], [0.03, -0.01, 1.0]], [0.1, 0.0, -0.2])

    def shift_middle_layer(x, y, z):
        mid = np.isclose(x, 0.45)
        return frame(x, y + np.where(mid, 0.3, 0.0), z + np.where(mid, 0.1, 0.0))
    mesh = mg.box_mesh(2, 1, 1, lambda i, j, k: np.zeros(np.shape(i), int), xs=[0.0, 0.45, 1.0], ys=[0.0, 1.0],
                       zs=[0.0, 1.0], bc=bc, mapping=shift_middle_layer)
    s, s_shared, s_unweighted, vols = _skew_values(mesh)
    assert abs(vols[0] - vols[1]) > 0.15 * max(vols)
    assert 0.05 < s < 0.95
    # the two mistakes would flip elsewhere
    assert s_shared < 0.9 * s and abs(s_unweighted - s) > 0.05 * s, (s, s_shared, s_unweighted)
    M = orc.Mesh(mesh)
    # one coarsening pass (a second pass would see each cell's boundary faces aggregated into one)
    for k, merged in ((s * (1.0 - 1e-9), True), (s * (1.0 + 1e-9), False)):
        S = orc.Solver(M, orc.params(mach=0.3, n_levels=2, passes_per_level=1, skew_min=k))
        assert S.level(1)["nc"] == (1 if merged else 2), (k, s)


def _ramp_steady(orc, steps=1200):
    """A small supersonic ramp driven to a steady state by the oracle's own single-grid steps."""
    mesh = mg.ramp_box(16, 8, 2, n_prism=2)
    M = orc.Mesh(mesh)
    prm = dict(mach=3.0, n_levels=3)
    S = orc.Solver(M, orc.params(**prm))
    W, G = mg.uniform_state(M.nc, mach=3.0)
    S.set_state(W, G)
    h = S.run(steps)
    return mesh, M, prm, S, h


@pytest.fixture(scope="module")
def ramp(orc):
    return _ramp_steady(orc)


def test_vcycle_leaves_a_converged_state_unchanged(orc, ramp):
    """At a steady state of the fine residual the restricted defect is zero, so the FAS forcing
    cancels the coarse residual and the coarse correction is zero: one V-cycle changes W only at
    round-off.  The coarse KFVS residual of the restricted state is far from zero there (a forcing
    with the wrong sign would move W by about 2 dt_c Res_2h(W^0)/V)."""
    mesh, M, prm, S, h = ramp
    assert h[-1] < 1e-12 * h[0], "the steady state is not converged"
    W, G, a = S.state()
    S2 = orc.Solver(M, orc.params(**prm))
    S2.set_state(W, G, a)
    S2.run(1, multigrid=True)
    W2 = S2.state()[0]
    scale = np.abs(W).max(axis=1)[:, None]
    assert np.abs(W2 - W).max() / scale.max() < 1e-12
    # the quantity the forcing must cancel is not small
    L1 = S2.level(1)
    vol = M.cells()[0]
    W0 = np.zeros((5, L1["nc"]))
    np.add.at(W0.T, L1["map"], (W * vol).T)
    W0 /= L1["vol"]
    R0 = S2.kfvs_residual(1, W0)
    dtc = S2.level_dt(1, W0)
    assert (np.abs(R0) * dtc / L1["vol"]).max() / scale.max() > 1e-4


def test_vcycle_damps_a_smooth_perturbation_faster_than_the_single_grid(orc, ramp):
    """A smooth density perturbation of the steady state: after the same number of iterations the
    V-cycle has reduced the state error well below what single-grid steps reach (the coarse
    correction removes the smooth error that the explicit fine step damps slowly; with the wrong
    sign the correction would amplify it)."""
    mesh, M, prm, S, _ = ramp
    W, G, a = S.state()
    _, ctr, _ = M.cells()
    bump = 0.02 * np.exp(-((ctr[:, 0] - 0.3) ** 2 + (ctr[:, 1] - 0.25) ** 2) / 0.05)
    Wp = W.copy()
    Wp *= 1.0 + bump[None, :]
    errs = {}
    for mgrid in (False, True):
        T = orc.Solver(M, orc.params(**prm))
        T.set_state(Wp, G, a)
        T.run(30, multigrid=mgrid)
        errs[mgrid] = np.abs(T.state()[0] - W).max()
    e0 = np.abs(Wp - W).max()
    assert errs[True] < 0.5 * errs[False] < 0.5 * e0, (e0, errs)


@pytest.mark.parametrize("mk", [lambda: mg.periodic_box(6), lambda: mg.scale_box(12), lambda: mg.pyramid_box(6)],
                         ids=["jittered quadrant box", "jittered scale box", "pyramids"])
def test_coarsening_volumes_equal_the_solver_volumes(orc, mk):
    """The coarsening takes its own geometry of the fine level (node-mean centres, diagonal area
    vectors, divergence-theorem volumes), so that merges are decided on the same bits in the oracle
    and on the GPU.  Its volumes are the solver's Gauss-rule volumes to round-off on jittered mixed
    cells (both formulas are exact for the trilinear cells), so the restriction weights, the coarse
    volumes (sums of them) and the injected corrections conserve the solver's sum |Omega| W: the
    V-cycle conservation test with one global time step holds to 1e-14 for that reason."""
    M = orc.Mesh(mk())
    V = M.cells()[0]
    Vc = M.coarsening_geometry()[0]
    assert np.abs(V - Vc).max() <= 1e-14 * V.max()
    S = orc.Solver(M, orc.params(mach=0.3, n_levels=3))
    for lev in (1, 2):
        L, F = S.level(lev), S.level(lev - 1)
        agg = np.zeros(L["nc"])
        np.add.at(agg, L["map"], V if lev == 1 else F["vol"])
        assert np.abs(agg - L["vol"]).max() <= 1e-13 * L["vol"].max()


def test_coarse_time_step_from_grid_lines(orc):
    """The KFVS levels' local time step (reading 12 without the viscous term: dt_c = CFL |Omega_c| /
    sum_p A_p (|u . n_p| + c), A_p the summed area of the fine faces that make coarse face p and n_p
    the direction of their summed area vector) on a graded Cartesian box, worked out here from the
    grid lines and the coarse maps alone: a coarse face is the set of fine faces between the same two
    coarse cells, or of one coarse cell on boundary sides with the same tag (reading 10)."""
    xs = np.cumsum(np.r_[0.0, 0.10, 0.15, 0.12, 0.20, 0.18, 0.25])
    ys = np.cumsum(np.r_[0.0, 0.30, 0.20, 0.25, 0.15, 0.10])
    zs = np.cumsum(np.r_[0.0, 0.05, 0.08, 0.12, 0.30])
    bc = dict(xmin=4, xmax=5, ymin=1, ymax=1, zmin=2, zmax=3)
    mesh = mg.box_mesh(6, 5, 4, lambda i, j, k: np.zeros(np.shape(i), dtype=int), xs=xs, ys=ys, zs=zs, bc=bc)
    M = orc.Mesh(mesh)
    S = orc.Solver(M, orc.params(n_levels=3, cfl_coarse=0.9, mach=0.5))
    rho, u, p = 1.1, np.array([0.3, -0.2, 0.1]), 0.9
    c = np.sqrt(GAMMA * p / rho)
    # fine cells by grid index, from their node means
    lines = (xs, ys, zs)
    dims = (6, 5, 4)
    idx = {}
    for cell in range(len(mesh["cell_type"])):
        m = _cell_nodes(mesh, cell).mean(0)
        idx[tuple(int(np.searchsorted(lines[a], m[a])) - 1 for a in range(3))] = cell
    assert len(idx) == 120
    width = [np.diff(l) for l in lines]
    side_tag = {(0, -1): 4, (0, 1): 5, (1, -1): 1, (1, 1): 1, (2, -1): 2, (2, 1): 3}
    cmap = np.arange(120)
    for lev in (1, 2):
        L = S.level(lev)
        cmap = L["map"][cmap]  # fine cell -> cell of this level
        groups = {}  # (coarse cell, key) -> [summed area vector, summed area]
        for (i, j, k), a in idx.items():
            ijk = (i, j, k)
            for axis in range(3):
                area = np.prod([width[b][ijk[b]] for b in range(3) if b != axis])
                for sgn in (-1, 1):
                    nb = list(ijk)
                    nb[axis] += sgn
                    if 0 <= nb[axis] < dims[axis]:
                        B = cmap[idx[tuple(nb)]]
                        if B == cmap[a]:
                            continue
                        key = ("cell", int(B))
                    else:
                        key = ("tag", side_tag[(axis, sgn)])
                    g = groups.setdefault((int(cmap[a]), key), [np.zeros(3), 0.0])
                    g[0][axis] += sgn * area
                    g[1] += area
        vol = np.zeros(L["nc"])
        np.add.at(vol, cmap[[idx[t] for t in idx]], [np.prod([width[b][t[b]] for b in range(3)]) for t in idx])
        denom = np.zeros(L["nc"])
        for (A, _), (Sv, area) in groups.items():
            s = np.linalg.norm(Sv)
            denom[A] += area * ((abs(u @ Sv) / s if s > 0 else 0.0) + c)
        expected = 0.9 * vol / denom
        W = np.tile(_state(rho, u, p)[:, None], (1, L["nc"]))
        got = S.level_dt(lev, W)
        np.testing.assert_allclose(got, expected, rtol=1e-12, atol=0)
        assert L["nc"] < 120 and len(groups) > L["nc"]  # cells really merged, faces really grouped
