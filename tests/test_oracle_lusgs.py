"""Pins of the oracle's implicit coarse smoother (Sec. 4.3: backward Euler linearised with the
Lax-Friedrichs Jacobian splitting, relaxed by one symmetric Gauss-Seidel sweep, "LU-SGS").

For a small defect the increments satisfy (D + L) D^-1 (D + U) dU = defect, with D the diagonal
|Omega_i|/dt_i + 1/2 sum_p lambda_p S_p and L / U the parts of the off-diagonal operator
1/2 (A_j(n) - lambda I) S that couple a cell to neighbours before / after it in the sweep order.
The test assembles that matrix from an independent Euler-flux Jacobian (central differences of the
flux written out here) and solves it densely."""
import numpy as np
import pytest

import meshgen as mg

GAMMA = 1.4


def euler_flux_n(W, n):
    rho = W[0]
    u = W[1:4] / rho
    p = (GAMMA - 1.0) * (W[4] - 0.5 * rho * u @ u)
    un = u @ n
    return np.concatenate([[rho * un], W[1:4] * un + p * n, [(W[4] + p) * un]])


def jacobian(W, n, h=1e-6):
    J = np.zeros((5, 5))
    for k in range(5):
        e = np.zeros(5)
        e[k] = h * max(abs(W[k]), 1.0)
        J[:, k] = (euler_flux_n(W + e, n) - euler_flux_n(W - e, n)) / (2 * e[k])
    return J


def wave_speed(W, n):
    rho = W[0]
    u = W[1:4] / rho
    p = (GAMMA - 1.0) * (W[4] - 0.5 * rho * u @ u)
    return abs(u @ n) + np.sqrt(GAMMA * p / rho)


def _setup(orc, mesh, lev, seed=4):
    M = orc.Mesh(mesh)
    S = orc.Solver(M, orc.params(n_levels=3, mach=0.5, coarse_smoother=1))
    L = S.level(lev)
    n = L["nc"]
    rng = np.random.default_rng(seed)
    W, _ = mg.uniform_state(n, mach=0.5)
    W = W * (1 + 0.05 * rng.standard_normal(W.shape))
    dt = S.level_dt(lev, W)
    return S, L, W, dt, rng


@pytest.mark.parametrize("mk,lev", [(lambda: mg.periodic_box(6), 2), (lambda: mg.wall_box(10, 6, 8, n_prism=3), 2)])
def test_colouring_is_proper_and_complete(orc, mk, lev):
    S, L, W, dt, _ = _setup(orc, mk(), lev)
    col, k = S.colors(lev)
    assert col.min() == 0 and col.max() == k - 1
    inner = (L["fR"] >= 0) & (L["fL"] != L["fR"])
    assert not np.any(col[L["fL"][inner]] == col[L["fR"][inner]])


@pytest.mark.parametrize("mk,lev", [(lambda: mg.periodic_box(6), 2), (lambda: mg.wall_box(10, 6, 8, n_prism=3), 2)])
def test_small_defect_solves_the_factored_system(orc, mk, lev):
    S, L, W, dt, rng = _setup(orc, mk(), lev)
    n = L["nc"]
    col, _ = S.colors(lev)
    eps = 1e-7
    rhs = eps * rng.standard_normal((5, n)) * np.abs(W).max(axis=1, keepdims=True) * L["vol"] / dt
    Wn, skipped = S.lusgs(lev, W, rhs, dt)
    assert skipped == 0
    dU = Wn - W
    # assemble D, L, U in the cell-major layout [n][5]
    Snorm = np.linalg.norm(L["Sn"], axis=1)
    D = L["vol"] / dt
    Lo = np.zeros((5 * n, 5 * n))
    Up = np.zeros((5 * n, 5 * n))
    for f in range(len(Snorm)):
        a, b = L["fL"][f], L["fR"][f]
        if Snorm[f] == 0.0 or a == b:
            continue
        nf = L["Sn"][f] / Snorm[f]
        lam = wave_speed(W[:, a], nf) if b < 0 else max(wave_speed(W[:, a], nf), wave_speed(W[:, b], nf))
        D[a] += 0.5 * lam * Snorm[f]
        if b < 0:
            continue
        D[b] += 0.5 * lam * Snorm[f]
        for i, j, sg in ((a, b, 1.0), (b, a, -1.0)):
            blk = 0.5 * (jacobian(W[:, j], sg * nf) - lam * np.eye(5)) * Snorm[f]
            tgt = Lo if col[j] < col[i] else Up
            tgt[5 * i:5 * i + 5, 5 * j:5 * j + 5] += blk
    Dm = np.kron(np.diag(D), np.eye(5))
    A = (Dm + Lo) @ np.linalg.inv(Dm) @ (Dm + Up)
    ref = np.linalg.solve(A, rhs.T.reshape(-1)).reshape(n, 5).T
    err = np.abs(dU - ref).max() / np.abs(ref).max()
    assert err < 1e-6, err
    # and it is not the plain (Jacobi) diagonal step
    assert np.abs(dU - rhs / D).max() > 1e-3 * np.abs(ref).max()


def test_vanishing_time_step_is_the_explicit_step(orc):
    """dt -> 0: D -> |Omega|/dt dominates and dU -> dt/|Omega| x defect (forward Euler)."""
    S, L, W, dt, rng = _setup(orc, mg.periodic_box(6), 2)
    t = dt * 1e-8
    rhs = 1e-6 * L["vol"] / t * rng.standard_normal(W.shape)  # increments of about 1e-6
    Wn, _ = S.lusgs(2, W, rhs, t)
    fe = t / L["vol"] * rhs
    np.testing.assert_allclose(Wn - W, fe, rtol=1e-6, atol=1e-6 * np.abs(fe).max())


def test_free_stream_is_a_fixed_point(orc):
    M = orc.Mesh(mg.periodic_box(6))
    S = orc.Solver(M, orc.params(n_levels=3, mach=0.3, coarse_smoother=1))
    L = S.level(2)
    W, _ = mg.uniform_state(L["nc"], mach=0.3)
    Wn, _ = S.lusgs(2, W, np.zeros_like(W), S.level_dt(2, W))
    assert np.array_equal(Wn, W)
