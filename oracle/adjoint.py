"""Discrete adjoint of the oracle's steady CGKS problem, dense and by definition.

TEST INFRASTRUCTURE ONLY (like the rest of this package): the CUDA library never imports it.

The steady problem of the compact scheme (Sec. 2.4 and 4 of the paper) has the cell averages W
and the cell gradients G as unknowns, u = (W [5][N], G [15][N]).  At a steady state

    F(u, beta) = ( Res(W, G),  Gnew(W, G) - G ) = 0,

with Res the residual of the explicit update and Gnew the Gauss-Green gradient of the interface
states (compression factor off: the factor's non-smooth pressure-jump terms are outside the
linearisation).  For a functional J(u, beta) and parameters beta (free-stream Mach number, node
displacement modes), the discrete adjoint gives

    dJ/dbeta = dJ/dbeta|_u + lambda^T dF/dbeta|_u,     (dF/du)^T lambda = -(dJ/du)^T.

Here every piece is formed in the plainest way: dF/du as a dense matrix whose columns are central
differences of the oracle residual, lambda by a dense solve, and the parameter partials by central
differences of F and J at the frozen state u.  The functional is the wall force

    J = sum over wall faces (tags 1, 2) of p(W_L) S_y,

p the pressure of the wall cell's average and S the face's area vector, outward from that cell.
"""
from __future__ import annotations

import numpy as np

from . import Mesh, Solver, params

WALL_TAGS = (1, 2)


def wall_faces(om: Mesh):
    """(left cells, area vectors [n][3]) of the wall faces of an oracle mesh."""
    F = om.faces()
    sel = np.isin(F["tag"], WALL_TAGS) & (F["fR"] < 0)
    S = np.zeros((om.nf, 3))
    for k in range(4):
        S += np.where((F["ngp"] > k)[:, None], F["gA"][:, k], 0.0)
    return F["fL"][sel].astype(np.int64), S[sel]


def pressure(W, gamma):
    return (gamma - 1.0) * (W[4] - 0.5 * (W[1] ** 2 + W[2] ** 2 + W[3] ** 2) / W[0])


def wall_force(om: Mesh, W, gamma, comp=1):
    L, S = wall_faces(om)
    return float(np.sum(pressure(W[:, L], gamma) * S[:, comp]))


def wall_force_du(om: Mesh, W, gamma, comp=1):
    """dJ/du in the layout of u (W part from dp/dW; zero for G)."""
    L, S = wall_faces(om)
    w = W[:, L]
    u = w[1:4] / w[0]
    dp = (gamma - 1.0) * np.stack([0.5 * (u ** 2).sum(0), -u[0], -u[1], -u[2], np.ones(len(L))])
    g = np.zeros((20, W.shape[1]))
    np.add.at(g[:5].T, L, (dp * S[:, comp]).T)
    return g.ravel()


def steady_F(sol: Solver, W, G):
    """F(u) = (Res, Gnew - G), flattened in the layout of u."""
    sol.set_state(W, G, np.ones(W.shape[1]))
    r = sol.residual()
    return np.concatenate([r["res"].ravel(), (r["grad"] - G).ravel()])


def split(u, nc):
    return u[:5 * nc].reshape(5, nc), u[5 * nc:].reshape(15, nc)


def jacobian(sol: Solver, W, G, rel=1e-6):
    """Dense dF/du by central differences, step rel * max(1, |u_j|)."""
    nc = W.shape[1]
    u = np.concatenate([W.ravel(), G.ravel()])
    A = np.empty((u.size, u.size))
    for j in range(u.size):
        h = rel * max(1.0, abs(u[j]))
        up, um = u.copy(), u.copy()
        up[j] += h
        um[j] -= h
        A[:, j] = (steady_F(sol, *split(up, nc)) - steady_F(sol, *split(um, nc))) / (2.0 * h)
    return A


def solve_steady(mesh, prm: dict, W, G, tol=5e-14, chunk=100, max_steps=20000):
    """Single-grid CGKS from (W, G) until the density-residual norm is below tol (absolute: runs
    started near a steady state have no meaningful first residual); returns (W, G, steps)."""
    sol = Solver(Mesh(mesh), params(**dict(prm, n_levels=1)))
    sol.set_state(W, G, np.ones(W.shape[1]))
    steps = 0
    while steps < max_steps:
        h = sol.run(chunk)
        steps += chunk
        if h[-1] <= tol:
            break
    Ws, Gs, _ = sol.state()
    return Ws, Gs, steps


def adjoint_gradient(mesh, prm: dict, W, G, modes=(), h_mach=1e-6, h_mode=1e-6, comp=1, A=None):
    """dJ/dMach and dJ/d(mode amplitudes) at the steady state (W, G) of `mesh` with parameters prm
    (compression_factor 0).  Returns a dict with the gradients, lambda and the Jacobian."""
    prm = dict(prm, n_levels=1, compression_factor=0)
    gamma = prm.get("gamma", 1.4)
    om = Mesh(mesh)
    sol = Solver(om, params(**prm))
    if A is None:
        A = jacobian(sol, W, G)
    g = wall_force_du(om, W, gamma, comp)
    lam = np.linalg.solve(A.T, -g)
    # Mach: the flow state is frozen, the free stream (boundary states, viscosity) moves
    M = prm["mach"]
    Fp = steady_F(Solver(om, params(**dict(prm, mach=M + h_mach))), W, G)
    Fm = steady_F(Solver(om, params(**dict(prm, mach=M - h_mach))), W, G)
    d_mach = float(lam @ ((Fp - Fm) / (2.0 * h_mach)))
    d_modes = []
    for field in modes:
        vals = []
        for s in (1.0, -1.0):
            m2 = Mesh(_displace(mesh, field, s * h_mode))
            vals.append((steady_F(Solver(m2, params(**prm)), W, G), wall_force(m2, W, gamma, comp)))
        dF = (vals[0][0] - vals[1][0]) / (2.0 * h_mode)
        dJ = (vals[0][1] - vals[1][1]) / (2.0 * h_mode)
        d_modes.append(dJ + float(lam @ dF))
    return dict(dJ_dmach=d_mach, dJ_dmodes=np.array(d_modes), lam=lam, dJdu=g, A=A)


def _displace(mesh, field, eps):
    out = dict(mesh)
    out["xyz"] = np.ascontiguousarray(mesh["xyz"] + eps * field)
    return out


def fd_gradient(mesh, prm: dict, W, G, field=None, h=1e-6, comp=1, tol=5e-14):
    """Central difference of the converged J in the Mach number (field None) or in one mode
    amplitude: two steady solves started from (W, G)."""
    prm = dict(prm, n_levels=1, compression_factor=0)
    gamma = prm.get("gamma", 1.4)
    J = []
    for s in (1.0, -1.0):
        if field is None:
            m, p = mesh, dict(prm, mach=prm["mach"] + s * h)
        else:
            m, p = _displace(mesh, field, s * h), prm
        Ws, _, _ = solve_steady(m, p, W, G, tol=tol)
        J.append(wall_force(Mesh(m), Ws, gamma, comp))
    return (J[0] - J[1]) / (2.0 * h)
