"""Closed forms used to pin the oracle: the Euler flux and its Jacobians (complex-step), the
Chapman-Enskog Navier-Stokes flux of the BGK model, and brute-force quadrature of Maxwellian moments.
Nothing here calls the oracle."""
from __future__ import annotations

import numpy as np


def prim(W, gamma):
    rho = W[0]
    u = W[1:4] / rho
    p = (gamma - 1.0) * (W[4] - 0.5 * rho * (u @ u))
    return rho, u, p


def euler_flux(W, n, gamma):
    """F(W) . n for the conservative state W (works on complex arrays)."""
    rho = W[0]
    u = W[1:4] / rho
    p = (gamma - 1.0) * (W[4] - 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]))
    un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2]
    return np.array([rho * un, W[1] * un + p * n[0], W[2] * un + p * n[1], W[3] * un + p * n[2], (W[4] + p) * un])


def euler_jacobian(W, n, gamma):
    """dF.n/dW by complex-step differentiation (exact to round-off)."""
    J = np.zeros((5, 5))
    h = 1e-30
    for j in range(5):
        Wc = W.astype(complex)
        Wc[j] += 1j * h
        J[:, j] = euler_flux(Wc, n, gamma).imag / h
    return J


def dWdt_euler(W, G, gamma):
    """Euler time derivative -sum_d J_d dW/dx_d; G[3q+d] = dW_q/dx_d."""
    dW = np.zeros(5)
    for d in range(3):
        e = np.zeros(3)
        e[d] = 1.0
        dW -= euler_jacobian(W, e, gamma) @ G.reshape(5, 3)[:, d]
    return dW


def ns_flux(W, G, n, gamma, mu):
    """Chapman-Enskog (first order) viscous flux of the BGK model through n:
    sigma = mu (grad u + grad u^T) - mu 2/(K+3) (div u) I, q = -mu c_p grad(p/rho),
    c_p = (K+5)/2, K = (5 - 3 gamma)/(gamma - 1); returns (0, -sigma.n, -(sigma u).n + q.n)."""
    K = (5.0 - 3.0 * gamma) / (gamma - 1.0)
    rho, u, p = prim(W, gamma)
    g = G.reshape(5, 3)
    du = np.array([(g[1 + i] - u[i] * g[0]) / rho for i in range(3)])  # du[i][d] = d u_i / dx_d
    dp = (gamma - 1.0) * (g[4] - 0.5 * (u @ u) * g[0] - rho * (u @ du))
    dT = (dp - (p / rho) * g[0]) / rho
    div = np.trace(du)
    sigma = mu * (du + du.T) - mu * 2.0 / (K + 3.0) * div * np.eye(3)
    q = -mu * (K + 5.0) / 2.0 * dT
    sn = sigma @ n
    return np.array([0.0, -sn[0], -sn[1], -sn[2], -(u @ sn) + q @ n])


def heat_functional(F, W, Ubar, n):
    """Heat flux about the velocity Ubar through n of a distribution whose flux moments are F and
    whose state moments are W (both global frame)."""
    U2 = Ubar @ Ubar
    un = Ubar @ n
    return (F[4] - Ubar @ F[1:4] + 0.5 * U2 * F[0]) - un * (W[4] - Ubar @ W[1:4] + 0.5 * U2 * W[0])


def gauss_hermite_maxwellian(rho, U, lam, K, npts=8):
    """Nodes/weights integrating f(u, v, w, xi_1..xi_K) against the Maxwellian of density rho,
    velocity U (3), lam = rho/(2p) with K internal degrees (K integer)."""
    x, w = np.polynomial.hermite.hermgauss(npts)
    s = 1.0 / np.sqrt(lam)
    dims = 3 + K
    grids = np.meshgrid(*([x] * dims), indexing="ij")
    wts = np.prod(np.stack(np.meshgrid(*([w] * dims), indexing="ij")), axis=0)
    wts = wts / np.pi ** (dims / 2.0) * rho
    coords = [s * grids[d] + (U[d] if d < 3 else 0.0) for d in range(dims)]
    return [c.ravel() for c in coords], wts.ravel()


def psi(coords, K):
    u, v, w = coords[:3]
    xi2 = sum(c * c for c in coords[3:3 + K]) if K else np.zeros_like(u)
    return np.stack([np.ones_like(u), u, v, w, 0.5 * (u * u + v * v + w * w + xi2)])


def half_space_rule(rho, U, lam, K, sign, n_u=400, n_h=6):
    """Product rule for int_{sign*u > 0} (.) g dXi: Gauss-Legendre on the (truncated) half line in u,
    Gauss-Hermite in v, w and the K internal coordinates."""
    xg, wg = np.polynomial.legendre.leggauss(n_u)
    L = abs(U[0]) + 14.0 / np.sqrt(lam)
    a, b = (0.0, L) if sign > 0 else (-L, 0.0)
    un = 0.5 * (b - a) * xg + 0.5 * (b + a)
    wu = 0.5 * (b - a) * wg * np.sqrt(lam / np.pi) * np.exp(-lam * (un - U[0]) ** 2)
    hx, hw = np.polynomial.hermite.hermgauss(n_h)
    s = 1.0 / np.sqrt(lam)
    axes = [un] + [U[1] + s * hx, U[2] + s * hx] + [s * hx] * K
    wax = [wu] + [hw / np.sqrt(np.pi)] * (2 + K)
    grids = np.meshgrid(*axes, indexing="ij")
    wts = np.prod(np.stack(np.meshgrid(*wax, indexing="ij")), axis=0) * rho
    return [g.ravel() for g in grids], wts.ravel()
