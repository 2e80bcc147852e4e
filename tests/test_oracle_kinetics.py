"""Pins of the oracle's gas-kinetic solver (Sec. 2.1, 2.3 of the paper) against quadrature and
closed forms that do not use the oracle's own moment code."""
import warnings

import numpy as np
import pytest
from scipy import integrate, special

from closed_forms import (dWdt_euler, euler_flux, euler_jacobian, gauss_hermite_maxwellian, half_space_rule,
                          heat_functional, ns_flux, psi)

INF = np.inf
warnings.filterwarnings("ignore", category=integrate.IntegrationWarning)


@pytest.mark.parametrize("U,lam", [(0.3, 0.7), (-1.2, 2.5), (0.0, 1.0), (2.0, 0.3), (-0.05, 40.0)])
def test_gaussian_moments_vs_quadrature(orc, U, lam):
    """<u^n> full and half space (u > 0, u < 0) against adaptive quadrature of u^n g(u)."""
    for space, (lo, hi) in ((0, (-INF, INF)), (1, (0.0, INF)), (-1, (-INF, 0.0))):
        m = orc.moments(1.0, U, 0.4, -0.2, lam, 2.0, space)
        for n in range(9):
            def f(u):
                return u ** n * np.sqrt(lam / np.pi) * np.exp(-lam * (u - U) ** 2)
            pts = sorted(set([lo, hi, U]) - {INF, -INF}) if space else [U]
            edges = [lo] + [p for p in pts if lo < p < hi] + [hi]
            val = sum(integrate.quad(f, a, b, epsabs=1e-15, epsrel=1e-14, limit=400)[0] for a, b in zip(edges[:-1], edges[1:]))
            scale = integrate.quad(lambda u: abs(f(u)), -INF, INF, epsabs=1e-15, limit=400)[0]
            assert abs(m["u"][n] - val) <= 1e-12 * max(scale, 1e-300), (space, n)
        # tangential moments are full-space Gaussians with mean V = 0.4, W = -0.2
        for key, mean in (("v", 0.4), ("w", -0.2)):
            for n in range(7):
                val = integrate.quad(lambda u: u ** n * np.sqrt(lam / np.pi) * np.exp(-lam * (u - mean) ** 2),
                                     -INF, INF, epsabs=1e-15, epsrel=1e-14)[0]
                assert abs(m[key][n] - val) <= 1e-12 * max(1.0, abs(val))


@pytest.mark.parametrize("K", [2, 3, 4])
def test_internal_moments_vs_radial_quadrature(orc, K):
    """<|xi|^2>, <|xi|^4> of the K-dimensional Gaussian exp(-lam xi^2) by radial quadrature."""
    lam = 0.83
    area = 2.0 * np.pi ** (K / 2.0) / special.gamma(K / 2.0)
    m = orc.moments(1.0, 0.0, 0.0, 0.0, lam, float(K), 0)
    for d in (1, 2):
        val = integrate.quad(lambda r: r ** (2 * d) * (lam / np.pi) ** (K / 2.0) * np.exp(-lam * r * r) * area * r ** (K - 1),
                             0.0, INF, epsabs=1e-15, epsrel=1e-14)[0]
        assert abs(m["xi"][d] - val) <= 1e-12 * val


@pytest.mark.parametrize("K", [2, 4])
def test_micro_slope_reproduces_its_moments(orc, K):
    """Eq. co: the slope s solves <s psi> = dW; checked by a (3+K)-dimensional Gauss-Hermite rule."""
    rng = np.random.default_rng(7 + K)
    rho, U, lam = 1.3, np.array([0.4, -0.3, 0.2]), 0.8
    coords, w = gauss_hermite_maxwellian(rho, U, lam, K, npts=6)
    P = psi(coords, K)
    for _ in range(3):
        dW = rng.normal(size=5)
        s = orc.slope(rho, *U, lam, float(K), dW)
        got = (P * (s @ P)) @ w
        np.testing.assert_allclose(got, dW, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("dt,tau,tn", [(0.1, 0.001, 0.002), (1e-3, 1e-3, 1e-3), (0.5, 0.0, 0.005),
                                       (2e-5, 7e-5, 7.5e-5), (1.0, 0.3, 0.3)])
def test_time_integrals_vs_quadrature(orc, dt, tau, tn):
    """Integrals over [0, dt] of the time coefficients of Eq. 2nd-flux."""
    q = orc.time_integrals(dt, tau, tn)
    fs = [lambda t: 1 - np.exp(-t / tn), lambda t: (t + tau) * np.exp(-t / tn) - tau,
          lambda t: t - tau + tau * np.exp(-t / tn), lambda t: np.exp(-t / tn), lambda t: (tau + t) * np.exp(-t / tn)]
    for k, f in enumerate(fs):
        val = integrate.quad(f, 0.0, dt, epsabs=0.0, epsrel=1e-13, limit=400)[0]
        scale = integrate.quad(lambda t: abs(f(t)), 0.0, dt, epsabs=0.0, epsrel=1e-13, limit=400)[0]
        assert abs(q[k] - val) <= 1e-11 * scale, k


def _unit(v):
    v = np.asarray(v, float)
    return v / np.linalg.norm(v)


def test_frame_is_orthonormal_right_handed(orc):
    rng = np.random.default_rng(3)
    for n in [rng.normal(size=3) for _ in range(20)] + [[0, 0, 1.0], [0, 0, -1.0], [1.0, 0, 0]]:
        n = _unit(n)
        t1, t2 = orc.frame(n)
        E = np.stack([n, t1, t2])
        np.testing.assert_allclose(E @ E.T, np.eye(3), atol=1e-15)
        assert np.linalg.det(E) > 0


@pytest.mark.parametrize("viscous", [0, 1])
def test_uniform_state_gives_exact_euler_flux(orc, viscous):
    """f = g for a uniform state: the CGKS and KFVS fluxes equal the Euler flux, W(dt) = W."""
    prm = orc.params(mach=0.5, reynolds=100.0, viscous=viscous, prandtl=0.72)
    rng = np.random.default_rng(11)
    for _ in range(5):
        rho, u, p = 0.5 + rng.random(), rng.normal(size=3) * 0.7, 0.3 + rng.random()
        W = np.array([rho, *(rho * u), p / 0.4 + 0.5 * rho * u @ u])
        n = _unit(rng.normal(size=3))
        F, Wt = orc.gks_point(prm, W, np.zeros(15), W, np.zeros(15), n, 0.013)
        np.testing.assert_allclose(F, euler_flux(W, n, 1.4), rtol=1e-13, atol=1e-14)
        np.testing.assert_allclose(Wt, W, rtol=1e-14, atol=1e-14)
        np.testing.assert_allclose(orc.kfvs_point(prm, W, W, n), euler_flux(W, n, 1.4), rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("viscous,prandtl", [(0, 1.0), (1, 1.0), (1, 0.72)])
def test_smooth_state_chapman_enskog_limit(orc, viscous, prandtl):
    """With identical left/right states and gradients, Eq. 2nd-flux time-averaged over dt gives
    exactly F_Euler + F_NS(mu = tau p) + (dt/2) dF_Euler/dt, and W(dt) = W + dt dW/dt (Euler);
    for Pr != 1 the energy flux adds (1/Pr - 1) x the heat flux of the non-equilibrium part."""
    gamma = 1.4
    prm = orc.params(mach=0.5, reynolds=300.0, viscous=viscous, prandtl=prandtl, eps_inviscid=0.01)
    rng = np.random.default_rng(21 + viscous)
    for _ in range(6):
        rho, u, p = 0.8 + 0.4 * rng.random(), rng.normal(size=3) * 0.5, 0.6 + 0.3 * rng.random()
        W = np.array([rho, *(rho * u), p / (gamma - 1) + 0.5 * rho * u @ u])
        G = rng.normal(size=15) * 0.3
        n = _unit(rng.normal(size=3))
        dt = 0.02
        F, Wt = orc.gks_point(prm, W, G, W, G, n, dt)
        mu_eff = (prm.mach / prm.reynolds) if viscous else prm.eps_inviscid * dt * p
        dWdt = dWdt_euler(W, G, gamma)
        dFdt = euler_jacobian(W, n, gamma) @ dWdt
        Fns = ns_flux(W, G, n, gamma, mu_eff)
        expect = euler_flux(W, n, gamma) + Fns + 0.5 * dt * dFdt
        if viscous and prandtl != 1.0:
            expect[4] += (1.0 / prandtl - 1.0) * heat_functional(Fns + 0.5 * dt * dFdt, 0.5 * dt * dWdt, u, n)
        scale = np.abs(euler_flux(W, n, gamma)).max()
        np.testing.assert_allclose(F, expect, rtol=0, atol=2e-13 * scale)
        np.testing.assert_allclose(Wt, W + dt * dWdt, rtol=0, atol=2e-13 * np.abs(W).max())


def test_flux_antisymmetry_and_rotation(orc):
    """Seen from the other side (n -> -n, L <-> R) the flux changes sign; rotating every vector
    rotates the momentum flux (frame independence of the local face frame)."""
    prm = orc.params(mach=0.5, reynolds=500.0, viscous=1, prandtl=0.72)
    rng = np.random.default_rng(5)

    def state():
        rho, u, p = 0.8 + 0.4 * rng.random(), rng.normal(size=3) * 0.5, 0.6 + 0.3 * rng.random()
        return np.array([rho, *(rho * u), p / 0.4 + 0.5 * rho * u @ u])

    for _ in range(4):
        WL, WR = state(), state()
        GL, GR = rng.normal(size=15) * 0.2, rng.normal(size=15) * 0.2
        n = _unit(rng.normal(size=3))
        F, Wt = orc.gks_point(prm, WL, GL, WR, GR, n, 0.01)
        F2, Wt2 = orc.gks_point(prm, WR, GR, WL, GL, -n, 0.01)
        np.testing.assert_allclose(F2, -F, rtol=0, atol=1e-13)
        np.testing.assert_allclose(Wt2, Wt, rtol=0, atol=1e-13)
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        if np.linalg.det(Q) < 0:
            Q[:, 0] *= -1

        def rotW(W):
            return np.array([W[0], *(Q @ W[1:4]), W[4]])

        def rotG(G):
            g = G.reshape(5, 3)
            out = np.zeros((5, 3))
            out[0] = Q @ g[0]
            out[4] = Q @ g[4]
            out[1:4] = Q @ g[1:4] @ Q.T
            return out.ravel()

        F3, Wt3 = orc.gks_point(prm, rotW(WL), rotG(GL), rotW(WR), rotG(GR), Q @ n, 0.01)
        np.testing.assert_allclose(F3, rotW(F), rtol=0, atol=1e-13)
        np.testing.assert_allclose(Wt3, rotW(Wt), rtol=0, atol=1e-13)


def test_kfvs_half_space_fluxes_vs_brute_force(orc):
    """KFVS (the coarse-level flux): int_{u>0} u psi g^l + int_{u<0} u psi g^r by a product rule
    (Gauss-Legendre in the normal velocity, Gauss-Hermite in the others, K = 2)."""
    prm = orc.params()
    rng = np.random.default_rng(9)
    for _ in range(3):
        Ws, total = [], np.zeros(5)
        for sgn in (1, -1):
            rho, u, p = 0.7 + 0.6 * rng.random(), rng.normal(size=3) * 0.6, 0.5 + 0.5 * rng.random()
            Ws.append(np.array([rho, *(rho * u), p / 0.4 + 0.5 * rho * u @ u]))
            coords, w = half_space_rule(rho, u, rho / (2 * p), 2, sgn)
            total += (psi(coords, 2) * coords[0]) @ w
        F = orc.kfvs_point(prm, Ws[0], Ws[1], np.array([1.0, 0.0, 0.0]))
        np.testing.assert_allclose(F, total, rtol=1e-11, atol=1e-13)


def test_slip_wall_ghost_blocks_mass_and_energy_flux(orc):
    """The mirrored slip-wall ghost makes the KFVS mass, tangential momentum and energy fluxes
    through the wall vanish; a farfield ghost of a free-stream interior is the free stream."""
    prm = orc.params(mach=0.5)
    rng = np.random.default_rng(2)
    for _ in range(4):
        rho, u, p = 0.8 + 0.4 * rng.random(), rng.normal(size=3) * 0.4, 0.6 + 0.3 * rng.random()
        W = np.array([rho, *(rho * u), p / 0.4 + 0.5 * rho * u @ u])
        n = _unit(rng.normal(size=3))
        Wg, _ = orc.bc_ghost(prm, 1, n, W, np.zeros(15))
        F = orc.kfvs_point(prm, W, Wg, n)
        assert abs(F[0]) < 1e-14 and abs(F[4]) < 1e-14
        tang = F[1:4] - (F[1:4] @ n) * n
        assert np.abs(tang).max() < 1e-14
    Winf = np.array([1.0, 0.5, 0.0, 0.0, 1.0 / 1.4 / 0.4 + 0.5 * 0.25])
    for n in ([1.0, 0, 0], [-1.0, 0, 0], [0, 0, 1.0]):
        Wg, Gg = orc.bc_ghost(prm, 3, np.array(n), Winf, np.ones(15))
        np.testing.assert_allclose(Wg, Winf, rtol=1e-14, atol=1e-15)
        assert not Gg.any()


def test_mirrored_ghost_gradient_is_gradient_of_mirrored_field(orc):
    """Ghost gradients (slip and no-slip walls) equal the gradient of the mirrored linear field
    x -> M W(Refl x), computed by finite differences."""
    prm = orc.params()
    rng = np.random.default_rng(4)
    n = _unit(rng.normal(size=3))
    R = np.eye(3) - 2 * np.outer(n, n)
    W0, G = np.array([1.1, 0.2, -0.1, 0.3, 2.6]), rng.normal(size=15)
    Gm = G.reshape(5, 3)

    def field(x):
        return W0 + Gm @ x

    for tag in (1, 2):
        def ghost_field(x):
            Wg, _ = orc.bc_ghost(prm, tag, n, field(R @ x), np.zeros(15))
            return Wg
        _, Gg = orc.bc_ghost(prm, tag, n, W0, G)
        h = 1e-6
        fd = np.stack([(ghost_field(h * e) - ghost_field(-h * e)) / (2 * h) for e in np.eye(3)], axis=1)
        np.testing.assert_allclose(Gg.reshape(5, 3), fd, atol=1e-8)


def test_compression_factor_special_cases(orc):
    """alpha = 1/(1 + A^2) (Sec. 3.3): equal states give 1; a pure pressure jump p_l = 2 p_r at rest
    gives A = 1/2 + 1 and alpha = 1/(1 + 9/4)."""
    prm = orc.params()
    W = np.array([1.0, 0.1, 0.0, 0.0, 2.5])
    assert orc.cf_alpha(prm, W, W, np.array([1.0, 0, 0])) == 1.0
    WL = np.array([1.0, 0.0, 0.0, 0.0, 2.0 / 0.4])
    WR = np.array([1.0, 0.0, 0.0, 0.0, 1.0 / 0.4])
    assert abs(orc.cf_alpha(prm, WL, WR, np.array([0.0, 1.0, 0])) - 1.0 / (1.0 + 2.25)) < 1e-15


def _sutherland(t, s):
    """Sutherland's law mu(T)/mu(T_inf) written out: t^(3/2) (1 + s) / (t + s)."""
    return t ** 1.5 * (1.0 + s) / (t + s)


def test_sutherland_viscosity_enters_as_mu_of_the_interface_temperature(orc):
    """With Sutherland's law (s = 110.4 K / 288.15 K) the gas-kinetic flux of a smooth state at
    temperature ratio t equals the constant-viscosity flux with mu = mu_inf x the law at t (the
    interface equilibrium of a state without jumps has that temperature), and differs from the
    constant-mu_inf flux; at t = 1 the law returns mu_inf."""
    g, mach, re, s = 1.4, 0.5, 200.0, 110.4 / 288.15
    rho, p = 0.9, 1.3 / 1.4
    t = g * p / rho
    u = np.array([0.4, 0.1, -0.05])
    W = np.array([rho, *(rho * u), p / (g - 1) + 0.5 * rho * u @ u])
    G = 0.05 * np.sin(np.arange(15) + 1.0)
    n = np.array([0.6, 0.8, 0.0])
    base = dict(gamma=g, mach=mach, viscous=1, prandtl=0.72)
    Fs, Ws = orc.gks_point(orc.params(reynolds=re, sutherland=s, **base), W, G, W, G, n, 1e-3)
    Fe, We = orc.gks_point(orc.params(reynolds=re / _sutherland(t, s), **base), W, G, W, G, n, 1e-3)
    F0, _ = orc.gks_point(orc.params(reynolds=re, **base), W, G, W, G, n, 1e-3)
    np.testing.assert_allclose(Fs, Fe, rtol=1e-12, atol=1e-15)
    assert np.abs(Fs - F0).max() > 1e-6 * np.abs(F0).max()
    assert _sutherland(1.0, s) == 1.0


def test_moment_terms_with_slopes_vs_brute_force(orc):
    """The building block of every moment of the gas-kinetic flux, int u^a v^b w^c (s . psi) psi g
    over the half spaces u > 0, u < 0 and the full space, for random Maxwellians and slopes s,
    against product-rule quadrature (Gauss-Legendre in u, Gauss-Hermite elsewhere, K = 2).  This
    pins, among others, the kinetic-weighted interface gradient sum_sides int_{side} psi (a . psi)
    g_side and the interface state sum_sides int_{side} psi g_side."""
    rng = np.random.default_rng(21)
    K = 2
    for _ in range(3):
        rho, lam = 0.6 + 0.8 * rng.random(), 0.4 + 1.5 * rng.random()
        U = rng.normal(size=3) * 0.8
        s = rng.normal(size=5)
        for space in (1, -1, 0):
            if space:
                coords, w = half_space_rule(rho, U, lam, K, space)
            else:
                coords, w = gauss_hermite_maxwellian(rho, U, lam, K, npts=8)
            ps = psi(coords, K)
            sp = s @ ps
            for ku, kv, kw in ((0, 0, 0), (1, 0, 0), (2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 1, 0)):
                mono = coords[0] ** ku * coords[1] ** kv * coords[2] ** kw
                for a in range(5):
                    ref = float((mono * sp * ps[a]) @ w)
                    scale = float((np.abs(mono * sp * ps[a])) @ w)
                    got = orc.mom_term(rho, *U, lam, K, space, ku, kv, kw, s, a)
                    assert abs(got - ref) <= 1e-11 * scale, (space, ku, kv, kw, a, got, ref)
                    ref0 = float((mono * ps[a]) @ w)
                    got0 = orc.mom_term(rho, *U, lam, K, space, ku, kv, kw, None, a)
                    assert abs(got0 - ref0) <= 1e-11 * float(np.abs(mono * ps[a]) @ w)
