"""Mixed precision (precision 1): the coarse levels smooth the correction W - W^0 with the FP32
linearised KFVS operator (defect correction); the fine level, the defect and its restriction, the
states and the correction stay FP64.

The fine FP64 CGKS residual alone decides the converged state; the coarse levels only change the
path to it.  And as the coarse defect Res* + J(W^0)(W - W^0) is linear in the correction, its FP32
error shrinks with the correction, so the V-cycle converges to 1e-10 like the FP64 one."""
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


def _flux_scale(lv, W, gamma=1.4):
    """[5][nc] sum over a cell's faces of |S| x (rho s, rho |u| s + p, .., (E + p) s) with
    s = |u| + c: a bound of the magnitude of the face fluxes that a KFVS residual sums."""
    rho = W[0]
    u = np.sqrt((W[1] ** 2 + W[2] ** 2 + W[3] ** 2)) / rho
    p = (gamma - 1.0) * (W[4] - 0.5 * rho * u * u)
    s = u + np.sqrt(gamma * p / rho)
    m = np.stack([rho * s, rho * u * s + p, rho * u * s + p, rho * u * s + p, (W[4] + p) * s])
    area = np.linalg.norm(lv["Sn"], axis=1)
    out = np.zeros_like(W)
    fL, fR = lv["fL"], lv["fR"]
    np.add.at(out, (slice(None), fL), area * m[:, fL])
    inner = fR >= 0
    np.add.at(out, (slice(None), fR[inner]), area[inner] * m[:, fR[inner]])
    return out


@pytest.mark.parametrize("mk,mach", [(lambda: mg.periodic_box(8), 0.6), (lambda: mg.wall_box(16, 8, 16, n_prism=6), 0.6),
                                     (lambda: mg.ramp_box(24, 12, 8, n_prism=3), 3.0)])
def test_fp32_kfvs_jvp(cg, orc, mk, mach):
    """J(W0) dW in FP32 forward mode against the central difference of the oracle's FP64 KFVS
    residual, (Res(W0 + h dW) - Res(W0 - h dW)) / 2h with h = 1e-4 (truncation ~h^2 = 1e-8 of the
    curvature terms, rounding ~1e-16/h).  The FP32 derivative of each face flux carries a few tens of
    2^-24 of the flux magnitude times |dW|/|W| (states and normals rounded on entry, expf, erfcf and
    powf of a few ulp), so the error bound is 1e-5 of that scale on every level, boundaries included
    (walls, Riemann farfield, supersonic in/outflow)."""
    mesh = mk()
    prm = dict(n_levels=3, mach=mach)
    ctx = cg.upload_mesh(mesh, cg.default_params(precision=1, **prm))
    om = orc.Mesh(mesh)
    os_ = orc.Solver(om, orc.params(**prm))
    rng = np.random.default_rng(5)
    h = 1e-4
    for lev in (0, 1, 2):
        n = ctx.level_info(lev)[0]
        W0, _ = mg.uniform_state(n, mach=mach)
        W0 = W0 * (1 + 0.03 * rng.standard_normal(W0.shape))
        # perturb every component, the momentum ones on the scale of the momentum vector
        sw = np.abs(W0).max(axis=1)
        sw[1:4] = sw[1:4].max()
        dW = 0.01 * sw[:, None] * rng.standard_normal(W0.shape)
        got = ctx.kfvs_jvp(lev, _t(W0), _t(dW)).cpu().numpy()
        ref = (os_.kfvs_residual(lev, W0 + h * dW) - os_.kfvs_residual(lev, W0 - h * dW)) / (2 * h)
        rel = (np.abs(dW) / sw[:, None]).max()
        e = assert_normwise(got, ref, 1e-5, f"KFVS JVP level {lev}", scale=_flux_scale(os_.level(lev), W0) * rel)
        assert e > 0.0
        # linear in dW, exactly zero at dW = 0
        z = ctx.kfvs_jvp(lev, _t(W0), _t(np.zeros_like(W0))).cpu().numpy()
        assert not z.any()


def test_mixed_vcycle_keeps_freestream(cg):
    """A uniform free stream is a fixed point of the fine residual (to round-off); the mixed V-cycle
    leaves it there: the coarse defect starts at the restricted fine defect and its linear part acts
    on a round-off-sized correction."""
    mesh = mg.periodic_box(8)
    W, G = mg.uniform_state(len(mesh["cell_type"]), mach=0.2)
    ctx = cg.upload_mesh(mesh, cg.default_params(mach=0.2, precision=1, n_levels=3))
    ctx.state_init(_t(W), _t(G))
    ctx.vcycle(3)
    Wg = ctx.state_get()[0].cpu().numpy()
    assert np.abs(Wg - W).max() <= 1e-14 * np.abs(W).max()


def _state_err(Wa, Wb):
    """max |Wa - Wb| relative to the largest |Wb| of each variable, the momentum components sharing
    the magnitude of the momentum vector (a component with no flow is zero up to round-off)."""
    sw = np.abs(Wb).max(axis=1)
    sw[1:4] = sw[1:4].max()
    return (np.abs(Wa - Wb).max(axis=1) / sw).max()


def _run(cg, mesh, W, G, n, precision, **prm):
    ctx = cg.upload_mesh(mesh, cg.default_params(n_levels=3, precision=precision, **prm))
    ctx.state_init(_t(W), _t(G))
    h = ctx.vcycle(n)
    out = [x.cpu().numpy() for x in ctx.state_get()]
    ctx.close()
    return h, out


@pytest.mark.parametrize("case", ["wave", "wall", "ramp"])
def test_mixed_vcycles_track_fp64(cg, case):
    """The linearised coarse equations differ from the FAS ones by terms quadratic in the coarse
    correction (plus FP32 rounding of its linear part), so a few mixed and FP64 V-cycles from the
    same start differ by a small fraction of the change they make to the state."""
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
    h64, (W64, G64, a64) = _run(cg, mesh, W, G, 5, 0, **prm)
    h32, (W32, G32, a32) = _run(cg, mesh, W, G, 5, 1, **prm)
    change = np.abs(W64 - W).max(axis=1)
    diff = np.abs(W32 - W64).max(axis=1)
    print(case, "diff/change", (diff / change.max()).max(), "hist", np.abs(h32 / h64 - 1).max())
    assert (diff <= 0.05 * change.max()).all(), (diff, change)
    assert not np.array_equal(W32, W64)  # the coarse levels really ran another operator
    np.testing.assert_allclose(h32[0], h64[0], rtol=1e-14)  # first norm precedes any coarse work


def test_mixed_steady_state_matches_oracle(cg, orc):
    """Small Mach 3 compression ramp driven to a 1e-10 residual drop by the mixed V-cycle on the
    GPU and by FP64 single-grid CGKS in the oracle: the steady states agree within 1e-7 relative
    (the difference left is the 1e-10 convergence tolerance times the solution's sensitivity)."""
    mesh = mg.ramp_box(16, 8, 2, n_prism=2)
    prm = dict(mach=3.0)
    n = len(mesh["cell_type"])
    W, G = mg.uniform_state(n, mach=3.0)
    om = orc.Mesh(mesh)
    os_ = orc.Solver(om, orc.params(n_levels=3, **prm))
    os_.set_state(W, G)
    r0 = None
    for _ in range(40):
        h = os_.run(100, multigrid=False)
        r0 = h[0] if r0 is None else r0
        if h[-1] / r0 < 1e-10:
            break
    assert h[-1] / r0 < 1e-10
    Wo = os_.state()[0]
    for precision in (1, 0):
        ctx = cg.upload_mesh(mesh, cg.default_params(n_levels=3, precision=precision, **prm))
        ctx.state_init(_t(W), _t(G))
        out = ctx.steady_solve(multigrid=True, drop=1e-10, max_iters=20000)
        assert out["converged"], out
        Wg = ctx.state_get()[0].cpu().numpy()
        err = _state_err(Wg, Wo)
        print("precision", precision, "V-cycles", out["iters"], "max relative state error", err)
        assert err <= 1e-7, (precision, err)
        ctx.close()
