"""Writes the oracle's steady states that the GPU steady-state tests and the benchmark compare with.

Calls only the CPU oracle (oracle/) on the seeded synthetic meshes of meshgen; nothing here comes
from the CUDA library.  Each case is iterated from the uniform free stream by the oracle's own
single-grid steps or V-cycles (Sec. 4.2 of the paper) until the density-residual norm has fallen by
`drop` relative to its first value, and stored as tests/golden/steady_<name>_<sg|vc>.npz with W [5][N],
alpha [N], the iteration count and the final drop.  The ramps have one steady state,
so their single-grid state serves every iteration; the boundary layer's nonlinear WENO weights admit
more than one near the leading-edge corner, so it is stored for both iterations and each is compared
with the same iteration of the library.

  python tests/golden/make_steady_states.py [name[:sg|:vc] ...]
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import meshgen as mg  # noqa: E402

VISCOUS = dict(mach=0.5, reynolds=1e4, prandtl=0.72, viscous=1)

# name: (mesh factory, physics, oracle iterations ("sg" single grid, "vc" V-cycle), drop, iteration limit)
CASES = {
    # Mach 3 over a 15-degree ramp: shock from the corner, compression factor active at the shock
    "ramp_32x16x2": (lambda: mg.ramp_box(32, 16, 2, n_prism=2), dict(mach=3.0), ("sg",), 1e-12, 20000),
    "ramp_64x32x8": (lambda: mg.ramp_box(64, 32, 8, n_prism=4), dict(mach=3.0), ("sg",), 1e-12, 20000),
    # laminar boundary layer with the extrapolation outflow, compression factor active
    "wall_12x2x12": (lambda: mg.wall_box(12, 2, 12, first=2e-3, ratio=1.3, outflow=mg.BC_SUPER_OUT), VISCOUS,
                     ("sg", "vc"), 1e-12, 60000),
}


def case_mesh(name):
    return CASES[name][0]()


def case_params(name):
    return dict(CASES[name][1], n_levels=3)


def path(name, it):
    return os.path.join(HERE, f"steady_{name}_{it}.npz")


def reference(name, it):
    """path of the stored oracle state that a library run of iteration `it` ("sg"/"vc") is compared
    with: the same iteration where it is stored, else the case's single-grid state"""
    its = CASES[name][2]
    return path(name, it if it in its else its[0])


def make(name, only=None, chunk=200):
    import oracle
    oracle.build()
    mk, phys, iterations, drop, limit = CASES[name]
    mesh = mk()
    M = oracle.Mesh(mesh)
    for itn in iterations:
        if only and itn != only:
            continue
        multigrid = itn == "vc"
        S = oracle.Solver(M, oracle.params(**case_params(name)))
        W, G = mg.uniform_state(M.nc, mach=phys["mach"])
        S.set_state(W, G)
        t0, it, r0, last = time.time(), 0, None, 1.0
        while it < limit:
            h = S.run(chunk, multigrid=multigrid)
            r0 = r0 if r0 is not None else h[0]
            it += chunk
            last = h[-1] / r0
            if last <= drop:
                break
        W, G, a = S.state()
        np.savez_compressed(path(name, itn), W=W, alpha=a, iters=it, drop=last, multigrid=multigrid)
        print(f"{name} {itn}: {M.nc} cells, {it} {'V-cycles' if multigrid else 'steps'}, drop {last:.2e}, "
              f"{time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    # arguments: case names, each optionally with ":sg" or ":vc" for one of its iterations
    for arg in sys.argv[1:] or list(CASES):
        n, _, it = arg.partition(":")
        make(n, it or None)
