"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module holds NO arithmetic of the method (no geometry, no fluxes, no
reconstruction): it only lays out nodes, cell connectivity, boundary-face node
lists with tags, periodic face pairs and pointwise initial fields.  Every mesh
is a structured n_x x n_y x n_z grid whose hexahedra are split by a conforming
rule into hexahedra, prisms and Kuhn tetrahedra (the mixed-element meshes of
Sec. 2.2 of the paper), optionally graded, sheared and jittered by a
counter-based generator (splitmix64, Steele/Lea/Flood 2014 as published by
Vigna) keyed by (seed, node id, axis).

Local node orderings (VTK-like) that the consumers rely on:
  tet   : 4 nodes, positively oriented (det[x1-x0, x2-x0, x3-x0] > 0)
  prism : 6 nodes, bottom triangle (0,1,2) counter-clockwise seen from the
          top triangle (3,4,5), node 3 above node 0
  hex   : 8 nodes, bottom quad (0,1,2,3) counter-clockwise seen from the top
          quad (4,5,6,7), node 4 above node 0

Boundary tags (the BC kind of each boundary face):
  1 slip wall, 2 no-slip adiabatic wall, 3 farfield (Riemann invariants),
  4 supersonic inflow (free stream), 5 supersonic outflow (extrapolation),
  >= 100 periodic side (paired through ``periodic_pairs``).
"""
from __future__ import annotations

import numpy as np

TET, PRISM, HEX, PYRAMID = 4, 5, 6, 7
BC_SLIP, BC_NOSLIP, BC_FARFIELD, BC_SUPER_IN, BC_SUPER_OUT = 1, 2, 3, 4, 5
PERIODIC_TAG0 = 100

_HEX, _PRZ, _PRX, _TET, _PYR = 0, 1, 2, 3, 4  # grid-cell split kinds


def splitmix64(x):
    """splitmix64 output function on uint64 arrays (counter-based)."""
    with np.errstate(over="ignore"):
        z = (np.asarray(x, dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15))
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def _uniform01(seed, key):
    """Uniform [0,1) doubles from (seed, integer key) via splitmix64."""
    with np.errstate(over="ignore"):
        z = splitmix64(np.uint64(seed) * np.uint64(0x100000001B3) ^ np.asarray(key, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _graded(n, first, ratio):
    k = np.arange(n + 1, dtype=np.float64)
    if ratio == 1.0:
        return first * k
    return first * (ratio ** k - 1.0) / (ratio - 1.0)


def box_mesh(nx, ny, nz, split, xs=None, ys=None, zs=None, periodic=(False, False, False),
             bc=None, jitter=0.0, seed=2402, jitter_mask=None, mapping=None):
    """Mixed-element mesh of a structured box.

    split(i, j, k) -> int array of grid-cell kinds (0 hex, 1 prism_z, 2 prism_x, 3 Kuhn tets,
    4 six pyramids on the faces of the cell with a new apex node at its node mean: all faces of the
    grid cell stay quadrilaterals, so pyramid cells border hexahedra or the boundary),
    evaluated on index arrays.  xs/ys/zs are the grid-line coordinates (default [0,1]).
    bc maps 'xmin','xmax','ymin','ymax','zmin','zmax' to a tag for non-periodic sides.
    jitter is the +-fraction of the local spacing applied per coordinate; boundary nodes
    of a non-periodic side keep that coordinate, periodic sides are jittered identically.
    jitter_mask(i, j, k) -> bool array, False disables jitter of that node.
    mapping(x, y, z) -> (x, y, z) is applied after jitter (e.g. a ramp shear).
    """
    xs = np.linspace(0.0, 1.0, nx + 1) if xs is None else np.asarray(xs, dtype=np.float64)
    ys = np.linspace(0.0, 1.0, ny + 1) if ys is None else np.asarray(ys, dtype=np.float64)
    zs = np.linspace(0.0, 1.0, nz + 1) if zs is None else np.asarray(zs, dtype=np.float64)
    assert len(xs) == nx + 1 and len(ys) == ny + 1 and len(zs) == nz + 1
    bc = dict(bc or {})
    dims = (nx, ny, nz)
    lines = (xs, ys, zs)

    # ---- nodes -------------------------------------------------------------------------------
    I, J, K = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    I, J, K = (a.transpose(2, 1, 0).ravel() for a in (I, J, K))  # node id = i + (nx+1)(j + (ny+1)k)
    idx = (I, J, K)
    xyz = np.stack([xs[I], ys[J], zs[K]], axis=1)
    if jitter > 0.0:
        wrapped = [np.where(p & (a == n), 0, a) if p else a for a, n, p in zip(idx, dims, periodic)]
        key = wrapped[0] + (nx + 1) * (wrapped[1] + (ny + 1) * wrapped[2])
        mask = np.ones(len(I), dtype=bool) if jitter_mask is None else np.asarray(jitter_mask(I, J, K))
        for ax in range(3):
            a, n, line, per = idx[ax], dims[ax], lines[ax], periodic[ax]
            d = np.diff(line)
            if per:
                left = np.concatenate([[d[-1]], d])
                right = np.concatenate([d, [d[0]]])
            else:
                left = np.concatenate([[d[0]], d])
                right = np.concatenate([d, [d[-1]]])
            h = np.minimum(left, right)[a]
            u = _uniform01(seed, key.astype(np.uint64) * np.uint64(3) + np.uint64(ax)) - 0.5
            move = mask.copy()
            if not per:
                move &= (a > 0) & (a < n)
            xyz[:, ax] += np.where(move, 2.0 * jitter * u * h, 0.0)
    if mapping is not None:
        x, y, z = mapping(xyz[:, 0].copy(), xyz[:, 1].copy(), xyz[:, 2].copy())
        xyz = np.stack([x, y, z], axis=1)

    def nid(i, j, k):
        return i + (nx + 1) * (j + (ny + 1) * k)

    # ---- cells -------------------------------------------------------------------------------
    gi, gj, gk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    gi, gj, gk = (a.transpose(2, 1, 0).ravel() for a in (gi, gj, gk))  # grid-cell order: i fastest
    kind = np.asarray(split(gi, gj, gk), dtype=np.int64)
    c = {}
    for a in (0, 1):
        for b in (0, 1):
            for cc in (0, 1):
                c[(a, b, cc)] = nid(gi + a, gj + b, gk + cc)
    nsub = np.array([1, 2, 2, 6, 6])[kind]
    sub_types = {_HEX: [HEX], _PRZ: [PRISM, PRISM], _PRX: [PRISM, PRISM], _TET: [TET] * 6, _PYR: [PYRAMID] * 6}
    blocks = {}
    blocks[_HEX] = [[c[0, 0, 0], c[1, 0, 0], c[1, 1, 0], c[0, 1, 0], c[0, 0, 1], c[1, 0, 1], c[1, 1, 1], c[0, 1, 1]]]
    blocks[_PRZ] = [[c[0, 0, 0], c[1, 0, 0], c[1, 1, 0], c[0, 0, 1], c[1, 0, 1], c[1, 1, 1]],
                    [c[0, 0, 0], c[1, 1, 0], c[0, 1, 0], c[0, 0, 1], c[1, 1, 1], c[0, 1, 1]]]
    blocks[_PRX] = [[c[0, 0, 0], c[0, 1, 0], c[0, 1, 1], c[1, 0, 0], c[1, 1, 0], c[1, 1, 1]],
                    [c[0, 0, 0], c[0, 1, 1], c[0, 0, 1], c[1, 0, 0], c[1, 1, 1], c[1, 0, 1]]]
    tets = []
    unit = {0: (1, 0, 0), 1: (0, 1, 0), 2: (0, 0, 1)}
    for perm in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
        p0 = (0, 0, 0)
        p1 = tuple(np.add(p0, unit[perm[0]]))
        p2 = tuple(np.add(p1, unit[perm[1]]))
        p3 = (1, 1, 1)
        sign = np.linalg.det(np.array([unit[perm[0]], unit[perm[1]], unit[perm[2]]], dtype=float))
        verts = [p0, p1, p2, p3] if sign > 0 else [p0, p2, p1, p3]
        tets.append([c[v] for v in verts])
    blocks[_TET] = tets
    # pyramids: apex nodes appended after the grid nodes, one per pyramid grid cell (node mean)
    pyr = np.nonzero(kind == _PYR)[0]
    apex = np.zeros(len(kind), dtype=np.int64)
    if len(pyr):
        corners = np.stack([c[v][pyr] for v in c], axis=1)  # [m][8]
        apex[pyr] = len(xyz) + np.arange(len(pyr))
        xyz = np.concatenate([xyz, xyz[corners].mean(axis=1)])
    hexv = [c[0, 0, 0], c[1, 0, 0], c[1, 1, 0], c[0, 1, 0], c[0, 0, 1], c[1, 0, 1], c[1, 1, 1], c[0, 1, 1]]
    # base = the grid cell's outward face reversed (counter-clockwise seen from the apex), then apex
    blocks[_PYR] = [[hexv[i] for i in f] + [apex] for f in ((1, 2, 3, 0), (7, 6, 5, 4), (4, 5, 1, 0),
                                                            (5, 6, 2, 1), (6, 7, 3, 2), (7, 4, 0, 3))]

    ncell = int(nsub.sum())
    cell_type = np.empty(ncell, dtype=np.int8)
    counts = np.empty(ncell, dtype=np.int64)
    first_cell = np.concatenate([[0], np.cumsum(nsub)[:-1]])
    for kd in (_HEX, _PRZ, _PRX, _TET, _PYR):
        sel = np.nonzero(kind == kd)[0]
        for s, t in enumerate(sub_types[kd]):
            cell_type[first_cell[sel] + s] = t
            counts[first_cell[sel] + s] = {TET: 4, PRISM: 6, HEX: 8, PYRAMID: 5}[t]
    cell_ptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    cell_nodes = np.empty(cell_ptr[-1], dtype=np.int32)
    for kd in (_HEX, _PRZ, _PRX, _TET, _PYR):
        sel = np.nonzero(kind == kd)[0]
        for s, nodes in enumerate(blocks[kd]):
            start = cell_ptr[first_cell[sel] + s]
            for q, arr in enumerate(nodes):
                cell_nodes[start + q] = arr[sel]

    # ---- boundary faces ----------------------------------------------------------------------
    tri_x = np.isin(kind, (_PRX, _TET))
    tri_y = kind == _TET
    tri_z = np.isin(kind, (_PRZ, _TET))
    kind3 = kind.reshape(nz, ny, nx)  # [k, j, i]
    bfaces = []  # (nodes list arrays, tag, side, position key)

    def side_faces(axis, lo):
        # grid faces on the side: returns list of (node arrays (m, nv), position index array, sub index)
        if axis == 0:
            i = 0 if lo else nx
            ci = 0 if lo else nx - 1
            jj, kk = np.meshgrid(np.arange(ny), np.arange(nz), indexing="ij")
            jj, kk = jj.T.ravel(), kk.T.ravel()
            tri = tri_x.reshape(nz, ny, nx)[kk, jj, ci]
            q = [nid(i, jj, kk), nid(i, jj + 1, kk), nid(i, jj + 1, kk + 1), nid(i, jj, kk + 1)]
            pos = jj + ny * kk
        elif axis == 1:
            j = 0 if lo else ny
            cj = 0 if lo else ny - 1
            ii, kk = np.meshgrid(np.arange(nx), np.arange(nz), indexing="ij")
            ii, kk = ii.T.ravel(), kk.T.ravel()
            tri = tri_y.reshape(nz, ny, nx)[kk, cj, ii]
            q = [nid(ii, j, kk), nid(ii + 1, j, kk), nid(ii + 1, j, kk + 1), nid(ii, j, kk + 1)]
            pos = ii + nx * kk
        else:
            k = 0 if lo else nz
            ck = 0 if lo else nz - 1
            ii, jj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
            ii, jj = ii.T.ravel(), jj.T.ravel()
            tri = tri_z.reshape(nz, ny, nx)[ck, jj, ii]
            q = [nid(ii, jj, k), nid(ii + 1, jj, k), nid(ii + 1, jj + 1, k), nid(ii, jj + 1, k)]
            pos = ii + nx * jj
        out = []
        quad = ~tri
        out.append((np.stack([a[quad] for a in q], axis=1), pos[quad], 0))
        out.append((np.stack([q[0][tri], q[1][tri], q[2][tri]], axis=1), pos[tri], 0))
        out.append((np.stack([q[0][tri], q[2][tri], q[3][tri]], axis=1), pos[tri], 1))
        return out, tri

    del kind3
    names = ("x", "y", "z")
    flist = []  # entries: (nodes(m,nv), tag, side_id, poskey)
    tri_by_side = {}
    for axis in range(3):
        for lo in (True, False):
            side = 2 * axis + (0 if lo else 1)
            faces, tri = side_faces(axis, lo)
            tri_by_side[side] = tri
            if periodic[axis]:
                tag = PERIODIC_TAG0 + side
            else:
                tag = bc.get(names[axis] + ("min" if lo else "max"))
                if tag is None:
                    raise ValueError(f"missing bc for side {names[axis]}{'min' if lo else 'max'}")
            for nodes, pos, sub in faces:
                if len(pos) == 0:
                    continue
                ntri = nodes.shape[1] == 3
                flist.append((nodes, tag, side, pos * 4 + sub * 2 + (1 if ntri else 0)))
    for axis in range(3):
        if periodic[axis] and not np.array_equal(tri_by_side[2 * axis], tri_by_side[2 * axis + 1]):
            raise ValueError(f"periodic axis {axis}: face splittings differ on the two sides")

    bnodes_list, btag_list, bcount_list, side_list, key_list = [], [], [], [], []
    for nodes, tag, side, key in flist:
        m, nv = nodes.shape
        bnodes_list.append(nodes.ravel())
        btag_list.append(np.full(m, tag, dtype=np.int32))
        bcount_list.append(np.full(m, nv, dtype=np.int64))
        side_list.append(np.full(m, side, dtype=np.int64))
        key_list.append(key)
    bface_nodes = np.concatenate(bnodes_list).astype(np.int32) if bnodes_list else np.zeros(0, np.int32)
    bface_tag = np.concatenate(btag_list) if btag_list else np.zeros(0, np.int32)
    bcount = np.concatenate(bcount_list) if bcount_list else np.zeros(0, np.int64)
    bface_ptr = np.concatenate([[0], np.cumsum(bcount)]).astype(np.int64)
    side_arr = np.concatenate(side_list) if side_list else np.zeros(0, np.int64)
    key_arr = np.concatenate(key_list) if key_list else np.zeros(0, np.int64)

    pairs = []
    for axis in range(3):
        if not periodic[axis]:
            continue
        lo_ids = np.nonzero(side_arr == 2 * axis)[0]
        hi_ids = np.nonzero(side_arr == 2 * axis + 1)[0]
        lo_sorted = lo_ids[np.argsort(key_arr[lo_ids], kind="stable")]
        hi_sorted = hi_ids[np.argsort(key_arr[hi_ids], kind="stable")]
        assert np.array_equal(key_arr[lo_sorted], key_arr[hi_sorted])
        pairs.append(np.stack([lo_sorted, hi_sorted], axis=1))
    periodic_pairs = (np.concatenate(pairs).astype(np.int32) if pairs else np.zeros((0, 2), np.int32))

    return dict(xyz=np.ascontiguousarray(xyz), cell_type=cell_type, cell_ptr=cell_ptr,
                cell_nodes=cell_nodes, bface_ptr=bface_ptr, bface_nodes=bface_nodes,
                bface_tag=bface_tag.astype(np.int32), periodic_pairs=np.ascontiguousarray(periodic_pairs),
                dims=(nx, ny, nz))


# ---- the workloads ---------------------------------------------------------------------------

def quadrant_split(a, b):
    """hex for i<a,k<b; prism_z for i>=a,k<b; prism_x for i<a,k>=b; Kuhn tets for i>=a,k>=b."""
    def split(i, j, k):
        return np.where(i < a, np.where(k < b, _HEX, _PRX), np.where(k < b, _PRZ, _TET))
    return split


def layered_split(n_prism, upper=_TET):
    """prism_z for k<n_prism, then `upper` (Kuhn tets by default) above."""
    def split(i, j, k):
        return np.where(k < n_prism, _PRZ, upper)
    return split


def periodic_box(n=16, jitter=0.05, seed=2402, split=None):
    """Periodic unit box, quadrant layout (a = b = 3n/4): the 16^3 density-wave workload
    (6,912 cells at n = 16) and its smaller/larger siblings."""
    a = (3 * n) // 4
    return box_mesh(n, n, n, split or quadrant_split(a, a), periodic=(True, True, True),
                    jitter=jitter, seed=seed)


def wall_layout(nx=96, nz=64, first=1e-4, ratio=1.1, tet_min=0.5, tet_max=2.0):
    """Wall-normal grid lines of the boundary-layer box and its number of prism layers: geometric
    growth from `first` by `ratio` until the spacing reaches tet_max * dx (then uniform), prism
    layers while the spacing is below tet_min * dx and Kuhn tetrahedra above, so that every
    tetrahedron is within tet_max : 1 and 1 : 1/tet_min of the in-plane spacing dx = 1/nx."""
    dx = 1.0 / nx
    z = _graded(nz, first, ratio)
    dz = np.diff(z)
    if (dz >= tet_max * dx).any():
        k = int(np.argmax(dz >= tet_max * dx))
        z = np.concatenate([z[:k + 1], z[k] + tet_max * dx * np.arange(1, nz - k + 1)])
        dz = np.diff(z)
    n_prism = int(np.argmax(dz >= tet_min * dx)) if (dz >= tet_min * dx).any() else nz
    return z, n_prism


def wall_box(nx=96, ny=64, nz=64, n_prism=None, first=1e-4, ratio=1.1, jitter=0.0, seed=2402, outflow=BC_FARFIELD):
    """Laminar boundary-layer box: x in [0,1], y periodic with dy = dx, z from a no-slip wall
    (first spacing `first`, growth `ratio`, capped at twice dx), prism_z layers at the wall and
    Kuhn tets above (wall_layout; n_prism overrides the count), farfield on x-in and top, and on x-out
    the kind `outflow` (farfield, or BC_SUPER_OUT: the extrapolation outflow).
    96x64x64 -> 42 prism layers, height 0.374, 1,327,104 cells."""
    xs = np.linspace(0.0, 1.0, nx + 1)
    ys = np.arange(ny + 1) * (1.0 / nx)
    zs, npz = wall_layout(nx, nz, first, ratio)
    n_prism = npz if n_prism is None else n_prism
    return box_mesh(nx, ny, nz, layered_split(n_prism), xs=xs, ys=ys, zs=zs,
                    periodic=(False, True, False),
                    bc=dict(xmin=BC_FARFIELD, xmax=outflow, zmin=BC_NOSLIP, zmax=BC_FARFIELD),
                    jitter=jitter, seed=seed,
                    jitter_mask=(lambda i, j, k: k > n_prism) if jitter > 0 else None)


def pyramid_box(n=6, jitter=0.05, seed=2402, periodic=True):
    """Box of hexahedra with a central block of pyramid-split cells (six pyramids per grid cell around
    a node-mean apex); periodic, or farfield on every side."""
    lo, hi = n // 3, n - n // 3

    def split(i, j, k):
        inside = (i >= lo) & (i < hi) & (j >= lo) & (j < hi) & (k >= lo) & (k < hi)
        return np.where(inside, _PYR, _HEX)
    bc = None if periodic else {k: BC_FARFIELD for k in ("xmin", "xmax", "ymin", "ymax", "zmin", "zmax")}
    return box_mesh(n, n, n, split, periodic=(periodic,) * 3, bc=bc, jitter=jitter, seed=seed)


def prism_slab(nx=32, ny=4, nz=24, first=1e-3, ratio=1.2, periodic=False):
    """All-prism boundary-layer slab: x in [0,1], y periodic with dy = dx, z graded from the wall
    (no-slip, farfield elsewhere) or periodic in every direction.  At 32x4x24 its level-2
    agglomerates include one wrapping around its neighbour (a coarse face of zero net area)."""
    z = _graded(nz, first, ratio)
    bc = None if periodic else dict(xmin=BC_FARFIELD, xmax=BC_FARFIELD, zmin=BC_NOSLIP, zmax=BC_FARFIELD)
    return box_mesh(nx, ny, nz, layered_split(nz), xs=np.linspace(0.0, 1.0, nx + 1), ys=np.arange(ny + 1) / nx,
                    zs=z, periodic=(True, True, True) if periodic else (False, True, False), bc=bc)


def ramp_box(nx=256, ny=128, nz=128, n_prism=8, angle_deg=15.0, jitter=0.0, seed=2402):
    """Compression ramp: x in [-0.5, 1.5], wall y = 0 for x < 0 and y = x tan(angle) after,
    pure vertical shear y = eta + y_wall(x) (height 1), z periodic with dz = dx;
    n_prism prism_z layers at the wall and hexahedra above.  Supersonic inflow at x-in,
    extrapolation at x-out and top, slip wall at the bottom.  256x128x128 -> 4,456,448 cells."""
    xs = np.linspace(-0.5, 1.5, nx + 1)
    ys = np.linspace(0.0, 1.0, ny + 1)
    zs = np.arange(nz + 1) * (2.0 / nx)
    t = np.tan(np.radians(angle_deg))

    def mapping(x, y, z):
        return x, y + np.where(x > 0.0, x * t, 0.0), z

    def split(i, j, k):
        return np.where(j < n_prism, _PRZ, _HEX)
    return box_mesh(nx, ny, nz, split, xs=xs, ys=ys, zs=zs, periodic=(False, False, True),
                    bc=dict(xmin=BC_SUPER_IN, xmax=BC_SUPER_OUT, ymin=BC_SLIP, ymax=BC_SUPER_OUT),
                    jitter=jitter, seed=seed, mapping=mapping)


def scale_box(n, jitter=0.05, seed=2402):
    """Quadrant layout (a = b = 3n/4) on n^3 with the boundary-layer box's boundaries
    (no-slip wall at z = 0, farfield elsewhere, y periodic); jitter away from the wall layer.
    n = 84 / 144 / 228 -> 1,000,188 / 5,038,848 / 20,000,844 cells."""
    a = (3 * n) // 4
    return box_mesh(n, n, n, quadrant_split(a, a), periodic=(False, True, False),
                    bc=dict(xmin=BC_FARFIELD, xmax=BC_FARFIELD, zmin=BC_NOSLIP, zmax=BC_FARFIELD),
                    jitter=jitter, seed=seed, jitter_mask=lambda i, j, k: k > 1)


# ---- initial fields (pointwise, at vertex averages; no cell geometry) -------------------------

def vertex_centers(mesh):
    ptr = mesh["cell_ptr"]
    counts = np.diff(ptr)
    xyz = mesh["xyz"][mesh["cell_nodes"]]
    owner = np.repeat(np.arange(len(counts)), counts)
    out = np.zeros((len(counts), 3))
    np.add.at(out, owner, xyz)
    return out / counts[:, None]


def freestream_velocity(mach, aoa=(0.0, 0.0)):
    a, b = np.radians(aoa[0]), np.radians(aoa[1])
    return mach * np.array([np.cos(a) * np.cos(b), np.sin(b), np.sin(a) * np.cos(b)])


def uniform_state(n_cells, gamma=1.4, mach=0.2, aoa=(0.0, 0.0)):
    """Free stream rho = 1, p = 1/gamma (unit sound speed), velocity mach along aoa:
    W [5][N] conservative, gradW [15][N] zero (row 3*q + d is d/dx_d of component q)."""
    u = freestream_velocity(mach, aoa)
    rho, p = 1.0, 1.0 / gamma
    w = np.array([rho, rho * u[0], rho * u[1], rho * u[2], p / (gamma - 1.0) + 0.5 * rho * u @ u])
    W = np.repeat(w[:, None], n_cells, axis=1)
    return np.ascontiguousarray(W), np.zeros((15, n_cells))


def density_wave_state(mesh, gamma=1.4, mach=0.2, amp=0.01):
    """rho = 1 + amp sin(2 pi (x+y+z)), p = 1/gamma, u = (mach, 0, 0) sampled at the
    vertex average of each cell, with the analytic gradient there."""
    x = vertex_centers(mesh)
    ph = 2.0 * np.pi * x.sum(axis=1)
    rho = 1.0 + amp * np.sin(ph)
    drho = amp * 2.0 * np.pi * np.cos(ph)
    U, p = mach, 1.0 / gamma
    n = len(rho)
    W = np.zeros((5, n))
    W[0] = rho
    W[1] = rho * U
    W[4] = p / (gamma - 1.0) + 0.5 * rho * U * U
    G = np.zeros((15, n))
    for d in range(3):
        G[0 * 3 + d] = drho
        G[1 * 3 + d] = U * drho
        G[4 * 3 + d] = 0.5 * U * U * drho
    return W, G


# ---- design perturbations of the compression ramp (inputs of the adjoint checks) ------------------

def ramp_wall_modes(mesh, n_modes=64, angle_deg=15.0, sigma=0.08, depth=0.5, seed=2402):
    """Node displacement fields [n_modes][n_nodes][3] of the ramp_box wall: mode m moves the nodes
    normal to the x axis in y by exp(-(x - x_m)^2 / (2 sigma^2)) (x_m seeded uniform in [-0.3, 1.3]),
    faded linearly to zero at height `depth` above the wall; independent of z, so periodic copies of
    a node move together."""
    xyz = mesh["xyz"]
    rng = np.random.default_rng(seed)
    xm = rng.uniform(-0.3, 1.3, n_modes)
    t = np.tan(np.radians(angle_deg))
    eta = xyz[:, 1] - np.where(xyz[:, 0] > 0.0, xyz[:, 0] * t, 0.0)
    fade = np.clip(1.0 - eta / depth, 0.0, 1.0)
    out = np.zeros((n_modes, len(xyz), 3))
    out[:, :, 1] = np.exp(-(xyz[None, :, 0] - xm[:, None]) ** 2 / (2.0 * sigma ** 2)) * fade[None, :]
    return out


def displaced(mesh, field, eps):
    """Copy of a mesh dict with its nodes moved by eps * field ([n_nodes][3])."""
    out = dict(mesh)
    out["xyz"] = np.ascontiguousarray(mesh["xyz"] + eps * field)
    return out
