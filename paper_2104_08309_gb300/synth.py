"""Seeded synthetic inputs: polygons, triangulated spheres and Q grids.

This module only builds geometry and sample points; it holds none of the
transform's arithmetic.  Both the CUDA path and the FP64 oracle consume what it
returns, so every coordinate is produced once, rounded to float32 (the storage
precision of vertices everywhere), and passed unchanged to both sides.

Shapes follow the families the paper computes on: single polygons (Sec. 4.1),
a rectangular prism (Sec. 4.2), a triangulated sphere (Sec. 4.3) and a union of
spheres (Sec. 4.4).  Random numbers come from NumPy's PCG64 (``default_rng``).
"""
from __future__ import annotations

import itertools

import numpy as np

__all__ = [
    "star_polygon", "regular_polygon", "rectangle", "batched_star_polygons",
    "icosahedron", "icosphere", "perturbed_icosphere", "sphere_union",
    "box_mesh", "q_grid_2d", "q_grid_3d", "q_subsample", "Workload",
    "workload_c1", "workload_c2", "workload_c3", "workload_c4", "workload_c5",
]


# ----------------------------------------------------------------------------
# 2D shapes: vertex arrays [n, 2] float32, counter-clockwise unless stated.
# ----------------------------------------------------------------------------

def star_polygon(n: int, seed: int, noise: float = 0.3, center=(0.0, 0.0)) -> np.ndarray:
    """Star-shaped polygon: theta_k = 2 pi k / n, r_k = 1 + noise * U[0, 1).

    Returned counter-clockwise, so its transform at Q = 0 is its (positive) area.
    """
    rng = np.random.default_rng(seed)
    return _star(n, rng, noise, center)


def _star(n, rng, noise, center):
    theta = 2.0 * np.pi * np.arange(n) / n
    r = 1.0 + noise * rng.random(n)
    xy = np.stack([center[0] + r * np.cos(theta), center[1] + r * np.sin(theta)], axis=1)
    return xy.astype(np.float32)


def regular_polygon(n: int, radius: float = 1.0) -> np.ndarray:
    """Regular n-gon inscribed in a circle of the given radius, CCW."""
    theta = 2.0 * np.pi * np.arange(n) / n
    return np.stack([radius * np.cos(theta), radius * np.sin(theta)], axis=1).astype(np.float32)


def rectangle(a: float, b: float) -> np.ndarray:
    """Rectangle with its lower-left corner at the origin, traversed CCW (Sec. 4.1)."""
    return np.array([[0, 0], [a, 0], [a, b], [0, b]], dtype=np.float32)


def batched_star_polygons(n_polys: int, seed: int, nmin: int = 8, nmax: int = 4096,
                          noise: float = 0.3):
    """Many star polygons with log-uniform vertex counts, packed as CSR.

    N_i = round(exp(U[ln nmin, ln nmax])), centres U[-1, 1)^2.
    Returns (verts [sum N_i, 2] float32, poly_off [n_polys + 1] int64).
    """
    rng = np.random.default_rng(seed)
    counts = np.rint(np.exp(rng.uniform(np.log(nmin), np.log(nmax), n_polys))).astype(np.int64)
    counts = np.clip(counts, 3, None)
    centers = rng.uniform(-1.0, 1.0, size=(n_polys, 2))
    parts = [_star(int(c), rng, noise, centers[i]) for i, c in enumerate(counts)]
    off = np.zeros(n_polys + 1, dtype=np.int64)
    off[1:] = np.cumsum(counts)
    return np.concatenate(parts, axis=0), off


# ----------------------------------------------------------------------------
# 3D closed triangle meshes: verts [V, 3] float32, faces [F, 3] int32, every
# face counter-clockwise seen from outside (outward normal by the right hand).
# ----------------------------------------------------------------------------

def icosahedron():
    """Unit icosahedron built from its 12 vertices (0, +-1, +-g) and cyclic shifts.

    Faces are the vertex triples at mutual distance 2 (the edge length before
    normalisation), oriented so that (p1-p0) x (p2-p0) points away from the centre.
    """
    g = (1.0 + 5.0 ** 0.5) / 2.0
    pts = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            pts += [(0.0, s1, s2 * g), (s1, s2 * g, 0.0), (s2 * g, 0.0, s1)]
    v = np.array(pts, dtype=np.float64)
    faces = []
    for i, j, k in itertools.combinations(range(12), 3):
        if all(abs(np.linalg.norm(v[a] - v[b]) - 2.0) < 1e-9 for a, b in ((i, j), (j, k), (i, k))):
            n = np.cross(v[j] - v[i], v[k] - v[i])
            faces.append((i, j, k) if np.dot(n, v[i]) > 0 else (i, k, j))
    assert len(faces) == 20
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v, np.array(faces, dtype=np.int64)


def _subdivide(v, f):
    """Split every triangle into four through its edge midpoints (projected to the unit sphere)."""
    nv = v.shape[0]
    e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]], axis=0)
    key = np.minimum(e[:, 0], e[:, 1]) * nv + np.maximum(e[:, 0], e[:, 1])
    uniq, inv = np.unique(key, return_inverse=True)
    a, b = uniq // nv, uniq % nv
    mid = v[a] + v[b]
    mid /= np.linalg.norm(mid, axis=1, keepdims=True)
    nf = f.shape[0]
    m = nv + inv.reshape(3, nf)            # midpoints of edges (0,1), (1,2), (2,0)
    m01, m12, m20 = m[0], m[1], m[2]
    f0, f1, f2 = f[:, 0], f[:, 1], f[:, 2]
    nfaces = np.concatenate([
        np.stack([f0, m01, m20], 1), np.stack([f1, m12, m01], 1),
        np.stack([f2, m20, m12], 1), np.stack([m01, m12, m20], 1)], axis=0)
    return np.concatenate([v, mid], axis=0), nfaces


def _unit_icosphere(level: int):
    v, f = icosahedron()
    for _ in range(level):
        v, f = _subdivide(v, f)
    return v, f


def icosphere(level: int, radius: float = 1.0, center=(0.0, 0.0, 0.0)):
    """Geodesic sphere: the icosahedron subdivided ``level`` times (20 * 4**level faces)."""
    v, f = _unit_icosphere(level)
    v = v * radius + np.asarray(center, dtype=np.float64)
    return v.astype(np.float32), f.astype(np.int32)


def perturbed_icosphere(level: int, seed: int, amp: float = 0.05, radius: float = 1.0):
    """Icosphere with each vertex moved radially by a factor 1 + amp * U[-1, 1)."""
    rng = np.random.default_rng(seed)
    v, f = _unit_icosphere(level)
    fac = 1.0 + amp * rng.uniform(-1.0, 1.0, size=v.shape[0])
    return (v * (radius * fac)[:, None]).astype(np.float32), f.astype(np.int32)


def sphere_union(n_spheres: int, level: int, seed: int, rmin: float = 0.2, rmax: float = 0.5,
                 perturb: float = 0.0, perturb_seed: int | None = None):
    """Concatenation of closed icospheres with radii U[rmin, rmax], centres U[0, 1)^3.

    The transform of the concatenated surface is that of the sum of the spheres'
    indicator functions (overlaps count twice).  With ``perturb`` > 0, every vertex
    is moved radially about its sphere's centre by a factor 1 + perturb * U[-1, 1)
    drawn from ``perturb_seed``; geometry otherwise matches the unperturbed call.
    """
    rng = np.random.default_rng(seed)
    radii = rng.uniform(rmin, rmax, n_spheres)
    centers = rng.uniform(0.0, 1.0, size=(n_spheres, 3))
    uv, uf = _unit_icosphere(level)
    prng = np.random.default_rng(perturb_seed) if perturb > 0 else None
    vs, fs = [], []
    for i in range(n_spheres):
        fac = radii[i] * (1.0 + perturb * prng.uniform(-1.0, 1.0, uv.shape[0])) if prng is not None \
            else np.full(uv.shape[0], radii[i])
        vs.append(uv * fac[:, None] + centers[i])
        fs.append(uf + i * uv.shape[0])
    return np.concatenate(vs).astype(np.float32), np.concatenate(fs).astype(np.int32)


def mesh_batch(n_meshes: int, seed: int, levels=(1, 2, 3, 4), rmin: float = 0.2, rmax: float = 0.5,
               amp: float = 0.05):
    """Many separate closed meshes for a batched transform: mesh i is an icosphere of a level drawn
    uniformly from ``levels``, radius U[rmin, rmax], centre U[-1, 1)^3, each vertex moved radially
    by 1 + amp * U[-1, 1).  Returns verts [V, 3] float32 (all meshes), faces [F, 3] int32 (global
    indices, mesh after mesh) and mesh_off [n_meshes + 1] int64 (CSR over faces)."""
    rng = np.random.default_rng(seed)
    lv = rng.choice(np.asarray(levels), n_meshes)
    radii = rng.uniform(rmin, rmax, n_meshes)
    centers = rng.uniform(-1.0, 1.0, size=(n_meshes, 3))
    cache = {}
    vs, fs, off, nv = [], [], [0], 0
    for i in range(n_meshes):
        if lv[i] not in cache:
            cache[lv[i]] = _unit_icosphere(int(lv[i]))
        uv, uf = cache[lv[i]]
        fac = radii[i] * (1.0 + amp * rng.uniform(-1.0, 1.0, uv.shape[0]))
        vs.append(uv * fac[:, None] + centers[i])
        fs.append(uf + nv)
        nv += uv.shape[0]
        off.append(off[-1] + uf.shape[0])
    return (np.concatenate(vs).astype(np.float32), np.concatenate(fs).astype(np.int32),
            np.asarray(off, dtype=np.int64))


def box_mesh(a: float, b: float, c: float):
    """Rectangular prism [0,a] x [0,b] x [0,c] as 12 outward triangles (Sec. 4.2).

    Faces 0-1 are the top (z = c) and 2-3 the bottom (z = 0).
    """
    v = np.array([[0, 0, 0], [a, 0, 0], [a, b, 0], [0, b, 0],
                  [0, 0, c], [a, 0, c], [a, b, c], [0, b, c]], dtype=np.float32)
    f = np.array([
        [4, 5, 6], [4, 6, 7],      # top, normal +z
        [0, 2, 1], [0, 3, 2],      # bottom, normal -z
        [0, 1, 5], [0, 5, 4],      # y = 0, normal -y
        [3, 7, 6], [3, 6, 2],      # y = b, normal +y
        [0, 4, 7], [0, 7, 3],      # x = 0, normal -x
        [1, 2, 6], [1, 6, 5],      # x = a, normal +x
    ], dtype=np.int32)
    return v, f


# ----------------------------------------------------------------------------
# 3D closed surfaces of planar polygon faces, CSR: verts [V, 3] float32,
# face_idx [sum of face sizes] int32, face_off [F + 1] int64; each face
# counter-clockwise seen from outside.
# ----------------------------------------------------------------------------

def box_quads(a: float, b: float, c: float):
    """Rectangular prism [0,a] x [0,b] x [0,c] as 6 outward quadrilaterals."""
    v = np.array([[0, 0, 0], [a, 0, 0], [a, b, 0], [0, b, 0],
                  [0, 0, c], [a, 0, c], [a, b, c], [0, b, c]], dtype=np.float32)
    idx = np.array([4, 5, 6, 7,       # top, normal +z
                    0, 3, 2, 1,       # bottom, normal -z
                    0, 1, 5, 4,       # y = 0
                    3, 7, 6, 2,       # y = b
                    0, 4, 7, 3,       # x = 0
                    1, 2, 6, 5],      # x = a
                   dtype=np.int32)
    return v, idx, np.arange(0, 25, 4, dtype=np.int64)


def extruded_polygon(poly, h: float, z0: float = 0.0):
    """The prism over a counter-clockwise simple polygon poly [n, 2] between z0 and z0 + h:
    two n-gon caps and n side quadrilaterals (planar faces, caps possibly non-convex)."""
    poly = np.asarray(poly, dtype=np.float64)
    n = poly.shape[0]
    v = np.concatenate([np.column_stack([poly, np.full(n, z0)]),
                        np.column_stack([poly, np.full(n, z0 + h)])]).astype(np.float32)
    k = np.arange(n)
    sides = np.stack([k, (k + 1) % n, n + (k + 1) % n, n + k], axis=1).reshape(-1)
    idx = np.concatenate([n + k, k[::-1], sides]).astype(np.int32)      # top, bottom, sides
    off = np.concatenate([[0, n, 2 * n], 2 * n + 4 * np.arange(1, n + 1)]).astype(np.int64)
    return v, idx, off


def voxel_ball(n: int, radius: float, d: float):
    """Occupancy [n, n, n] of the cubes of side d (grid centred on the origin) whose centres lie
    inside the ball of the given radius."""
    c = (np.arange(n) + 0.5 - 0.5 * n) * d
    x, y, z = np.meshgrid(c, c, c, indexing="ij")
    return x * x + y * y + z * z < radius * radius


def voxel_surface(occ, d: float):
    """The closed boundary of a set of cubes as outward quadrilaterals (CSR polygon mesh).

    occ [nx, ny, nz] bool; cube (i, j, k) spans [i d, (i+1) d] x ... shifted so the grid is centred
    on the origin.  A face is emitted wherever an occupied cube meets an empty one (or the grid's
    edge).  Returns verts [V, 3] float32 (grid points), face_idx int32, face_off int64.
    """
    occ = np.asarray(occ, dtype=bool)
    nx, ny, nz = occ.shape
    pad = np.zeros((nx + 2, ny + 2, nz + 2), dtype=bool)
    pad[1:-1, 1:-1, 1:-1] = occ
    quads = []
    # unit offsets of the 4 corners of the +axis face of a cube, counter-clockwise seen from outside
    corner = {0: [(1, 0, 0), (1, 1, 0), (1, 1, 1), (1, 0, 1)],
              1: [(0, 1, 0), (0, 1, 1), (1, 1, 1), (1, 1, 0)],
              2: [(0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]}
    for ax in range(3):
        e = np.zeros(3, dtype=int)
        e[ax] = 1
        nb = pad[1 + e[0]:nx + 1 + e[0], 1 + e[1]:ny + 1 + e[1], 1 + e[2]:nz + 1 + e[2]]
        nbm = pad[1 - e[0]:nx + 1 - e[0], 1 - e[1]:ny + 1 - e[1], 1 - e[2]:nz + 1 - e[2]]
        for sign, other in ((1, nb), (-1, nbm)):
            cells = np.argwhere(occ & ~other)
            # the -axis face: the same corners moved to the cube's low side, in reverse order
            offs = np.array(corner[ax]) if sign > 0 else \
                np.array([[0 if a == ax else c[a] for a in range(3)] for c in corner[ax]])[::-1]
            quads.append(cells[:, None, :] + offs[None, :, :])
    q = np.concatenate(quads).reshape(-1, 3)
    keys, inv = np.unique(q, axis=0, return_inverse=True)
    verts = ((keys - 0.5 * np.array([nx, ny, nz])) * d).astype(np.float32)
    idx = inv.reshape(-1).astype(np.int32)
    off = np.arange(0, idx.size + 1, 4, dtype=np.int64)
    return verts, idx, off


# ----------------------------------------------------------------------------
# Q samples (float64 at the boundary).
# ----------------------------------------------------------------------------

def _axis(n: int, L: float) -> np.ndarray:
    # Q_k = -L + k * 2L / n, k = 0..n-1: contains -L and 0, excludes +L.
    return -L + np.arange(n, dtype=np.float64) * (2.0 * L / n)


def q_grid_2d(n: int, L: float) -> np.ndarray:
    ax = _axis(n, L)
    qx, qy = np.meshgrid(ax, ax, indexing="ij")
    return np.stack([qx.ravel(), qy.ravel()], axis=1)


def q_grid_3d(n: int, L: float) -> np.ndarray:
    ax = _axis(n, L)
    qx, qy, qz = np.meshgrid(ax, ax, ax, indexing="ij")
    return np.stack([qx.ravel(), qy.ravel(), qz.ravel()], axis=1)


def q_subsample_indices(q: np.ndarray, n: int, seed: int, include_zero: bool = True) -> np.ndarray:
    """Sorted indices of a seeded subset of the rows of q (without replacement); keeps Q = 0 if present."""
    rng = np.random.default_rng(seed)
    idx = rng.choice(q.shape[0], size=min(n, q.shape[0]), replace=False)
    if include_zero:
        z = np.flatnonzero(np.all(q == 0.0, axis=1))
        if z.size and z[0] not in idx:
            idx[0] = z[0]
    return np.sort(idx)


def q_subsample(q: np.ndarray, n: int, seed: int, include_zero: bool = True) -> np.ndarray:
    """Seeded subset of the rows of q (without replacement); keeps Q = 0 if present."""
    return q[q_subsample_indices(q, n, seed, include_zero)]


# The seeded 4,096-point Q subsample of the 128^3 grid on which the 1.31M-face mesh is checked
# against the FP64 oracle (it includes Q = 0).
C5_SUBSAMPLE = (4096, 5)


def c5_subsample_indices(q: np.ndarray) -> np.ndarray:
    n, seed = C5_SUBSAMPLE
    return q_subsample_indices(q, n, seed, include_zero=True)


# ----------------------------------------------------------------------------
# The five named workloads.
# ----------------------------------------------------------------------------

class Workload(dict):
    """A named input set: geometry arrays plus the Q sample (attribute access)."""
    __getattr__ = dict.__getitem__


def workload_c1():
    """64-vertex star polygon (seed 1), Q on 128^2 over [-40, 40)^2."""
    return Workload(name="star64_q128x128", dim=2, verts=star_polygon(64, seed=1),
                    q=q_grid_2d(128, 40.0))


def workload_c2():
    """Unit icosphere, subdivision 5 (20,480 triangles), Q on 64^3 over [-30, 30)^3."""
    v, f = icosphere(5)
    return Workload(name="icosphere5_q64cubed", dim=3, verts=v, faces=f, q=q_grid_3d(64, 30.0))


def workload_c3(n_polys: int = 4096):
    """4,096 star polygons, vertex counts log-uniform in [8, 4096] (seed 3), Q 64^2 over [-50, 50)^2."""
    v, off = batched_star_polygons(n_polys, seed=3)
    return Workload(name="batched4096stars_q64x64", dim=2, verts=v, poly_off=off,
                    q=q_grid_2d(64, 50.0))


def workload_c4():
    """16 icospheres (subdivision 4) with radii U[0.2, 0.5], centres U[0,1)^3 (seed 4), Q 32^3 over [-30, 30)^3.

    ``verts_target`` is the same surface with each vertex moved radially by 2 %
    (seed 44); the intensity target of the loss is |F|^2 of that copy.
    """
    v, f = sphere_union(16, 4, seed=4)
    vt, _ = sphere_union(16, 4, seed=4, perturb=0.02, perturb_seed=44)
    return Workload(name="union16icospheres4_q32cubed", dim=3, verts=v, faces=f,
                    verts_target=vt, q=q_grid_3d(32, 30.0))


def workload_c5():
    """Icosphere subdivision 8 (1,310,720 triangles), radii x (1 + 0.05 U[-1,1)) (seed 5), Q 128^3 over [-60, 60)^3."""
    v, f = perturbed_icosphere(8, seed=5, amp=0.05)
    return Workload(name="icosphere8_perturbed_q128cubed", dim=3, verts=v, faces=f,
                    q=q_grid_3d(128, 60.0))
