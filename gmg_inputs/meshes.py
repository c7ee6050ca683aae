"""Seeded synthetic surfaces: the inputs the multigrid path is exercised on.

The paper evaluates on scanned meshes and point clouds (Sec. 5.3) that are not
available here; these generators stand in for them at comparable sizes and
structure (closed manifold triangle meshes with about 7 nonzeros per Laplacian
row, noisy point clouds with k-nearest-neighbour graphs, and a non-manifold
triangle mesh whose spine edges border more than two triangles, the kind of
input Sec. 5.4 smooths on non-manifold meshes).

Nothing in this module performs any step of the multigrid method itself.
"""
from __future__ import annotations

import numpy as np

_PHI = (1.0 + 5.0 ** 0.5) / 2.0


def sorted_unique(key: np.ndarray) -> np.ndarray:
    """np.unique of a 1-D integer array (sorted distinct values) by one sort and
    a mask of value changes: the same result, and far faster than np.unique on
    tens of millions of keys with some numpy versions."""
    s = np.sort(key, kind="stable")
    if s.size == 0:
        return s
    m = np.empty(s.size, dtype=bool)
    m[0] = True
    np.not_equal(s[1:], s[:-1], out=m[1:])
    return s[m]

# Regular icosahedron: 12 vertices at the cyclic permutations of (0, +-1, +-phi),
# 20 faces, outward orientation.
_ICO_V = np.array(
    [
        [-1, _PHI, 0], [1, _PHI, 0], [-1, -_PHI, 0], [1, -_PHI, 0],
        [0, -1, _PHI], [0, 1, _PHI], [0, -1, -_PHI], [0, 1, -_PHI],
        [_PHI, 0, -1], [_PHI, 0, 1], [-_PHI, 0, -1], [-_PHI, 0, 1],
    ],
    dtype=np.float64,
)
_ICO_F = np.array(
    [
        [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
        [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
        [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
        [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
    ],
    dtype=np.int64,
)


def icosphere(level: int):
    """Icosahedron subdivided `level` times by edge midpoints, projected to the
    unit sphere.  Returns (V float64 [n,3], F int64 [m,3]); n = 10*4^level + 2.
    Vertex numbering is creation order (the 12 corners first, then midpoints)."""
    V = [v / np.linalg.norm(v) for v in _ICO_V]
    F = [tuple(f) for f in _ICO_F]
    for _ in range(level):
        mid = {}

        def midpoint(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in mid:
                p = V[a] + V[b]
                V.append(p / np.linalg.norm(p))
                mid[key] = len(V) - 1
            return mid[key]

        nf = []
        for a, b, c in F:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        F = nf
    return np.asarray(V, dtype=np.float64), np.asarray(F, dtype=np.int64)


def torus_grid(n_major: int, n_minor: int, R: float = 1.0, r: float = 0.3):
    """Torus sampled on a regular (angle) grid.  Vertex (i, j) -> i*n_minor + j,
    position ((R + r cos v) cos u, (R + r cos v) sin u, r sin v) with
    u = 2 pi i / n_major, v = 2 pi j / n_minor.  Every grid quad is split along
    the same diagonal, so every vertex has degree 6."""
    i = np.arange(n_major)[:, None]
    j = np.arange(n_minor)[None, :]
    u = 2.0 * np.pi * i / n_major
    v = 2.0 * np.pi * j / n_minor
    x = (R + r * np.cos(v)) * np.cos(u)
    y = (R + r * np.cos(v)) * np.sin(u)
    z = r * np.sin(v) * np.ones_like(u)
    V = np.stack([x, y, z], axis=-1).reshape(-1, 3)
    ii = np.arange(n_major)[:, None]
    jj = np.arange(n_minor)[None, :]
    a = ii * n_minor + jj
    b = ((ii + 1) % n_major) * n_minor + jj
    c = ((ii + 1) % n_major) * n_minor + (jj + 1) % n_minor
    d = ii * n_minor + (jj + 1) % n_minor
    t1 = np.stack([a, b, c], axis=-1).reshape(-1, 3)
    t2 = np.stack([a, c, d], axis=-1).reshape(-1, 3)
    F = np.concatenate([t1, t2], axis=0).astype(np.int64)
    return V.astype(np.float64), F


def mesh_edges(F: np.ndarray) -> np.ndarray:
    """Unique undirected edges (i < j) of a triangle list, sorted."""
    e = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]], axis=0).astype(np.int64)
    e = np.sort(e, axis=1)
    n = int(e.max()) + 1 if e.size else 1
    key = sorted_unique(e[:, 0] * n + e[:, 1])  # lexicographic order of (i, j) is the order of i n + j
    return np.stack([key // n, key % n], axis=1)


def mean_edge_length(V: np.ndarray, E: np.ndarray) -> float:
    return float(np.linalg.norm(V[E[:, 0]] - V[E[:, 1]], axis=1).mean())


def jitter(V: np.ndarray, F: np.ndarray, rng: np.random.Generator, amount: float = 0.2):
    """Each coordinate += U(-amount, amount) * (mean edge length of the input)."""
    e = mean_edge_length(V, mesh_edges(F))
    return V + rng.uniform(-amount, amount, size=V.shape) * e


def jittered_torus(n_major: int, n_minor: int, seed: int):
    """Torus R=1, r=0.3 on an n_major x n_minor grid with every coordinate
    perturbed by U(-0.2, 0.2) x mean edge length.  Returns (V, F, rng) where rng
    is the seeded generator advanced past the jitter draws (the right-hand sides
    are drawn from it next)."""
    rng = np.random.default_rng(seed)
    V, F = torus_grid(n_major, n_minor)
    return jitter(V, F, rng), F, rng


def fibonacci_sphere(n: int) -> np.ndarray:
    """n points of the spherical Fibonacci lattice on the unit sphere."""
    k = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * k + 1.0) / n
    rad = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    golden = np.pi * (3.0 - 5.0 ** 0.5)
    th = golden * k
    return np.stack([rad * np.cos(th), rad * np.sin(th), z], axis=1)


def sphere_hull_mesh(P: np.ndarray) -> np.ndarray:
    """Triangulate points on the unit sphere by their convex hull (on a sphere
    this is the spherical Delaunay triangulation).  Faces oriented outward."""
    from scipy.spatial import ConvexHull

    F = ConvexHull(P).simplices.astype(np.int64)
    a, b, c = P[F[:, 0]], P[F[:, 1]], P[F[:, 2]]
    nrm = np.cross(b - a, c - a)
    flip = np.einsum("ij,ij->i", nrm, a + b + c) < 0
    F[flip] = F[flip][:, [0, 2, 1]]
    return F


def jittered_sphere(n: int, rng: np.random.Generator, amount: float = 0.2):
    """Fibonacci sphere with tangential jitter U(-amount, amount) x mean edge
    length per coordinate, re-projected to the sphere and re-triangulated."""
    P = fibonacci_sphere(n)
    F0 = sphere_hull_mesh(P)
    e = mean_edge_length(P, mesh_edges(F0))
    Q = P + rng.uniform(-amount, amount, size=P.shape) * e
    Q /= np.linalg.norm(Q, axis=1, keepdims=True)
    return Q, sphere_hull_mesh(Q)


def noisy_sphere_cloud(n: int, rng: np.random.Generator, sigma: float = 1e-3):
    """n points uniform on the unit sphere with Gaussian radial noise sigma."""
    g = rng.standard_normal((n, 3))
    u = g / np.linalg.norm(g, axis=1, keepdims=True)
    z = rng.standard_normal(n)
    return u * (1.0 + sigma * z)[:, None]


def book(pages: int, n_radial: int, n_spine: int, height: float = 1.0, seed: int = 0, amount: float = 0.2):
    """A non-manifold "book": `pages` rectangular sheets that share one spine
    line (the z axis).  Sheet p lies in the half-plane at angle 2 pi p / pages
    around the spine and is bent into a quarter-cylinder arc away from it;
    vertex (i, j) of a sheet sits at radial index i = 0..n_radial-1 and spine
    index j = 0..n_spine-1, and the i = 0 column is the shared spine (one vertex
    per j for all sheets).  Every grid quad is split along the same diagonal,
    so each spine edge borders one triangle of every sheet: `pages` triangles.  All vertices but the
    spine are then jittered by U(-amount, amount) x mean edge length per
    coordinate.  Returns (V, F, rng), rng advanced past the jitter draws."""
    rng = np.random.default_rng(seed)
    h = height / (n_spine - 1)
    spine = np.stack([np.zeros(n_spine), np.zeros(n_spine), h * np.arange(n_spine)], axis=1)
    V = [spine]
    F = []
    idx = lambda p, i, j: j if i == 0 else n_spine + p * (n_radial - 1) * n_spine + (i - 1) * n_spine + j
    for p in range(pages):
        th = 2.0 * np.pi * p / pages
        d = np.array([np.cos(th), np.sin(th), 0.0])        # radial direction of the sheet
        q = np.array([-np.sin(th), np.cos(th), 0.0])       # bending direction
        i = np.arange(1, n_radial)[:, None]
        j = np.arange(n_spine)[None, :]
        s = i * h                                          # arc length from the spine
        R = (n_radial - 1) * h * 2.0 / np.pi                # quarter circle over the sheet's width
        a = s / R
        pos = (R * np.sin(a))[..., None] * d + (R * (1.0 - np.cos(a)))[..., None] * q
        pos = np.broadcast_to(pos, (n_radial - 1, n_spine, 3)).copy()
        pos[..., 2] = (h * j) * np.ones_like(s)
        V.append(pos.reshape(-1, 3))
        for ii in range(n_radial - 1):
            for jj in range(n_spine - 1):
                a0, b0 = idx(p, ii, jj), idx(p, ii + 1, jj)
                c0, d0 = idx(p, ii + 1, jj + 1), idx(p, ii, jj + 1)
                F += [(a0, b0, c0), (a0, c0, d0)]
    V = np.concatenate(V, axis=0)
    F = np.asarray(F, dtype=np.int64)
    e = mean_edge_length(V, mesh_edges(F))
    J = rng.uniform(-amount, amount, size=V.shape) * e
    J[:n_spine] = 0.0  # the spine stays straight (it is shared by every sheet)
    return V + J, F, rng
