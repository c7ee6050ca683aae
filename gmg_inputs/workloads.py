"""The seeded synthetic workloads (systems A x = b plus their hierarchies).

Every workload is a data-smoothing system of the form of Eq. (smoothing),
(M + t L) x = M y, or its point-cloud analogue (I + t L) x = y, with the
prolongation hierarchy of Sec. 4 built on the surface's points and edges.

  icosphere5  : icosahedron subdivided 5x (10,242 vertices), t = 1e-3, seed 0
  torus1m     : jittered torus 2048 x 512 (1,048,576 vertices), t = 1e-4, seed 1
  cloud4m     : 4,194,304 noisy sphere points, k = 30 kNN Gaussian Laplacian,
                (I + 1e-3 L) x = y, seed 2
  spheres64   : 64 jittered spheres, sizes log-uniform in [5e3, 2e5], t = 1e-3,
                8 right-hand sides each, seed 3
  heat512k    : jittered torus 1024 x 512 (524,288 vertices), t = 1e-3, u0 one-hot
                at 16 random vertices, x_target ~ N(0, 1), seed 4

  book5       : data smoothing on a non-manifold mesh (5 bent sheets sharing a spine,
                149,200 vertices), t = 1e-3, seed 7

Two further systems of the paper on jittered tori, with the same hierarchy recipe:
  poisson     : Eq. (Poisson) of Sec. 5.2, (S + eta M) x = M y with eta = 1e-6
                (nearly singular: the constant mode has eigenvalue ~eta M)
  bilaplacian : the bi-Laplacian smoothing of Sec. 5.5,
                (M + alpha S + beta S M^-1 S) x = M y (two-ring stencil)

Small variants of the same recipes (fewer vertices) serve the tests.
"""
from __future__ import annotations

import os
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from . import meshes, operators
from .hierarchy import Prolongation, build_hierarchy

_CACHE = os.environ.get("GMG_CACHE", os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                                  "_cache"))


@dataclass
class System:
    name: str
    A: sp.csr_matrix            # system matrix, CSR, sorted columns, diagonal present
    b: np.ndarray               # right-hand side(s): [n] or [n, nrhs]
    Ps: list                    # list[Prolongation], finest first
    Mdiag: np.ndarray | None = None   # lumped mass (None for the point cloud: M = I)
    L: sp.csr_matrix | None = None    # Laplacian
    t: float = 0.0
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.A.shape[0]


def _mesh_system(name, V, F, t, y, phi=1.0 / 8.0, stop=1000):
    L = operators.cotan_laplacian(V, F)
    Md = operators.lumped_mass(V, F)
    A = operators.system_matrix(Md, L, t)
    rp, ci = operators.edges_to_adjacency(V.shape[0], meshes.mesh_edges(F))
    Ps = build_hierarchy(V, rp, ci, phi=phi, stop=stop)
    b = Md[:, None] * y if y.ndim == 2 else Md * y
    return System(name, A, b, Ps, Md, L, t)


def icosphere_system(level: int = 5, t: float = 1e-3, seed: int = 0, stop: int = 1000):
    V, F = meshes.icosphere(level)
    rng = np.random.default_rng(seed)
    y = rng.standard_normal(V.shape[0])
    return _mesh_system(f"icosphere{level}", V, F, t, y, stop=stop)


def torus_system(n_major: int, n_minor: int, t: float, seed: int, stop: int = 1000):
    V, F, rng = meshes.jittered_torus(n_major, n_minor, seed)
    y = rng.standard_normal(V.shape[0])
    return _mesh_system(f"torus{n_major}x{n_minor}", V, F, t, y, stop=stop)


def poisson_system(n_major: int = 256, n_minor: int = 120, eta: float = 1e-6, seed: int = 5, stop: int = 1000):
    """Eq. (Poisson) on a jittered torus: (S + eta M) x = M y, y ~ N(0, 1)."""
    V, F, rng = meshes.jittered_torus(n_major, n_minor, seed)
    L = operators.cotan_laplacian(V, F)
    Md = operators.lumped_mass(V, F)
    A = operators.poisson_matrix(Md, L, eta)
    rp, ci = operators.edges_to_adjacency(V.shape[0], meshes.mesh_edges(F))
    Ps = build_hierarchy(V, rp, ci, stop=stop)
    y = rng.standard_normal(V.shape[0])
    return System(f"poisson{n_major}x{n_minor}", A, Md * y, Ps, Md, L, eta)


def bilaplacian_system(n_major: int = 256, n_minor: int = 120, alpha: float = 1e-3, beta: float = 1e-7,
                       seed: int = 6, stop: int = 1000):
    """Bi-Laplacian smoothing (Sec. 5.5) on a jittered torus:
    (M + alpha S + beta S M^-1 S) x = M y, y ~ N(0, 1).  The hierarchy is
    built on the mesh edges, as for the other systems."""
    V, F, rng = meshes.jittered_torus(n_major, n_minor, seed)
    L = operators.cotan_laplacian(V, F)
    Md = operators.lumped_mass(V, F)
    A = operators.bilaplacian_matrix(Md, L, alpha, beta)
    rp, ci = operators.edges_to_adjacency(V.shape[0], meshes.mesh_edges(F))
    Ps = build_hierarchy(V, rp, ci, stop=stop)
    y = rng.standard_normal(V.shape[0])
    return System(f"bilaplacian{n_major}x{n_minor}", A, Md * y, Ps, Md, L, alpha,
                  extra=dict(beta=np.array(beta)))


def nonmanifold_system(pages: int = 5, n_radial: int = 150, n_spine: int = 200, t: float = 1e-3, seed: int = 7,
                       stop: int = 1000):
    """Data smoothing (M + t L) x = M y on the non-manifold book mesh
    (meshes.book: `pages` bent sheets sharing one spine whose edges border
    `pages` triangles), cotan Laplacian and lumped mass summed over every
    triangle (both stay well defined on non-manifold edges), y ~ N(0, 1).  The
    hierarchy of Sec. 4 is built on the mesh's edge graph."""
    V, F, rng = meshes.book(pages, n_radial, n_spine, seed=seed)
    y = rng.standard_normal(V.shape[0])
    return _mesh_system(f"book{pages}x{n_radial}x{n_spine}", V, F, t, y, stop=stop)


def cloud_system(n: int, k: int = 30, t: float = 1e-3, seed: int = 2, stop: int = 1000, graph_k: int = 6):
    """Point cloud: the system uses the k-nearest-neighbour Gaussian
    Laplacian; the hierarchy is built on the sparser union graph of the
    graph_k nearest neighbours, the point-cloud neighbourhood graph of Sec. 4.1
    (local 1-ring-sized neighbourhoods)."""
    rng = np.random.default_rng(seed)
    P = meshes.noisy_sphere_cloud(n, rng)
    E, h = operators.knn_graph(P, k)
    L = operators.knn_laplacian(P, E, h)
    A = operators.system_matrix(np.ones(n), L, t)
    y = rng.standard_normal(n)
    Eg, _ = operators.knn_graph(P, graph_k)
    rp, ci = operators.edges_to_adjacency(n, Eg)
    Ps = build_hierarchy(P, rp, ci, stop=stop)
    return System(f"cloud{n}", A, y, Ps, None, L, t, extra=dict(h=h))


def spheres_batch(count: int = 64, lo: float = 5e3, hi: float = 2e5, nrhs: int = 8, t: float = 1e-3,
                  seed: int = 3, stop: int = 1000):
    rng = np.random.default_rng(seed)
    sizes = np.round(np.exp(rng.uniform(np.log(lo), np.log(hi), size=count))).astype(np.int64)
    out = []
    for i, n in enumerate(sizes):
        V, F = meshes.jittered_sphere(int(n), rng)
        Y = rng.standard_normal((int(n), nrhs))
        out.append(_mesh_system(f"sphere{i}_{n}", V, F, t, Y, stop=stop))
    return out


def heat_system(n_major: int = 1024, n_minor: int = 512, t: float = 1e-3, seed: int = 4, hot: int = 16,
                stop: int = 1000):
    V, F, rng = meshes.jittered_torus(n_major, n_minor, seed)
    n = V.shape[0]
    hot_idx = np.sort(rng.choice(n, size=hot, replace=False))
    u0 = np.zeros(n)
    u0[hot_idx] = 1.0
    x_target = rng.standard_normal(n)
    s = _mesh_system(f"heat{n_major}x{n_minor}", V, F, t, u0, stop=stop)
    s.extra.update(u0=u0, hot=hot_idx, x_target=x_target)
    return s


# ---- caching (the big workloads take seconds to build) --------------------

def _save(path, s: System):
    d = dict(indptr=s.A.indptr, indices=s.A.indices, data=s.A.data, b=s.b, t=s.t, nlev=len(s.Ps))
    if s.Mdiag is not None:
        d["Mdiag"] = s.Mdiag
    if s.L is not None:
        d.update(L_indptr=s.L.indptr, L_indices=s.L.indices, L_data=s.L.data)
    for l, P in enumerate(s.Ps):
        d[f"P{l}_idx"], d[f"P{l}_w"], d[f"P{l}_nc"] = P.idx, P.w, P.n_coarse
    for k, v in s.extra.items():
        d[f"x_{k}"] = v
    tmp = path + f".{os.getpid()}.tmp.npz"
    np.savez(tmp, **d)
    os.replace(tmp, path)


def _load(path, name) -> System:
    z = np.load(path)
    n = z["indptr"].size - 1
    A = sp.csr_matrix((z["data"], z["indices"], z["indptr"]), shape=(n, n))
    L = None
    if "L_data" in z:
        L = sp.csr_matrix((z["L_data"], z["L_indices"], z["L_indptr"]), shape=(n, n))
    Ps, nf = [], n
    for l in range(int(z["nlev"])):
        P = Prolongation(nf, int(z[f"P{l}_nc"]), z[f"P{l}_idx"], z[f"P{l}_w"])
        Ps.append(P)
        nf = P.n_coarse
    extra = {k[2:]: z[k] for k in z.files if k.startswith("x_")}
    return System(name, A, z["b"], Ps, z["Mdiag"] if "Mdiag" in z else None, L, float(z["t"]), extra)


def is_cached(name: str) -> bool:
    """Whether the named workload's inputs are in the cache already."""
    return os.path.exists(os.path.join(_CACHE, name + ".npz")) or os.path.exists(os.path.join(_CACHE, name, "count"))


def cached(name: str, maker, *args, **kw) -> System:
    os.makedirs(_CACHE, exist_ok=True)
    path = os.path.join(_CACHE, name + ".npz")
    if os.path.exists(path):
        try:
            return _load(path, name)
        except Exception:
            pass
    s = maker(*args, **kw)
    s.name = name
    _save(path, s)
    return s


def cached_batch(name: str, maker, *args, **kw) -> list:
    """Like `cached` for a list of systems (one .npz per system under a
    directory named after the batch)."""
    d = os.path.join(_CACHE, name)
    try:
        with open(os.path.join(d, "count")) as f:
            count = int(f.read())
        return [_load(os.path.join(d, f"{k}.npz"), f"{name}_{k}") for k in range(count)]
    except Exception:
        pass
    out = maker(*args, **kw)
    os.makedirs(d, exist_ok=True)
    for k, s in enumerate(out):
        _save(os.path.join(d, f"{k}.npz"), s)
    tmp = os.path.join(d, f"count.{os.getpid()}")
    with open(tmp, "w") as f:
        f.write(str(len(out)))
    os.replace(tmp, os.path.join(d, "count"))
    return out


def workload(name: str) -> System:
    """The named full-size workloads (see the module docstring)."""
    if name == "icosphere5":
        return cached(name, icosphere_system, 5, 1e-3, 0)
    if name == "torus1m":
        return cached(name, torus_system, 2048, 512, 1e-4, 1)
    if name == "heat512k":
        return cached(name, heat_system)
    if name == "cloud4m":
        return cached(name, cloud_system, 4194304)
    if name == "cloud1m":  # the same recipe at 1,048,576 points (kernel captures that must stay small)
        return cached(name, cloud_system, 1048576)
    if name == "book5":
        return cached(name, nonmanifold_system)
    raise KeyError(name)
