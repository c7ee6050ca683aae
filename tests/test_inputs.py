"""Pins of the input generators and of the operators of Sec. 5.2 (cotan
Laplacian S, lumped mass M) against facts that do not depend on this code:
mesh topology counts, the linear precision of the cotan Laplacian on flat
meshes, the exact area of flat patches, and the Laplace-Beltrami spectrum of
the unit sphere (first eigenvalue 2)."""
import numpy as np
import pytest
import scipy.sparse as sp

from gmg_inputs import meshes, operators, workloads


@pytest.mark.parametrize("level", [0, 1, 2, 3])
def test_icosphere_topology(level):
    V, F = meshes.icosphere(level)
    E = meshes.mesh_edges(F)
    assert V.shape[0] == 10 * 4 ** level + 2
    assert F.shape[0] == 20 * 4 ** level
    assert V.shape[0] - E.shape[0] + F.shape[0] == 2  # Euler characteristic of the sphere
    assert np.allclose(np.linalg.norm(V, axis=1), 1.0, atol=1e-15)
    # every edge is shared by exactly two faces, with opposite orientation
    de = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]])
    key = de[:, 0] * V.shape[0] + de[:, 1]
    assert np.unique(key).size == key.size
    rev = de[:, 1] * V.shape[0] + de[:, 0]
    assert np.all(np.isin(rev, key))
    # outward orientation
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    assert np.all(np.einsum("ij,ij->i", np.cross(b - a, c - a), a + b + c) > 0)


def test_torus_topology():
    V, F = meshes.torus_grid(16, 8)
    E = meshes.mesh_edges(F)
    assert V.shape[0] == 128 and F.shape[0] == 256
    assert V.shape[0] - E.shape[0] + F.shape[0] == 0  # torus
    deg = np.bincount(E.ravel(), minlength=V.shape[0])
    assert np.all(deg == 6)


def _flat_patch(m=9, seed=0):
    """A jittered triangulated square [0,1]^2 in the plane z = 0."""
    rng = np.random.default_rng(seed)
    g = np.linspace(0.0, 1.0, m)
    X, Y = np.meshgrid(g, g, indexing="ij")
    V = np.stack([X.ravel(), Y.ravel(), np.zeros(m * m)], axis=1)
    interior = (X.ravel() > 0) & (X.ravel() < 1) & (Y.ravel() > 0) & (Y.ravel() < 1)
    V[interior, :2] += rng.uniform(-0.2, 0.2, size=(interior.sum(), 2)) / (m - 1)
    F = []
    for i in range(m - 1):
        for j in range(m - 1):
            a, b, c, d = i * m + j, (i + 1) * m + j, (i + 1) * m + j + 1, i * m + j + 1
            F += [(a, b, c), (a, c, d)]
    return V, np.asarray(F), interior


def test_cotan_linear_precision_and_area():
    V, F, interior = _flat_patch()
    L = operators.cotan_laplacian(V, F)
    # the cotan Laplacian annihilates linear functions at interior vertices
    for f in (V[:, 0], V[:, 1], 2.0 * V[:, 0] - 3.0 * V[:, 1] + 1.0):
        assert np.abs((L @ f)[interior]).max() <= 1e-12
    # lumped masses sum to the exact area of the square
    assert abs(operators.lumped_mass(V, F).sum() - 1.0) <= 1e-14


def test_cotan_structure_on_sphere():
    V, F = meshes.icosphere(3)
    L = operators.cotan_laplacian(V, F)
    assert abs(L - L.T).max() == 0.0
    assert np.abs(L @ np.ones(V.shape[0])).max() <= 1e-12
    assert L.diagonal().min() > 0
    ev = np.linalg.eigvalsh(L.toarray())
    assert ev.min() >= -1e-10 and abs(ev[0]) <= 1e-10  # PSD, constant kernel


def test_sphere_first_eigenvalue():
    """z is an l = 1 spherical harmonic, eigenvalue l (l + 1) = 2 of the
    Laplace-Beltrami operator of the unit sphere; on the icospheres the
    discrete Rayleigh quotient z^T S z / z^T M z reproduces it to rounding,
    and M^-1 S z approaches 2 z pointwise under refinement."""
    errs = []
    for level in (2, 3, 4):
        V, F = meshes.icosphere(level)
        L = operators.cotan_laplacian(V, F)
        M = operators.lumped_mass(V, F)
        z = V[:, 2]
        assert abs(z @ (L @ z) / (z @ (M * z)) - 2.0) <= 1e-12
        errs.append(np.sqrt(np.sum(M * ((L @ z) / M - 2.0 * z) ** 2)))
    assert errs[0] > errs[1] > errs[2]


def test_sphere_area_converges_second_order():
    areas = [operators.lumped_mass(*meshes.icosphere(k)).sum() for k in (2, 3, 4, 5)]
    errs = [abs(a - 4 * np.pi) for a in areas]
    assert all(e1 > e2 for e1, e2 in zip(errs, errs[1:]))
    assert all(3.5 < e1 / e2 < 4.5 for e1, e2 in zip(errs, errs[1:]))  # O(h^2), h halves per level
    assert errs[-1] < 5e-3


def test_system_matrix_and_rhs():
    s = workloads.icosphere_system(3)
    A, M, L = s.A, s.Mdiag, s.L
    assert abs(A - (sp.diags(M) + 1e-3 * L)).max() <= 1e-18
    assert np.all(np.diff(A.indptr) > 0) and A.has_sorted_indices
    assert np.allclose(A.diagonal(), M + 1e-3 * L.diagonal())
    rng = np.random.default_rng(0)
    assert np.array_equal(s.b, M * rng.standard_normal(A.shape[0]))


def test_heat_workload_inputs():
    s = workloads.heat_system(32, 16, hot=16)
    assert s.extra["u0"].sum() == 16 and np.all(np.isin(s.extra["u0"], [0.0, 1.0]))
    assert np.array_equal(s.b, s.Mdiag * s.extra["u0"])
    assert s.extra["x_target"].shape == (512,)


def test_knn_laplacian():
    rng = np.random.default_rng(2)
    P = meshes.noisy_sphere_cloud(2000, rng)
    E, h = operators.knn_graph(P, 10)
    L = operators.knn_laplacian(P, E, h)
    assert abs(L - L.T).max() == 0.0
    assert np.abs(L @ np.ones(P.shape[0])).max() <= 1e-12
    assert L.nnz == P.shape[0] + 2 * E.shape[0]
    # every point keeps at least its own k nearest neighbours
    assert np.diff(L.indptr).min() >= 11


def test_sorted_unique_and_edges_match_numpy():
    """The generators' distinct-key helper gives np.unique's result (sorted,
    distinct), and mesh_edges the lexicographically sorted distinct edges."""
    rng = np.random.default_rng(11)
    for size, hi in ((0, 5), (1, 5), (1000, 50), (20000, 1 << 40)):
        key = rng.integers(0, hi, size=size, dtype=np.int64)
        assert np.array_equal(meshes.sorted_unique(key), np.unique(key))
    V, F = meshes.icosphere(3)
    e = np.sort(np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]]), axis=1)
    assert np.array_equal(meshes.mesh_edges(F), np.unique(e, axis=0))
