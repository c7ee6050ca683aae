"""Discrete operators that set up the linear systems (paper Sec. 5.2).

* cotan Laplacian S and lumped (barycentric) mass M of a triangle mesh
  (Wardetzky et al. 2007, as used for Eq. (smoothing) and Eq. (Poisson));
* a Gaussian-weighted k-nearest-neighbour graph Laplacian for point clouds,
  standing in for the robust Laplacian the paper uses there.

Sign convention: S_ij = -(cot a_ij + cot b_ij)/2 for an edge ij, S_ii = -sum_j S_ij,
so S is symmetric positive semi-definite with S 1 = 0.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .meshes import sorted_unique


def _csr_sorted(m: sp.spmatrix) -> sp.csr_matrix:
    m = sp.csr_matrix(m)
    m.sum_duplicates()
    m.sort_indices()
    return m


def cotan_laplacian(V: np.ndarray, F: np.ndarray) -> sp.csr_matrix:
    n = V.shape[0]
    rows, cols, vals = [], [], []
    for k in range(3):
        i, j, o = F[:, k], F[:, (k + 1) % 3], F[:, (k + 2) % 3]
        # angle at o, opposite edge (i, j)
        e1 = V[i] - V[o]
        e2 = V[j] - V[o]
        cot = np.einsum("ij,ij->i", e1, e2) / np.linalg.norm(np.cross(e1, e2), axis=1)
        w = -0.5 * cot
        rows += [i, j]
        cols += [j, i]
        vals += [w, w]
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals)
    off = sp.coo_matrix((v, (r, c)), shape=(n, n)).tocsr()
    off.sum_duplicates()
    diag = -np.asarray(off.sum(axis=1)).ravel()
    return _csr_sorted(off + sp.diags(diag))


def lumped_mass(V: np.ndarray, F: np.ndarray) -> np.ndarray:
    """Diagonal of the barycentric lumped mass matrix: a third of the area of
    every incident triangle."""
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    area = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)
    m = np.zeros(V.shape[0])
    for k in range(3):
        np.add.at(m, F[:, k], area / 3.0)
    return m


def edges_to_adjacency(n: int, E: np.ndarray):
    """Symmetric CSR adjacency (rowptr int64, col int32, sorted, no self loops)
    from an undirected edge list."""
    i = np.concatenate([E[:, 0], E[:, 1]])
    j = np.concatenate([E[:, 1], E[:, 0]])
    m = sp.coo_matrix((np.ones(i.size, dtype=np.int8), (i, j)), shape=(n, n)).tocsr()
    m.sum_duplicates()
    m.sort_indices()
    return m.indptr.astype(np.int64), m.indices.astype(np.int32)


def knn_graph(P: np.ndarray, k: int, workers: int = -1):
    """Union-symmetrised k-nearest-neighbour graph (self excluded).  Returns the
    undirected edge list (i < j, unique) and the mean of all n*k kNN distances."""
    from scipy.spatial import cKDTree

    tree = cKDTree(P)
    d, nb = tree.query(P, k=k + 1, workers=workers)
    d, nb = d[:, 1:], nb[:, 1:]
    n = P.shape[0]
    i = np.repeat(np.arange(n, dtype=np.int64), k)
    j = nb.reshape(-1).astype(np.int64)
    e = np.stack([np.minimum(i, j), np.maximum(i, j)], axis=1)
    e = e[e[:, 0] != e[:, 1]]
    key = sorted_unique(e[:, 0] * n + e[:, 1])
    E = np.stack([key // n, key % n], axis=1)
    return E, float(d.mean())


def knn_laplacian(P: np.ndarray, E: np.ndarray, h: float) -> sp.csr_matrix:
    """L = D - W with W_ij = exp(-|p_i - p_j|^2 / h^2) on the symmetric graph E."""
    n = P.shape[0]
    d2 = np.einsum("ij,ij->i", P[E[:, 0]] - P[E[:, 1]], P[E[:, 0]] - P[E[:, 1]])
    w = np.exp(-d2 / (h * h))
    W = sp.coo_matrix(
        (np.concatenate([w, w]), (np.concatenate([E[:, 0], E[:, 1]]), np.concatenate([E[:, 1], E[:, 0]]))),
        shape=(n, n),
    ).tocsr()
    deg = np.asarray(W.sum(axis=1)).ravel()
    return _csr_sorted(sp.diags(deg) - W)


def system_matrix(Mdiag: np.ndarray, L: sp.csr_matrix, t: float) -> sp.csr_matrix:
    """A = M + t L (M diagonal), CSR with sorted columns and explicit diagonal."""
    return _csr_sorted(sp.diags(Mdiag) + t * L)


def poisson_matrix(Mdiag: np.ndarray, L: sp.csr_matrix, eta: float) -> sp.csr_matrix:
    """A = S + eta M of Eq. (Poisson) (S = L here, M diagonal), CSR with sorted
    columns and explicit diagonal."""
    return _csr_sorted(L + sp.diags(eta * Mdiag))


def bilaplacian_matrix(Mdiag: np.ndarray, L: sp.csr_matrix, alpha: float, beta: float) -> sp.csr_matrix:
    """A = M + alpha S + beta S M^-1 S: the normal equations of the smoothing
    energy (x - y)^T M (x - y) + alpha x^T S x + beta x^T S M^-1 S x of Sec. 5.5."""
    SMS = L @ sp.diags(1.0 / Mdiag) @ L
    B = sp.diags(Mdiag) + alpha * L + beta * SMS
    # the sparse product rounds (i, j) and (j, i) in different orders: average
    # the two halves so the matrix is exactly symmetric
    return _csr_sorted(0.5 * (B + B.T))
