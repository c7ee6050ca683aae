"""CPU pins of the further systems of the paper (Sec. 5.2 Eq. (Poisson),
Sec. 5.5 bi-Laplacian smoothing, Sec. 5.4 smoothing on a non-manifold mesh)
and of the oracle on them: the matrices against their definitions, closed
forms, and a direct sparse solve."""
import numpy as np
import pytest
import scipy.sparse.linalg as sla

import gmg_inputs as gi
import oracle


@pytest.fixture(scope="module")
def poisson():
    return gi.workloads.poisson_system(96, 48)


@pytest.fixture(scope="module")
def bilap():
    return gi.workloads.bilaplacian_system(96, 48)


def test_poisson_matrix_definition(poisson):
    s = poisson
    ref = s.L.toarray() + 1e-6 * np.diag(s.Mdiag)
    assert np.allclose(s.A.toarray(), ref, rtol=0, atol=1e-15 * abs(ref).max())
    # S 1 = 0, so A 1 = eta M 1
    one = np.ones(s.n)
    assert np.abs(s.A @ one - 1e-6 * s.Mdiag).max() <= 1e-12 * abs(s.A).max()


def test_bilaplacian_matrix_definition(bilap):
    s = bilap
    Minv = np.diag(1.0 / s.Mdiag)
    S = s.L.toarray()
    ref = np.diag(s.Mdiag) + 1e-3 * S + 1e-7 * S @ Minv @ S
    assert np.allclose(s.A.toarray(), ref, rtol=0, atol=1e-13 * abs(ref).max())
    assert (s.A != s.A.T).nnz == 0  # exactly symmetric
    # a two-ring stencil: more entries per row than the one-ring Laplacian
    assert s.A.nnz > 2 * s.L.nnz


@pytest.mark.parametrize("which", ["poisson", "bilap"])
def test_constant_mode_is_solved_exactly(which, poisson, bilap):
    """S 1 = 0: for b = A 1 (eta M 1, resp. M 1) the solution is the constant 1."""
    s = poisson if which == "poisson" else bilap
    o = oracle.Oracle(s.A, s.Ps)
    b = s.A @ np.ones(s.n)
    # the Poisson right-hand side eta M 1 is tiny against the entries of A, so
    # its relative-residual floor in FP64 is near 1e-7
    x, it, _, ok = o.solve(b, tol=1e-6 if which == "poisson" else 1e-9, max_iter=100, pcg=True)
    assert ok
    assert np.abs(x - 1.0).max() <= 1e-6


@pytest.mark.parametrize("which", ["poisson", "bilap"])
def test_oracle_matches_direct_solve(which, poisson, bilap):
    s = poisson if which == "poisson" else bilap
    tol = 1e-7 if which == "poisson" else 1e-10   # the Poisson system stalls near 1e-8 in FP64
    o = oracle.Oracle(s.A, s.Ps)
    xe = sla.spsolve(s.A.tocsc(), s.b)
    x, it, _, ok = o.solve(s.b, tol=tol, max_iter=100, pcg=True)
    assert ok
    assert np.linalg.norm(x - xe) <= 1e-6 * np.linalg.norm(xe)


@pytest.fixture(scope="module")
def book():
    return gi.nonmanifold_system(3, 30, 40, stop=200)


def test_book_mesh_is_non_manifold(book):
    """Every spine edge of the book mesh borders one triangle of each of the 3
    sheets (a manifold edge borders at most two), and the other edges at most
    two."""
    from gmg_inputs import meshes

    V, F, _ = meshes.book(3, 30, 40, seed=7)
    e = np.sort(np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]]), axis=1)
    keys, counts = np.unique(e, axis=0, return_counts=True)
    spine = (keys[:, 0] < 40) & (keys[:, 1] < 40)
    assert spine.sum() == 39 and np.all(counts[spine] == 3)
    assert np.all(counts[~spine] <= 2)


def test_book_operators(book):
    """On the non-manifold mesh the cotan Laplacian (a sum of per-triangle FEM
    stiffness matrices) stays symmetric, annihilates constants and is
    positive semi-definite; the lumped mass sums to the mesh area; so
    A = M + t L is SPD and (M + t L) x = M 1 has the solution x = 1."""
    s = book
    L = s.L.toarray()
    assert np.abs(L - L.T).max() == 0.0
    assert np.abs(L @ np.ones(s.n)).max() <= 1e-12 * np.abs(L).max()
    ev = np.linalg.eigvalsh(L)
    assert ev[0] >= -1e-10 * ev[-1]
    from gmg_inputs import meshes

    V, F, _ = meshes.book(3, 30, 40, seed=7)
    area = 0.5 * np.linalg.norm(np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]]), axis=1).sum()
    assert abs(s.Mdiag.sum() - area) <= 1e-12 * area
    o = oracle.Oracle(s.A, s.Ps)
    x, it, _, ok = o.solve(s.Mdiag * np.ones(s.n), tol=1e-12)
    assert ok and np.abs(x - 1.0).max() <= 1e-9


def test_book_oracle_matches_direct_solve(book):
    s = book
    o = oracle.Oracle(s.A, s.Ps)
    assert o.nlev >= 3
    for pcg in (False, True):
        x, it, hist, ok = o.solve(s.b, tol=1e-10, pcg=pcg)
        assert ok
        xe = sla.spsolve(s.A.tocsc(), s.b)
        assert np.linalg.norm(x - xe) <= 1e-8 * np.linalg.norm(xe)
