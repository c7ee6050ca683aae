"""CPU pins of the two further systems of the paper (Sec. 5.2 Eq. (Poisson),
Sec. 5.5 bi-Laplacian smoothing) and of the oracle on them: the matrices
against their definitions, closed forms, and a direct sparse solve."""
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
