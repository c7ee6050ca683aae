"""Pins of the CPU oracle (oracle/gmg_oracle.c) against facts fixed by the
mathematics or by independent routines, chosen so that a plausible mistake
(a dropped term, a wrong sign or index, a transposed operand, the wrong
iterate in the coarse correction, the wrong sweep order) fails one of them.

  Galerkin product  dense P^T A P (numpy), exact symmetry, constant mode
  Cholesky          L L^T = A, LAPACK's factor, solve residual
  colouring         proper, complete (first fit: every smaller colour among the
                    neighbours), never more colours than plain first fit
  Gauss-Seidel      matrix-splitting form (D + L_pi)^-1 (b - U_pi x)
  transfers         b - A x, P^T r, x + P u with scipy sparse products
  V-cycle           P = I is exact in one cycle; MGI(x, b) = x + B (b - A x)
                    with B symmetric for the symmetric cycle and not for the
                    forward-forward cycle; rho(I - B A) < 1 and it matches
                    the observed rate; solutions match sparse direct solves
  closed forms      constant vector (L 1 = 0) and the l = 1 harmonic
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import gmg_inputs as gi
import oracle
from gmg_inputs import Prolongation

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def ico4():
    s = gi.icosphere_system(4, stop=100)  # 2562 -> 402 -> about 60 rows
    return s, oracle.Oracle(s.A, s.Ps)


@pytest.fixture(scope="module")
def torus_small():
    s = gi.torus_system(64, 30, 1e-4, 11, stop=60)  # ragged sizes, three or more levels
    return s, oracle.Oracle(s.A, s.Ps)


def _dense_galerkin(A, P):
    Pd = P.to_scipy().toarray()
    return Pd.T @ A.toarray() @ Pd


@pytest.mark.parametrize("fx", ["ico4", "torus_small"])
def test_galerkin_matches_dense_product(fx, request):
    s, o = request.getfixturevalue(fx)
    assert o.nlev == len(s.Ps) + 1 >= 3
    for l in range(o.nlev - 1):
        Al, _ = o.level(l)
        Ac, _ = o.level(l + 1)
        D = _dense_galerkin(Al, s.Ps[l])
        assert np.abs(Ac.toarray() - D).max() <= 1e-14 * np.abs(D).max()
        nzD = np.abs(D) > 0
        # entries of the product well above its rounding level are stored non-zero
        big = np.abs(D) > 1e-12 * np.abs(D).max()
        assert np.all(Ac.toarray()[big] != 0), "a clearly non-zero product entry is zero in the Galerkin operator"
        pattern = np.zeros(D.shape, bool)
        pattern[np.repeat(np.arange(Ac.shape[0]), np.diff(Ac.indptr)), Ac.indices] = True
        assert np.all(pattern[nzD]), "a non-zero of P^T A P is missing from the Galerkin pattern"


@pytest.mark.parametrize("fx", ["ico4", "torus_small"])
def test_galerkin_symmetry_and_mass(fx, request):
    s, o = request.getfixturevalue(fx)
    for l in range(1, o.nlev):
        Ac, _ = o.level(l)
        assert abs(Ac - Ac.T).max() == 0.0, "mirroring must give exact symmetry"
        Af, _ = o.level(l - 1)
        one_f, one_c = np.ones(Af.shape[0]), np.ones(Ac.shape[0])
        # P 1 = 1  =>  1^T A_{l+1} 1 = 1^T A_l 1
        assert abs(one_c @ (Ac @ one_c) - one_f @ (Af @ one_f)) <= 1e-12 * abs(one_f @ (Af @ one_f))


def test_galerkin_preserves_the_laplacian_kernel():
    """With A = L + eps I the coarse operators satisfy A_{l+1} 1 = eps P^T 1
    (L 1 = 0 and P 1 = 1): a sign or transpose slip in the product breaks it."""
    s = gi.icosphere_system(4, stop=100)
    eps = 1e-3
    A = (s.L + eps * sp.identity(s.n)).tocsr()
    A.sort_indices()
    o = oracle.Oracle(A, s.Ps)
    for l in range(o.nlev - 1):
        Al, _ = o.level(l)
        Ac, _ = o.level(l + 1)
        lhs = Ac @ np.ones(Ac.shape[0])
        P = s.Ps[l].to_scipy()
        rhs = P.T @ (Al @ np.ones(Al.shape[0]))
        assert np.abs(lhs - rhs).max() <= 1e-12 * np.abs(Ac).max()
        if l == 0:
            assert np.abs(lhs - eps * (P.T @ np.ones(P.shape[0]))).max() <= 1e-12 * np.abs(Ac).max()


def test_cholesky_of_coarsest(ico4):
    s, o = ico4
    C, _ = o.level(o.nlev - 1)
    Cd = C.toarray()
    L = o.chol()
    assert np.allclose(np.triu(L, 1), 0.0)
    assert np.abs(L @ L.T - Cd).max() <= 1e-14 * np.abs(Cd).max()
    assert np.abs(L - np.linalg.cholesky(Cd)).max() <= 1e-12 * np.abs(L).max()
    b = np.random.default_rng(3).standard_normal(Cd.shape[0])
    x = o.coarse_solve(b)
    assert np.linalg.norm(Cd @ x - b) <= 1e-13 * np.linalg.norm(b)


def _first_fit_count(A):
    """Colours of the textbook greedy colouring in increasing row index."""
    n = A.shape[0]
    col = -np.ones(n, np.int64)
    for i in range(n):
        used = {col[j] for j in A.indices[A.indptr[i]:A.indptr[i + 1]] if j != i and col[j] >= 0}
        c = 0
        while c in used:
            c += 1
        col[i] = c
    return int(col.max()) + 1


@pytest.mark.parametrize("fx", ["ico4", "torus_small"])
def test_colouring(fx, request):
    """Every level's colouring is proper (rows of a colour are independent, so
    the in-place multicolour sweep is a Gauss-Seidel sweep), complete (it is
    the output of a first-fit pass: each row sees every smaller colour among
    its neighbours), uses colours 0..C-1, and has no more colours than plain
    first fit in increasing row index."""
    s, o = request.getfixturevalue(fx)
    fewer = 0
    for l in range(o.nlev):
        A, col = o.level(l)
        rows = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
        off = rows != A.indices
        assert np.all(col[rows[off]] != col[A.indices[off]]), "adjacent rows share a colour"
        for i in range(A.shape[0]):
            nb = A.indices[A.indptr[i]:A.indptr[i + 1]]
            assert set(range(col[i])) <= set(col[nb[nb != i]].tolist()), f"row {i} of level {l} is not first fit"
        assert set(np.unique(col).tolist()) == set(range(o.dims[l][2]))
        ff = _first_fit_count(A)
        assert o.dims[l][2] <= ff
        fewer += o.dims[l][2] < ff
    assert fewer >= 1, "the iterated colouring should beat plain first fit somewhere"


def _gs_splitting(A, col, x, b, descending):
    """One multicolour sweep in matrix form: with rows ordered by colour
    (ascending, or descending), x_new = (D + L)^-1 (b - U x)."""
    n = A.shape[0]
    key = -col if descending else col
    pi = np.lexsort((np.arange(n), key))
    Ap = A.toarray()[np.ix_(pi, pi)]
    DL, U = np.tril(Ap), np.triu(Ap, 1)
    xp = sla.solve_triangular(DL, b[pi] - U @ x[pi], lower=True)
    out = np.empty(n)
    out[pi] = xp
    return out


@pytest.mark.parametrize("descending", [False, True])
def test_gauss_seidel_is_the_splitting(ico4, descending):
    s, o = ico4
    rng = np.random.default_rng(5)
    for l in range(o.nlev - 1):
        A, col = o.level(l)
        x, b = rng.standard_normal(A.shape[0]), rng.standard_normal(A.shape[0])
        got = o.smooth(l, x, b, 1, descending)
        ref = _gs_splitting(A, col, x, b, descending)
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
        two = o.smooth(l, x, b, 2, descending)
        assert np.linalg.norm(two - _gs_splitting(A, col, ref, b, descending)) <= 1e-12 * np.linalg.norm(ref)


def test_transfer_and_residual(ico4):
    s, o = ico4
    rng = np.random.default_rng(6)
    for l in range(o.nlev - 1):
        A, _ = o.level(l)
        P = s.Ps[l].to_scipy()
        x, b = rng.standard_normal(A.shape[0]), rng.standard_normal(A.shape[0])
        u = rng.standard_normal(P.shape[1])
        assert np.linalg.norm(o.residual(l, x, b) - (b - A @ x)) <= 1e-13 * np.linalg.norm(b - A @ x)
        assert np.linalg.norm(o.restrict(l, b) - P.T @ b) <= 1e-13 * np.linalg.norm(P.T @ b)
        assert np.linalg.norm(o.prolong_add(l, u, x) - (x + P @ u)) <= 1e-13 * np.linalg.norm(x + P @ u)


def test_identity_prolongation_is_exact_in_one_cycle():
    s = gi.icosphere_system(2)
    n = s.n
    idx = np.repeat(np.arange(n, dtype=np.int32)[:, None], 3, axis=1)
    w = np.zeros((n, 3))
    w[:, 0] = 1.0
    o = oracle.Oracle(s.A, [Prolongation(n, n, idx, w)])
    x = o.vcycle(np.random.default_rng(1).standard_normal(n), s.b)
    xs = spla.spsolve(s.A.tocsc(), s.b)
    assert np.linalg.norm(x - xs) <= 1e-12 * np.linalg.norm(xs)


def _cycle_matrix(o, n):
    """B with MGI(0, b) = B b, column by column."""
    B = np.empty((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        B[:, j] = o.vcycle(np.zeros(n), e)
    return B


def test_vcycle_is_affine_symmetric_and_contracting():
    s = gi.icosphere_system(3, stop=100)  # 642 -> about 100 -> about 15 rows
    n = s.n
    o = oracle.Oracle(s.A, s.Ps)
    assert o.nlev == 3
    B = _cycle_matrix(o, n)
    # the symmetric cycle (colours ascending before, descending after) gives B = B^T
    assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
    # MGI(x, b) = x + B (b - A x): the post-relaxation starts from y + P u
    rng = np.random.default_rng(2)
    x = rng.standard_normal(n)
    lhs = o.vcycle(x, s.b)
    rhs = x + B @ (s.b - s.A @ x)
    assert np.linalg.norm(lhs - rhs) <= 1e-11 * np.linalg.norm(rhs)
    # contraction: the error propagator I - B A has spectral radius < 1, and the
    # stationary iteration converges at that rate
    E = np.eye(n) - B @ s.A.toarray()
    rho = np.abs(np.linalg.eigvals(E)).max()
    assert rho < 0.5
    _, it, hist, ok = o.solve(s.b, tol=1e-12, max_iter=200)
    assert ok
    observed = (hist[-1] / hist[-4]) ** (1.0 / 3.0)
    assert observed <= 1.5 * rho + 1e-3
    # the forward-forward cycle is not symmetric
    of = oracle.Oracle(s.A, s.Ps, post_forward=True)
    Bf = _cycle_matrix(of, n)
    assert np.abs(Bf - Bf.T).max() > 1e-6 * np.abs(Bf).max()


@pytest.mark.parametrize("pcg", [False, True])
def test_solve_matches_direct_solution(ico4, pcg):
    s, o = ico4
    x, it, hist, ok = o.solve(s.b, tol=1e-10, pcg=pcg)
    assert ok and hist[-1] <= 1e-10
    assert abs(np.linalg.norm(s.b - s.A @ x) / np.linalg.norm(s.b) - hist[-1]) <= 1e-13
    xs = spla.spsolve(s.A.tocsc(), s.b)
    assert np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs)
    if pcg:
        # CG minimises the A-norm of the error over the Krylov space that holds
        # the stationary iterates of Alg. 1 (the symmetric cycle is an SPD
        # preconditioner), so after as many iterations its error is no larger
        xp, _, _, _ = o.solve(s.b, tol=0.0, max_iter=it, pcg=False)

        def anorm(e):
            return float(np.sqrt(e @ (s.A @ e)))

        assert anorm(x - xs) <= anorm(xp - xs) * (1 + 1e-6)
    else:
        # the stationary cycle iteration reduces the residual at every step
        assert np.all(np.diff(hist[1:]) < 0)


def test_zero_rhs_and_initial_guess(ico4):
    s, o = ico4
    x, it, hist, ok = o.solve(np.zeros(s.n), x0=np.ones(s.n))
    assert ok and it == 0 and not x.any()
    xs = spla.spsolve(s.A.tocsc(), s.b)
    x, it, hist, ok = o.solve(s.b, x0=xs, tol=1e-10)
    assert it == 1 and hist[0] <= 1e-12  # repeat-until: one cycle even from the solution


def test_closed_form_constant_mode():
    """(M + t L) 1 = M 1 since L 1 = 0: the solution for b = M 1 is 1."""
    s = gi.icosphere_system(4, t=1e-1)
    o = oracle.Oracle(s.A, s.Ps)
    x, it, hist, ok = o.solve(s.Mdiag * np.ones(s.n), tol=1e-12)
    assert ok and np.abs(x - 1.0).max() <= 1e-10


def test_closed_form_first_harmonic():
    """b = M z with z an l = 1 harmonic: x = (M + t L)^-1 M z approaches
    z / (1 + 2 t) as the sphere is refined."""
    errs = []
    for level in (3, 4, 5):
        s = gi.icosphere_system(level, t=1.0)
        V, _ = gi.meshes.icosphere(level)
        z = V[:, 2]
        o = oracle.Oracle(s.A, s.Ps)
        x, it, hist, ok = o.solve(s.Mdiag * z, tol=1e-12)
        assert ok
        errs.append(np.linalg.norm(x - z / 3.0) / np.linalg.norm(z / 3.0))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 2e-3


def test_iteration_counts_in_the_paper_band():
    """Iterations to 1e-4 for data smoothing on the synthetic meshes fall in
    the range the paper reports for its manifold meshes (plausibility)."""
    rows = [ln.split("\t") for ln in open(os.path.join(HERE, "golden", "paper_smoothing_iterations.txt"))
            if not ln.startswith("#")]
    its = np.array([int(r[2]) for r in rows])
    assert its.size == 50 and its.min() == 2 and its.max() == 36
    for s in (gi.icosphere_system(5), gi.torus_system(256, 96, 1e-4, 1)):
        o = oracle.Oracle(s.A, s.Ps)
        _, it, hist, ok = o.solve(s.b, tol=1e-4)
        assert ok and its.min() <= it <= its.max()


def _reverse_greedy(A):
    """A proper colouring different from the library default: greedy first fit
    in DECREASING row index."""
    n = A.shape[0]
    col = -np.ones(n, np.int64)
    for i in range(n - 1, -1, -1):
        used = {col[j] for j in A.indices[A.indptr[i]:A.indptr[i + 1]] if j != i and col[j] >= 0}
        c = 0
        while c in used:
            c += 1
        col[i] = c
    return col.astype(np.int32)


def test_given_colouring(ico4):
    """A caller's colouring replaces the greedy one level by level: the levels
    keep their Galerkin operators, report the given colours, and the sweeps
    are the Gauss-Seidel splitting in that colour order; an improper colouring
    (two adjacent rows alike) is refused."""
    s, o = ico4
    given = [_reverse_greedy(o.level(l)[0]) for l in range(o.nlev)]
    assert any(not np.array_equal(g, o.level(l)[1]) for l, g in enumerate(given))
    o2 = oracle.Oracle(s.A, s.Ps, coloring=given)
    rng = np.random.default_rng(15)
    for l in range(o.nlev):
        A1, _ = o.level(l)
        A2, c2 = o2.level(l)
        assert np.array_equal(A1.data, A2.data) and np.array_equal(c2, given[l])
        if l < o.nlev - 1:
            x, b = rng.standard_normal(A2.shape[0]), rng.standard_normal(A2.shape[0])
            ref = _gs_splitting(A2, c2, x, b, False)
            assert np.linalg.norm(o2.smooth(l, x, b, 1, False) - ref) <= 1e-12 * np.linalg.norm(ref)
    x, _, _, ok = o2.solve(s.b, tol=1e-10)
    assert ok and np.linalg.norm(s.b - s.A @ x) <= 1e-10 * np.linalg.norm(s.b)
    bad = [None] * o.nlev
    c0 = o.level(0)[1].copy()
    A0 = o.level(0)[0]
    i = 0
    j = next(j for j in A0.indices[A0.indptr[i]:A0.indptr[i + 1]] if j != i)
    c0[j] = c0[i]
    bad[0] = c0
    with pytest.raises(oracle.OracleError):
        oracle.Oracle(s.A, s.Ps, coloring=bad)
