"""The all-cores build of the oracle (the same C source with -fopenmp) gives
the single-threaded build's results bit for bit wherever its parallel loops
run over independent rows (Galerkin levels, Cholesky factor, Gauss-Seidel
sweeps, V-cycles); only the dot products of the outer iteration may sum in
another order, so solves agree to rounding.  It times the all-cores CPU
baseline, so it must compute the same method."""
import numpy as np
import pytest

import gmg_inputs as gi
import oracle


@pytest.fixture(scope="module")
def pair():
    path = oracle.compile_oracle_threaded()
    if path is None:
        pytest.skip("no OpenMP runtime in this compiler")
    s = gi.torus_system(96, 40, 1e-4, 3, stop=200)
    return s, oracle.Oracle(s.A, s.Ps), oracle.Oracle(s.A, s.Ps, lib_path=path)


def test_levels_and_factor_identical(pair):
    s, o1, o2 = pair
    assert o1.nlev == o2.nlev >= 3
    for l in range(o1.nlev):
        A1, c1 = o1.level(l)
        A2, c2 = o2.level(l)
        assert np.array_equal(A1.indptr, A2.indptr) and np.array_equal(A1.indices, A2.indices)
        assert np.array_equal(A1.data, A2.data) and np.array_equal(c1, c2)
    assert np.array_equal(o1.chol(), o2.chol())


def test_cycle_identical_and_solve_close(pair):
    s, o1, o2 = pair
    rng = np.random.default_rng(3)
    x0 = rng.standard_normal(s.n)
    assert np.array_equal(o1.vcycle(x0, s.b), o2.vcycle(x0, s.b))
    x1, it1, _, ok1 = o1.solve(s.b, tol=1e-10, pcg=True)
    x2, it2, _, ok2 = o2.solve(s.b, tol=1e-10, pcg=True)
    assert ok1 and ok2 and abs(it1 - it2) <= 1
    assert np.linalg.norm(x1 - x2) <= 1e-9 * np.linalg.norm(x1)
