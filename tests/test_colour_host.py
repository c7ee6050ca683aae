"""The library's host colouring (`gmg_colour`, the colouring gmg_setup gives a
level when the caller passes none) against the oracle's, which implements the
same deterministic rules on its own: first fit in increasing row index and in
smallest-last order, eight iterated-greedy passes each, fewer colours kept.
Runs without a GPU.  Levels of 65,536 rows or more take the library's
class-parallel passes, so the 512 x 256 torus covers those too."""
import numpy as np
import pytest
import scipy.sparse as sp

import gmg_inputs as gi
import oracle


@pytest.fixture(scope="module")
def g():
    import paper_2307_04886_gb300 as g

    g.build_library()
    return g


def _cases():
    return {
        "icosphere4": lambda: gi.icosphere_system(4, stop=100),
        "torus512x256": lambda: gi.torus_system(512, 256, 1e-4, 3),
        "book_small": lambda: gi.nonmanifold_system(pages=3, n_radial=40, n_spine=60),
        "bilaplacian": lambda: gi.workloads.bilaplacian_system(),
        "cloud16k": lambda: gi.cloud_system(16384, stop=300),  # kNN pattern, random order, about 20 colours
    }


@pytest.mark.parametrize("name", list(_cases()))
def test_colour_matches_oracle_on_every_level(g, name):
    s = _cases()[name]()
    o = oracle.Oracle(s.A, s.Ps)
    big = False
    for l in range(o.nlev):
        Al, col_oracle = o.level(l)
        Al = sp.csr_matrix(Al)
        Al.sort_indices()
        col, nc = g.colour(Al)
        assert np.array_equal(col, col_oracle), (name, l)
        assert nc == int(col_oracle.max()) + 1
        big |= Al.shape[0] >= 65536
        # proper: no stored off-diagonal entry joins two rows of one colour
        C = Al.tocoo()
        off = C.row != C.col
        assert not np.any(col[C.row[off]] == col[C.col[off]])
    if name == "torus512x256":
        assert big


def _lap1d(n):
    return sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1], format="csr")


def test_colour_small_patterns(g):
    col, nc = g.colour(_lap1d(9))
    assert nc == 2 and np.array_equal(col, np.arange(9) % 2)
    col, nc = g.colour(sp.identity(5, format="csr"))  # no edges: one colour
    assert nc == 1 and not col.any()
    col, nc = g.colour(sp.csr_matrix(np.ones((4, 4))))  # a clique: every row its own colour
    assert nc == 4 and sorted(col) == [0, 1, 2, 3]
    col, nc = g.colour(sp.csr_matrix((0, 0)))
    assert nc == 0 and col.size == 0


def test_colour_rejects_bad_patterns(g):
    A = _lap1d(8).tolil()
    A[1, 6] = -0.1  # no mirror entry
    with pytest.raises(g.GMGError, match="not symmetric"):
        g.colour(A.tocsr())
    B = _lap1d(8)
    B.indices[[0, 1]] = B.indices[[1, 0]]  # row 0 unsorted
    B.has_sorted_indices = False
    with pytest.raises(g.GMGError, match="unsorted"):
        g.colour(B)
    C = _lap1d(8)
    C.indices[2] = 9  # out of range
    with pytest.raises(g.GMGError, match="out of range"):
        g.colour(C)
