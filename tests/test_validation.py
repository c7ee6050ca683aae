"""Input validation of gmg_setup (host-side, before any device call, so it
runs without a GPU): every malformed system or prolongation is rejected with
its documented status and a message naming the defect.  The cases are the
degenerate inputs the method has: an empty system, a zero or negative
diagonal (Gauss-Seidel divides by it), an asymmetric A, non-finite values,
an empty column of P (the origin of the zero coarse diagonals Sec. 5 of the
paper reports), sizes that do not chain, and a coarsest level beyond the
dense-inverse limit."""
import ctypes

import numpy as np
import pytest
import scipy.sparse as sp


@pytest.fixture(scope="module")
def g():
    import paper_2307_04886_gb300 as g

    try:
        g.build_library()
    except Exception as e:  # pragma: no cover - nvcc missing
        pytest.skip(f"cannot build libgmg: {e}")
    return g


def _setup(g, A, Ps=(), colour0=None):
    """Calls gmg_setup through the C ABI (with a caller colouring of level 0
    when given); returns (status, last error)."""
    lib = g.load_library()
    A = sp.csr_matrix(A)
    rp = np.ascontiguousarray(A.indptr, dtype=np.int64)
    ci = np.ascontiguousarray(A.indices, dtype=np.int32)
    va = np.ascontiguousarray(A.data, dtype=np.float64)
    csr = g.gmg_csr(A.shape[0], rp.ctypes.data, ci.ctypes.data, va.ctypes.data)
    keep = [rp, ci, va]
    arr = (g.gmg_prolong * max(1, len(Ps)))()
    for l, (nf, nc, idx, w) in enumerate(Ps):
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        w = np.ascontiguousarray(w, dtype=np.float64)
        keep += [idx, w]
        arr[l] = g.gmg_prolong(nf, nc, idx.ctypes.data, w.ctypes.data)
    coloring = None
    if colour0 is not None:
        c0 = np.ascontiguousarray(colour0, dtype=np.int32)
        keep.append(c0)
        coloring = (ctypes.c_void_p * (len(Ps) + 1))(c0.ctypes.data)
    h = ctypes.c_void_p()
    st = lib.gmg_setup(ctypes.byref(h), ctypes.byref(csr), len(Ps), arr, coloring, None, None)
    assert not h.value  # nothing is handed out on failure
    return st, lib.gmg_last_error().decode()


def _lap1d(n, shift=1.0):
    return sp.diags([-np.ones(n - 1), (2.0 + shift) * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tocsr()


def _pair_p(n):
    """P merging rows 2k, 2k+1 into coarse point k (weights 1)."""
    nc = (n + 1) // 2
    idx = np.zeros((n, 3), np.int32)
    w = np.zeros((n, 3))
    idx[:, 0] = np.arange(n) // 2
    w[:, 0] = 1.0
    return n, nc, idx, w


def test_empty_system(g):
    st, msg = _setup(g, sp.csr_matrix((0, 0)))
    assert st == g.GMG_ERR_INVALID_ARG and "n <= 0" in msg


def test_zero_and_negative_diagonal(g):
    A = _lap1d(8).tolil()
    A[3, 3] = 0.0
    st, msg = _setup(g, A.tocsr())
    assert st == g.GMG_ERR_NOT_SPD and "row 3" in msg
    A = _lap1d(8).tolil()
    A[5, 5] = -1.0
    st, msg = _setup(g, A.tocsr())
    assert st == g.GMG_ERR_NOT_SPD and "row 5" in msg


def test_missing_diagonal(g):
    A = sp.csr_matrix(np.array([[2.0, 1.0], [1.0, 0.0]]))
    A.eliminate_zeros()
    st, msg = _setup(g, A)
    assert st == g.GMG_ERR_NOT_SPD and "missing diagonal" in msg


def test_asymmetric(g):
    A = _lap1d(8).tolil()
    A[2, 3] = -0.5
    st, msg = _setup(g, A.tocsr())
    assert st == g.GMG_ERR_NOT_SPD and "not symmetric" in msg


def test_asymmetric_pattern(g):
    # an entry without its mirror, early and late in the row order
    for i, j in ((1, 6), (6, 1), (0, 7)):
        A = _lap1d(8).tolil()
        A[i, j] = -0.1
        st, msg = _setup(g, A.tocsr())
        assert st == g.GMG_ERR_NOT_SPD and "not symmetric" in msg, (i, j, msg)


def test_non_finite_values(g):
    A = _lap1d(8).tolil()
    A[4, 4] = np.nan
    st, _ = _setup(g, A.tocsr())
    assert st == g.GMG_ERR_NONFINITE
    nf, nc, idx, w = _pair_p(8)
    w[6, 0] = np.inf
    st, msg = _setup(g, _lap1d(8), [(nf, nc, idx, w)])
    assert st == g.GMG_ERR_NONFINITE and "P[0]" in msg


def test_empty_prolongation_column(g):
    nf, nc, idx, w = _pair_p(8)
    idx[2:4, 0] = 0  # coarse point 1 loses both fine rows
    st, msg = _setup(g, _lap1d(8), [(nf, nc, idx, w)])
    assert st == g.GMG_ERR_EMPTY_P_COLUMN and "coarse point 1" in msg


def test_prolongation_index_out_of_range_and_sizes(g):
    nf, nc, idx, w = _pair_p(8)
    idx[7, 0] = nc
    st, msg = _setup(g, _lap1d(8), [(nf, nc, idx, w)])
    assert st == g.GMG_ERR_INVALID_ARG and "out of range" in msg
    nf, nc, idx, w = _pair_p(8)
    st, msg = _setup(g, _lap1d(8), [(nf + 1, nc, np.zeros((9, 3), np.int32), np.ones((9, 3)))])
    assert st == g.GMG_ERR_INVALID_ARG and "chain" in msg


def test_unsorted_or_repeated_columns(g):
    A = _lap1d(6)
    A.indices[[0, 1]] = A.indices[[1, 0]]  # swap the first row's two columns
    st, msg = _setup(g, A)
    assert st == g.GMG_ERR_INVALID_ARG and "row 0" in msg


def test_coarsest_level_above_the_dense_limit(g):
    """A single-level hierarchy of 8,193 rows would need a dense inverse beyond
    the 8,192-row limit of the coarsest level."""
    st, msg = _setup(g, _lap1d(8193))
    assert st == g.GMG_ERR_TOO_LARGE and "8192" in msg


def test_improper_caller_colouring_rejected(g):
    """A caller colouring of level 0 in which two adjacent rows share a colour
    (their Gauss-Seidel updates would race) or a colour lies outside [0, n)
    is rejected before any device work."""
    n = 10
    A = _lap1d(n)
    even_odd = np.arange(n) % 2  # proper for the path graph
    bad = even_odd.copy()
    bad[4] = bad[3]  # rows 3 and 4 are adjacent
    st, msg = _setup(g, A, colour0=bad)
    assert st == g.GMG_ERR_INVALID_ARG and "share colour" in msg
    neg = even_odd.copy()
    neg[2] = -1
    st, msg = _setup(g, A, colour0=neg)
    assert st == g.GMG_ERR_INVALID_ARG and "outside" in msg
