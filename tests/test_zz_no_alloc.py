"""The allocation-free residual entry point (gmg_residual_norm_noalloc).

Some callers cannot allocate device memory (a host framework's pool owns it,
or an allocation would synchronise the device); this entry point serves them
with a static device scratch array instead of library allocations.  Its
result must agree with the library's regular residual entry point
(gmg_residual on the finest level, FP64) within the FP64 step tolerance of
the parity tests (1e-12, normwise and element-wise), on two calls in a row,
and repeated calls must give identical bits.  The residual and both norms
are also checked against the CPU oracle's residual (the plain row-by-row
definition r = b - A x in FP64).  This file is collected last so that a run stopping
at its first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import gmg_inputs as gi
import oracle
from parity_util import assert_close as close

pytestmark = pytest.mark.gpu


def test_noalloc_residual_matches_regular_entry_point(cuda):
    import torch

    import paper_2307_04886_gb300 as g

    lib = g.load_library()
    s = gi.icosphere_system(5)
    A = s.A
    n = A.shape[0]
    rng = np.random.default_rng(77)
    x = torch.tensor(rng.standard_normal(n), device=cuda)
    b = torch.tensor(s.b, device=cuda)
    rowptr = torch.tensor(A.indptr.astype(np.int64), device=cuda)
    col = torch.tensor(A.indices.astype(np.int32), device=cuda)
    val = torch.tensor(A.data, device=cuda)

    solver = g.Solver(A, s.Ps, precision=g.GMG_FP64)
    r_ref = solver.residual(0, x.clone(), b.clone(), torch.zeros_like(b))
    torch.cuda.synchronize()
    norms_ref = np.array([torch.linalg.norm(r_ref).item(), torch.linalg.norm(b).item()])
    r_oracle = oracle.Oracle(A, s.Ps).residual(0, x.cpu().numpy(), s.b)
    norms_oracle = np.array([np.linalg.norm(r_oracle), np.linalg.norm(s.b)])

    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    outs = []
    for _ in range(2):
        r = torch.full_like(b, np.nan)
        norms = torch.full((2,), np.nan, dtype=torch.float64, device=cuda)
        st = lib.gmg_residual_norm_noalloc(n, ctypes.c_void_p(rowptr.data_ptr()), ctypes.c_void_p(col.data_ptr()),
                                           ctypes.c_void_p(val.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                           ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(r.data_ptr()),
                                           ctypes.c_void_p(norms.data_ptr()), stream)
        assert st == g.GMG_OK, lib.gmg_last_error()
        torch.cuda.synchronize()
        rn, nn = r.cpu().numpy(), norms.cpu().numpy()
        rr = r_ref.cpu().numpy()
        close(rn, rr, 1e-12, "against gmg_residual")
        assert np.all(np.abs(nn - norms_ref) <= 1e-12 * norms_ref)
        close(rn, r_oracle, 1e-12, "against the oracle's residual")
        assert np.all(np.abs(nn - norms_oracle) <= 1e-12 * norms_oracle)
        outs.append((rn, nn))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    solver.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(cuda):
    import paper_2307_04886_gb300 as g

    lib = g.load_library()
    st = lib.gmg_residual_norm_noalloc(16777217, ctypes.c_void_p(8), ctypes.c_void_p(8), ctypes.c_void_p(8),
                                       ctypes.c_void_p(8), ctypes.c_void_p(8), ctypes.c_void_p(8),
                                       ctypes.c_void_p(8), None)
    assert st == g.GMG_ERR_TOO_LARGE
    assert b"16777216" in lib.gmg_last_error()
