"""GPU parity: every step of Alg. 2, whole V-cycles and whole solves of the
CUDA library against the CPU FP64 oracle, through the C ABI.

Every comparison asserts the tolerance both normwise,
||gpu - oracle|| / ||oracle||, and element by element,
max_i |gpu_i - oracle_i| <= tol * max_i |oracle_i| (parity_util.assert_close):
  * FP64 steps and FP64 V-cycles: 1e-12 (only the summation order, the
    reciprocal diagonal and the explicit coarse inverse differ);
  * FP32 steps and FP32 V-cycles: 1e-6 (inputs rounded to FP32, about
    6e-8 relative, amplified by a few operator applications); element-wise
    the bound is scaled by parity_util.stencil_factor of the operator;
  * solves: both sides reach ||b - A x|| <= 1e-10 ||b||; the solutions agree
    to 1e-8 relative (the residual bound times the system's condition).
Integer results (Galerkin patterns, colourings) must be identical.
"""
import numpy as np
import pytest

import gmg_inputs as gi
import oracle
from parity_util import assert_close as close
from parity_util import stencil_factor

pytestmark = pytest.mark.gpu

SEED = 1234


@pytest.fixture(scope="module")
def gmg(cuda):
    import paper_2307_04886_gb300 as g

    g.load_library()
    return g


def _systems():
    return {
        "icosphere5": lambda: gi.icosphere_system(5),
        "torus256x120": lambda: gi.torus_system(256, 120, 1e-4, 7),
    }


@pytest.fixture(scope="module", params=["icosphere5", "torus256x120"])
def pair(request, gmg):
    s = _systems()[request.param]()
    o = oracle.Oracle(s.A, s.Ps)
    g = gmg.Solver(s.A, s.Ps)
    yield s, o, g
    g.close()


def _t(x):
    import torch

    return torch.tensor(np.asarray(x, dtype=np.float64), device="cuda")


def _np(t):
    return t.detach().cpu().numpy()


def test_levels_and_colourings_match(pair):
    s, o, g = pair
    assert g.nlev == o.nlev
    for l in range(o.nlev):
        Ao, co = o.level(l)
        Ag, cg = g.level(l)
        assert np.array_equal(Ao.indptr, Ag.indptr) and np.array_equal(Ao.indices, Ag.indices), f"pattern of level {l}"
        assert np.array_equal(co, cg), f"colouring of level {l}"
        # same products, same accumulation order, same mirroring: bitwise equal
        assert np.array_equal(Ag.data, Ao.data), f"values of level {l} (max diff {abs(Ag.data - Ao.data).max()})"
        d = Ag - Ag.T
        assert abs(d).max() == 0.0, "Galerkin operator must be exactly symmetric"


@pytest.mark.parametrize("fp32,tol", [(False, 1e-12), (True, 1e-6)])
def test_steps_match(pair, fp32, tol):
    s, o, g = pair
    rng = np.random.default_rng(SEED)
    for l in range(o.nlev - 1):
        n, nc = o.n(l), o.n(l + 1)
        ef = stencil_factor(o.level(l)[0]) if fp32 else 1.0
        x, b, u = rng.standard_normal(n), rng.standard_normal(n), rng.standard_normal(nc)
        for desc in (False, True):
            xo = o.smooth(l, x, b, 2, desc)
            xg = _np(g.smooth(l, _t(x), _t(b), 2, desc, fp32=fp32))
            close(xg, xo, tol, f"smooth level {l} desc={desc}", ef)
        ro = o.residual(l, x, b)
        rg = _np(g.residual(l, _t(x), _t(b), _t(np.zeros(n)), fp32=fp32))
        close(rg, ro, tol * 10, f"residual level {l}", ef)
        bo = o.restrict(l, b)
        bg = _np(g.restrict(l, _t(b), _t(np.zeros(nc)), fp32=fp32))
        close(bg, bo, tol, f"restrict level {l}")
        po = o.prolong_add(l, u, x)
        pg = _np(g.prolong_add(l, _t(u), _t(x), fp32=fp32))
        close(pg, po, tol, f"prolong level {l}")
    nl = o.n(o.nlev - 1)
    b = rng.standard_normal(nl)
    co = o.coarse_solve(b)
    cg = _np(g.coarse_solve(_t(b), _t(np.zeros(nl)), fp32=fp32))
    close(cg, co, max(tol, 1e-11), "coarse solve")


@pytest.mark.parametrize("fp32,tol", [(False, 1e-12), (True, 1e-6)])
def test_vcycle_matches(pair, fp32, tol):
    s, o, g = pair
    rng = np.random.default_rng(SEED + 1)
    x0 = rng.standard_normal(s.n)
    b = s.b
    xo = o.vcycle(x0, b)
    xg = _np(g.vcycle(_t(x0), _t(b), fp32=fp32))
    ef = stencil_factor(s.A) if fp32 else 1.0
    close(xg, xo, tol, "first V-cycle", ef)
    # a second cycle from the first one's output
    xo2 = o.vcycle(xo, b)
    xg2 = _np(g.vcycle(_t(xg), _t(b), fp32=fp32))
    close(xg2, xo2, tol, "second V-cycle", ef)


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
def test_solve_matches(gmg, precision):
    """Solves to 1e-10 in every precision mode.  The FP64 modes (the
    stationary iteration of Alg. 1 and CG preconditioned by the FP64 cycle)
    take the oracle's iteration count with the same residual history."""
    s = gi.icosphere_system(5)
    o = oracle.Oracle(s.A, s.Ps)
    xo, ito, ho, ok = o.solve(s.b, tol=1e-10, pcg=precision in (2, 3))
    assert ok
    g = gmg.Solver(s.A, s.Ps, precision=precision)
    xg, it, rr, hist, st = g.solve(_t(s.b), tol=1e-10, history=101)
    xg = _np(xg)
    true_rel = np.linalg.norm(s.b - s.A @ xg) / np.linalg.norm(s.b)
    assert true_rel <= 1e-10
    assert abs(true_rel - rr) <= 1e-12
    close(xg, xo, 1e-8, "solution")
    if precision in (0, 3):
        assert it == ito
        assert np.allclose(hist, ho, rtol=1e-6, atol=0)
    else:
        assert abs(it - ito) <= 2
    g.close()


def test_host_and_device_paths_agree(gmg):
    s = gi.icosphere_system(4)
    g = gmg.Solver(s.A, s.Ps)
    xd, itd, _, _, _ = g.solve(_t(s.b), tol=1e-10)
    xh, ith, _, _, _ = g.solve(np.asarray(s.b), tol=1e-10)
    assert itd == ith
    assert np.array_equal(_np(xd), xh)
    g.close()


def test_deterministic(gmg):
    s = gi.torus_system(128, 64, 1e-4, 3)
    g = gmg.Solver(s.A, s.Ps)
    x1 = _np(g.solve(_t(s.b), tol=1e-10)[0])
    x2 = _np(g.solve(_t(s.b), tol=1e-10)[0])
    assert np.array_equal(x1, x2)
    g2 = gmg.Solver(s.A, s.Ps)
    x3 = _np(g2.solve(_t(s.b), tol=1e-10)[0])
    assert np.array_equal(x1, x3)
    g.close()
    g2.close()


def test_zero_rhs(gmg):
    s = gi.icosphere_system(3)
    g = gmg.Solver(s.A, s.Ps)
    x, it, rr, _, st = g.solve(_t(np.zeros(s.n)), _t(np.ones(s.n)), tol=1e-10)
    assert it == 0 and st == 0
    assert float(abs(x).max()) == 0.0
    g.close()


def test_single_level_is_direct_solve(gmg):
    s = gi.icosphere_system(2)  # 162 vertices: no coarsening needed
    g = gmg.Solver(s.A, [])
    assert g.nlev == 1
    x, it, rr, _, st = g.solve(_t(s.b), tol=1e-10)
    assert it == 1 and rr <= 1e-12
    import scipy.sparse.linalg as sla

    close(_np(x), sla.spsolve(s.A.tocsc(), s.b), 1e-12, "direct solve")
    g.close()


def test_partition_of_unity_warning(gmg):
    """Barycentric prolongation weights sum to 1 (Sec. 4.4); weights that do
    not are flagged, not refused, and the solve runs as usual."""
    s = gi.icosphere_system(4)
    g = gmg.Solver(s.A, s.Ps)
    dev = max(float(np.abs(np.asarray(p.w).reshape(-1, 3).sum(1) - 1.0).max()) for p in s.Ps)
    assert g.warnings == 0 and g.p_unity_dev == pytest.approx(dev, abs=1e-15) and dev <= 1e-12
    x0, it0, _, _, _ = g.solve(_t(s.b), tol=1e-10)
    g.close()
    Ps = [gi.Prolongation(p.n_fine, p.n_coarse, p.idx, np.asarray(p.w) * 1.01) for p in s.Ps]
    g = gmg.Solver(s.A, Ps)
    assert g.warnings == gmg.GMG_WARN_P_UNITY and abs(g.p_unity_dev - 0.01) <= 1e-12
    x, it, rr, _, st = g.solve(_t(s.b), tol=1e-10)
    # a constant factor on P leaves the coarse correction P (P^T A P)^-1 P^T unchanged up to rounding
    assert st == 0 and abs(it - it0) <= 1 and rr <= 1e-10
    close(_np(x), _np(x0), 1e-8, "solution with scaled prolongation weights")
    g.close()


def test_bounded_wait_gives_up_and_reports(gmg):
    """The cluster level's wait for streamed entries is bounded: on a barrier
    that nothing arrives on it gives up within seconds, reports it, and the
    context stays usable (a solve that uses the cluster level follows)."""
    import ctypes

    lib = gmg.load_library()
    t, ms = ctypes.c_int(0), ctypes.c_double(0.0)
    assert lib.gmg_wait_selftest(4096, ctypes.byref(t), ctypes.byref(ms), None) == 0
    assert t.value == 1 and 0.0 < ms.value < 1000.0
    assert lib.gmg_wait_selftest(0, ctypes.byref(t), ctypes.byref(ms), None) == 0  # the solve kernels' limit
    assert t.value == 1 and 50.0 < ms.value < 5000.0
    s = gi.torus_system(512, 256, 1e-4, 3)
    g = gmg.Solver(s.A, s.Ps, precision=gmg.GMG_FP32_PCG)
    assert 1 in g.paths  # a level runs as a cluster level, on the bounded waits
    x, it, rr, _, st = g.solve(_t(s.b), tol=1e-10)
    assert st == 0 and rr <= 1e-10
    g.close()


def test_saved_hierarchy_gives_the_same_solver(gmg, tmp_path):
    """A hierarchy checkpoint (prolongations and colourings) reloaded as a
    caller colouring gives the same levels, colourings and solution bits."""
    s = gi.torus_system(250, 122, 1e-4, 5)
    g = gmg.Solver(s.A, s.Ps, precision=gmg.GMG_FP32_PCG)
    x1 = _np(g.solve(_t(s.b), tol=1e-10)[0])
    g.save_hierarchy(str(tmp_path / "h.npz"))
    Ps, cols = gmg.load_hierarchy(str(tmp_path / "h.npz"))
    g2 = gmg.Solver(s.A, Ps, precision=gmg.GMG_FP32_PCG, coloring=cols)
    assert g2.nlev == g.nlev and g2.dims == g.dims
    for l in range(g.nlev):
        A1, c1 = g.level(l)
        A2, c2 = g2.level(l)
        assert np.array_equal(c1, c2) and np.array_equal(A1.data, A2.data)
    x2 = _np(g2.solve(_t(s.b), tol=1e-10)[0])
    assert np.array_equal(x1, x2)
    g.close()
    g2.close()


def test_set_values_refresh(gmg):
    s = gi.icosphere_system(4)
    g = gmg.Solver(s.A, s.Ps)
    import scipy.sparse as sp

    A3 = (sp.diags(s.Mdiag) + 3e-3 * s.L).tocsr()
    A3.sort_indices()
    assert np.array_equal(A3.indices, s.A.indices)
    g.set_values(A3.data)
    o = oracle.Oracle(A3, s.Ps)
    for l in range(o.nlev):
        close(g.level(l)[0].data, o.level(l)[0].data, 1e-13, f"refreshed level {l}")
    x, it, rr, _, _ = g.solve(_t(s.b), tol=1e-10)
    assert np.linalg.norm(s.b - A3 @ _np(x)) / np.linalg.norm(s.b) <= 1e-10
    g.close()


def test_batched_matches_single(gmg):
    s = gi.icosphere_system(5)
    rng = np.random.default_rng(SEED + 2)
    for nrhs in (1, 3, 8):
        B = rng.standard_normal((s.n, nrhs)) * s.Mdiag[:, None]
        g = gmg.Solver(s.A, s.Ps)
        X, it, rr, _, st = g.solve_batched(_t(B), tol=1e-10)
        X = _np(X)
        for c in range(nrhs):
            r = np.linalg.norm(B[:, c] - s.A @ X[:, c]) / np.linalg.norm(B[:, c])
            assert r <= 1e-10
            xs = _np(g.solve(_t(B[:, c].copy()), tol=1e-10)[0])
            close(X[:, c], xs, 1e-8, f"batched column {c}")
        g.close()


@pytest.mark.slow
def test_full_size_torus(gmg):
    """The 1M-vertex torus in the launch configuration the bench times:
    FP32 V-cycle parity on the full system and a solve to 1e-10."""
    s = gi.workload("torus1m")
    o = oracle.Oracle(s.A, s.Ps)
    g = gmg.Solver(s.A, s.Ps, precision=1)
    for l in range(o.nlev):
        Ao, co = o.level(l)
        Ag, cg = g.level(l)
        assert np.array_equal(Ao.indices, Ag.indices) and np.array_equal(co, cg)
        assert np.array_equal(Ag.data, Ao.data), f"Galerkin level {l}"
    xo = o.vcycle(np.zeros(s.n), s.b)
    ef = stencil_factor(s.A)
    close(_np(g.vcycle(_t(np.zeros(s.n)), _t(s.b), fp32=True)), xo, 1e-6, "FP32 V-cycle, full size", ef)
    close(_np(g.vcycle(_t(np.zeros(s.n)), _t(s.b), fp32=False)), xo, 1e-12, "FP64 V-cycle, full size")
    rng = np.random.default_rng(SEED + 11)
    x0 = rng.standard_normal(s.n)
    xo = o.vcycle(x0, s.b)
    close(_np(g.vcycle(_t(x0), _t(s.b), fp32=True)), xo, 1e-6, "FP32 V-cycle from a random iterate, full size", ef)
    x, it, rr, _, _ = g.solve(_t(s.b), tol=1e-10)
    assert np.linalg.norm(s.b - s.A @ _np(x)) / np.linalg.norm(s.b) <= 1e-10
    g.close()


@pytest.mark.parametrize("split", [1, 2, 4, 8])
def test_fixed_warp_split_matches(gmg, split):
    """Every warps-per-row split of the smoothing sweeps gives the oracle's
    V-cycle (only the summation order of a row changes); an unsupported split
    is rejected and changes nothing."""
    s = gi.torus_system(256, 120, 1e-4, 7)
    o = oracle.Oracle(s.A, s.Ps)
    g = gmg.Solver(s.A, s.Ps)
    rng = np.random.default_rng(SEED + 5)
    x0 = rng.standard_normal(s.n)
    g.set_lanes([split] * (g.nlev - 1))
    xo = o.vcycle(x0, s.b)
    close(_np(g.vcycle(_t(x0), _t(s.b), fp32=False)), xo, 1e-12, f"FP64 cycle, split {split}")
    close(_np(g.vcycle(_t(x0), _t(s.b), fp32=True)), xo, 1e-6, f"FP32 cycle, split {split}", stencil_factor(s.A))
    with pytest.raises(gmg.GMGError):
        g.set_lanes([3] * (g.nlev - 1))
    x, _, _, _, _ = g.solve(_t(s.b), tol=1e-10)
    assert np.linalg.norm(s.b - s.A @ _np(x)) <= 1e-10 * np.linalg.norm(s.b)
    g.close()


def _dense_spd(n, seed, shift=1.0):
    """Symmetric matrix B B^T / n + shift I stored as a full CSR pattern."""
    import scipy.sparse as sp

    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, n))
    A = sp.csr_matrix(B @ B.T / n + shift * np.eye(n))
    A.sort_indices()
    return A


@pytest.mark.parametrize("n", [1, 7, 32, 33, 96, 130, 511])
def test_coarsest_inverse_sizes(gmg, n):
    """Single-level hierarchies are the coarsest direct solve alone: padded
    sizes (n not a multiple of the 32-row sweep block, one block, several)
    against a dense LU solve."""
    A = _dense_spd(n, 100 + n)
    g = gmg.Solver(A, [])
    rng = np.random.default_rng(n)
    b = rng.standard_normal(n)
    x, it, rr, _, st = g.solve(_t(b), tol=1e-10)
    assert st == 0 and it == 1
    xe = np.linalg.solve(A.toarray(), b)
    close(_np(x), xe, 1e-12 * max(1.0, np.linalg.cond(A.toarray()) / 100), f"coarsest solve n={n}")
    g.close()


def test_coarsest_not_positive_definite_is_reported(gmg):
    """A symmetric coarsest operator with a negative eigenvalue but a positive
    diagonal passes the diagonal check and must be rejected by the pivot check
    of the coarsest inverse."""
    import scipy.sparse as sp

    n = 40
    A = sp.lil_matrix((n, n))
    for i in range(n):
        A[i, i] = 1.0
    A[3, 4] = A[4, 3] = 2.0  # the 2 x 2 block [[1, 2], [2, 1]] has eigenvalue -1
    A = A.tocsr()
    A.sort_indices()
    with pytest.raises(gmg.GMGError) as e:
        gmg.Solver(A, [])
    assert e.value.status == gmg.GMG_ERR_CHOLESKY


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
def test_device_loop_matches_host_loop(gmg, precision):
    """The outer iterations run in a device-side graph loop (conditional WHILE
    node) unless per-cycle timing is on, which uses the host-driven loop: both
    give the same iterate, iteration count and residual history, bit for bit,
    including a run stopped by max_iter."""
    s = gi.torus_system(256, 120, 1e-4, 7)
    for max_iter, tol in ((100, 1e-10), (3, 1e-30)):
        g = gmg.Solver(s.A, s.Ps, precision=precision, max_iter=max_iter)
        runs = []
        for prof in (False, True):
            g.profile(prof)
            x, it, rr, hist, st = g.solve(_t(s.b), tol=tol, history=max_iter + 1, raise_on_fail=False)
            runs.append((_np(x), it, rr, np.array(hist), st))
        (x0, it0, rr0, h0, st0), (x1, it1, rr1, h1, st1) = runs
        assert (it0, st0) == (it1, st1)
        assert np.array_equal(x0, x1) and rr0 == rr1
        assert np.array_equal(h0[: it0 + 1], h1[: it1 + 1])
        if max_iter == 3:
            assert it0 == 3 and st0 == gmg.GMG_ERR_NOT_CONVERGED
        else:
            assert st0 == 0
        g.close()


def test_tail_cluster_matches_kernel_per_phase_path(gmg, monkeypatch):
    """The FP32 cycle runs its last levels as one thread-block-cluster launch
    (shared-memory copies, distributed shared-memory stores, cluster
    barriers).  With it switched off (GMG_NO_TAIL=1) every phase is its own
    kernel.  Both cycles match the oracle at the FP32 tolerance, and the
    cluster form launches fewer kernels."""
    s = gi.torus_system(256, 120, 1e-4, 7)
    o = oracle.Oracle(s.A, s.Ps)
    rng = np.random.default_rng(SEED + 9)
    x0 = rng.standard_normal(s.n)
    xo = o.vcycle(x0, s.b)
    res = {}
    for tail in (True, False):
        if tail:
            monkeypatch.delenv("GMG_NO_TAIL", raising=False)
        else:
            monkeypatch.setenv("GMG_NO_TAIL", "1")
        g = gmg.Solver(s.A, s.Ps, precision=gmg.GMG_FP32_PCG)
        assert g.nlev >= 3
        k0 = gmg.kernel_launches()
        xg = _np(g.vcycle(_t(x0), _t(s.b), fp32=True))
        res[tail] = (xg, gmg.kernel_launches() - k0)
        close(xg, xo, 1e-6, f"FP32 cycle, tail={tail}", stencil_factor(s.A))
        x, it, rr, _, st = g.solve(_t(s.b), tol=1e-10)
        assert st == 0 and np.linalg.norm(s.b - s.A @ _np(x)) <= 1e-10 * np.linalg.norm(s.b)
        g.close()
    assert res[True][1] < res[False][1]
    close(res[True][0], res[False][0], 1e-6, "tail vs per-phase kernels", stencil_factor(s.A))


@pytest.mark.parametrize("tail", [True, False])
def test_ragged_colour_slices(gmg, monkeypatch, tail):
    """A torus (250 x 122, 3 levels) on which the last 32-row slice of EVERY
    colour of every smoothed level is partial, so each colour launch ends in a
    padded slice: the steps and whole cycles match the oracle element by
    element, with the FP32 cycle's last levels in the cluster tail or as one
    kernel per phase."""
    if tail:
        monkeypatch.delenv("GMG_NO_TAIL", raising=False)
    else:
        monkeypatch.setenv("GMG_NO_TAIL", "1")
    s = gi.torus_system(250, 122, 1e-4, 11)
    o = oracle.Oracle(s.A, s.Ps)
    for l in range(o.nlev - 1):
        counts = np.bincount(o.level(l)[1])
        assert np.all(counts % 32 != 0), f"level {l}: a colour fills whole slices ({counts})"
    g = gmg.Solver(s.A, s.Ps, precision=gmg.GMG_FP32_PCG)
    rng = np.random.default_rng(SEED + 21)
    for l in range(o.nlev - 1):
        n = o.n(l)
        x, b = rng.standard_normal(n), rng.standard_normal(n)
        for fp32, tol in ((False, 1e-12), (True, 1e-6)):
            ef = stencil_factor(o.level(l)[0]) if fp32 else 1.0
            close(_np(g.smooth(l, _t(x), _t(b), 2, False, fp32=fp32)), o.smooth(l, x, b, 2, False), tol,
                  f"ragged smooth level {l} fp32={fp32}", ef)
            close(_np(g.residual(l, _t(x), _t(b), _t(np.zeros(n)), fp32=fp32)), o.residual(l, x, b), tol * 10,
                  f"ragged residual level {l} fp32={fp32}", ef)
    x0 = rng.standard_normal(s.n)
    xo = o.vcycle(x0, s.b)
    close(_np(g.vcycle(_t(x0), _t(s.b), fp32=False)), xo, 1e-12, "ragged FP64 cycle")
    close(_np(g.vcycle(_t(x0), _t(s.b), fp32=True)), xo, 1e-6, "ragged FP32 cycle", stencil_factor(s.A))
    x, it, rr, _, st = g.solve(_t(s.b), tol=1e-10)
    assert st == 0 and np.linalg.norm(s.b - s.A @ _np(x)) <= 1e-10 * np.linalg.norm(s.b)
    g.close()


@pytest.mark.parametrize("nrhs", [1, 2, 3, 8, 13, 16])
def test_batched_vcycle_matches_oracle_per_column(gmg, nrhs):
    """One FP32 multi-right-hand-side V-cycle (the SpMM-style kernels of the
    batched and many-mesh solves, column blocks of 1, 2, 4, 8 and 16 with zero
    padding for 3 and 13) against the oracle's cycle, column by column, on a
    ragged torus; a second cycle from the first one's output."""
    s = gi.torus_system(250, 122, 1e-4, 11)
    o = oracle.Oracle(s.A, s.Ps)
    g = gmg.Solver(s.A, s.Ps)
    rng = np.random.default_rng(SEED + 30 + nrhs)
    X0 = rng.standard_normal((s.n, nrhs))
    B = rng.standard_normal((s.n, nrhs)) * s.Mdiag[:, None]
    X1 = _np(g.vcycle_batched(_t(X0), _t(B)))
    X2 = _np(g.vcycle_batched(_t(X1), _t(B)))
    for c in range(nrhs):
        xo1 = o.vcycle(X0[:, c], B[:, c])
        ef = stencil_factor(s.A)
        close(X1[:, c], xo1, 1e-6, f"batched cycle column {c} of {nrhs}", ef)
        close(X2[:, c], o.vcycle(xo1, B[:, c]), 1e-6, f"second batched cycle column {c} of {nrhs}", ef)
    g.close()


def test_many_meshes_one_iteration_matches_oracle(gmg):
    """One outer iteration of the many-mesh solve (max_iter = 1) from random
    initial iterates: X1 = X0 + MGI32(0, B - A X0) per mesh and column, which
    equals the oracle's MGI(X0, B) up to the FP32 cycle's rounding (the cycle
    is affine in its iterate)."""
    systems = gi.spheres_batch(count=4, lo=800, hi=6000, nrhs=3, seed=8, stop=200)
    many = gmg.SolverMany([(s.A, s.Ps) for s in systems], max_iter=1)
    rng = np.random.default_rng(SEED + 40)
    X0 = [rng.standard_normal((s.n, 3)) for s in systems]
    Xs, its, rels, st = many.solve([_t(s.b) for s in systems], [_t(x) for x in X0], tol=1e-30,
                                   raise_on_fail=False)
    assert st == gmg.GMG_ERR_NOT_CONVERGED and all(i == 1 for i in its)
    for s, x0, X in zip(systems, X0, Xs):
        o = oracle.Oracle(s.A, s.Ps)
        Xn = _np(X)
        for c in range(3):
            close(Xn[:, c], o.vcycle(x0[:, c], s.b[:, c]), 1e-6, f"mesh n={s.n} column {c}", stencil_factor(s.A))
    many.close()


def test_pivot_reciprocal_within_one_ulp(gmg):
    """The Newton-Raphson reciprocal used for every pivot of the coarsest
    inverse against the correctly rounded division 1.0 / d: a log-spaced sweep
    over [1e-30, 1e30], values next to powers of two, the edges of the seeded
    range [2^-100, 2^101) and values beyond them (where the FP64 division
    takes over) stay within one unit in the last place."""
    import torch

    d = np.concatenate([
        np.logspace(-30, 30, 20001),
        np.ldexp(1.0, np.arange(-99, 100)) * (1 + 2.0**-52),
        np.ldexp(1.0, np.arange(-99, 100)) * (1 - 2.0**-53),
        np.random.default_rng(5).uniform(0.5, 2.0, 20000),
        np.array([1e-30, 1e30, 9.99e-31, 1.001e30, 3.0, 7.0, 1.0 / 3.0, np.pi]),
        np.array([np.ldexp(1.0, -100), np.ldexp(1.0, -100) * (1 - 2.0**-53), np.ldexp(1.0, 101) * (1 - 2.0**-53),
                  np.ldexp(1.0, 101), 1e-35, 1e35, 1e-300, 1e300, 1.7e308]),
    ])
    dd = torch.tensor(d, device="cuda")
    out = torch.empty_like(dd)
    lib = gmg.load_library()
    import ctypes

    st = lib.gmg_pivot_reciprocal(d.size, ctypes.c_void_p(dd.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == gmg.GMG_OK
    r = _np(out)
    exact = 1.0 / d
    ulps = np.abs(r - exact) / np.spacing(exact)
    assert ulps.max() <= 1.0, f"worst {ulps.max()} ulp at d = {d[ulps.argmax()]!r}"


def test_bit_conversions_match_ieee(gmg):
    """The FP64 -> FP32 (round to nearest even) and FP32 -> FP64 conversions
    that the kernels do on the bit patterns give the IEEE 754 results of the
    host's conversions, bit for bit: random bit patterns over every exponent,
    ties and near-ties at each rounding position, the edges of the normal
    float range (largest float and the overflow to infinity, smallest normal,
    subnormal results), zeros of both signs, infinities and NaN."""
    import ctypes

    import torch

    lib = gmg.load_library()
    rng = np.random.default_rng(11)
    bits = rng.integers(0, 2**63, 200000, dtype=np.uint64) | (rng.integers(0, 2, 200000, dtype=np.uint64) << np.uint64(63))
    d = bits.view(np.float64)
    # values around the float range: exponents 880..1160, mantissas with ties (bit 28 set, lower bits 0) and near-ties
    ex = rng.integers(880, 1161, 100000).astype(np.uint64)
    mant = rng.integers(0, 2**52, 100000, dtype=np.uint64)
    tie = (mant & ~np.uint64(0x1FFFFFFF)) | np.uint64(0x10000000)
    near = [tie, tie + np.uint64(1), tie - np.uint64(1), mant & ~np.uint64(0x1FFFFFFF)]
    edge = [((ex << np.uint64(52)) | m).view(np.float64) for m in near]
    f32max = float(np.finfo(np.float32).max)
    special = np.array([0.0, -0.0, np.inf, -np.inf, f32max, -f32max, np.nextafter(f32max, np.inf),
                        f32max * (1 + 2.0**-24), f32max * (1 + 2.0**-25), 2.0**-126, 2.0**-127, 2.0**-149, 2.0**-150,
                        2.0**-151, 1e-300, 1e300, 1.0, -1.0, 1.0 + 2.0**-24, 1.0 + 3 * 2.0**-24, 5e-324])
    d = np.concatenate([d, *edge, special, -special])
    dd = torch.tensor(d, device="cuda")
    out = torch.empty(d.size, dtype=torch.float32, device="cuda")
    st = lib.gmg_convert(d.size, 0, ctypes.c_void_p(dd.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == gmg.GMG_OK
    got = out.cpu().numpy()
    with np.errstate(over="ignore"):
        ref = d.astype(np.float32)
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(got), nan)
    bad = np.flatnonzero(got[~nan].view(np.uint32) != ref[~nan].view(np.uint32))
    assert bad.size == 0, f"{bad.size} narrowing mismatches, first at {d[~nan][bad[0]]!r}"
    # widening: every float exponent, random mantissas, zeros, subnormals, infinities, NaN
    fb = rng.integers(0, 2**32, 300000, dtype=np.uint64).astype(np.uint32)
    f = np.concatenate([fb.view(np.float32), np.array([0.0, -0.0, np.inf, -np.inf, 1e-45, -1e-45, 1.1754942e-38],
                                                        dtype=np.float32)])
    ff = torch.tensor(f, device="cuda")
    out64 = torch.empty(f.size, dtype=torch.float64, device="cuda")
    st = lib.gmg_convert(f.size, 1, ctypes.c_void_p(ff.data_ptr()), ctypes.c_void_p(out64.data_ptr()),
                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == gmg.GMG_OK
    got64 = out64.cpu().numpy()
    with np.errstate(invalid="ignore"):
        ref64 = f.astype(np.float64)
    nan = np.isnan(ref64)
    assert np.array_equal(np.isnan(got64), nan)
    assert np.array_equal(got64[~nan].view(np.uint64), ref64[~nan].view(np.uint64))
    assert lib.gmg_convert(4, 2, ctypes.c_void_p(dd.data_ptr()), ctypes.c_void_p(out.data_ptr()), None) == \
        gmg.GMG_ERR_INVALID_ARG


def test_cluster_level_matches_colour_launches(gmg, monkeypatch):
    """The level above the FP32 cycle's cluster tail runs as a cluster level
    (sweeps, residual, restriction in one cluster launch; prolongation and
    sweeps in another, halo copies in distributed shared memory).  Its
    arithmetic per row is that of one warp per row, so with that split the
    FP32 cycle is bitwise the one-launch-per-colour cycle; it matches the
    oracle's cycle, and its solves converge to the oracle's solution."""
    s = gi.torus_system(512, 256, 1e-4, 7)
    o = oracle.Oracle(s.A, s.Ps)
    g = gmg.Solver(s.A, s.Ps, precision=gmg.GMG_FP32_PCG)
    assert g.nlev == 4 and g.paths == [0, 1, 2, 3], g.paths
    monkeypatch.setenv("GMG_NO_CLUSTER_LEVEL", "1")
    h = gmg.Solver(s.A, s.Ps, precision=gmg.GMG_FP32_PCG)
    monkeypatch.delenv("GMG_NO_CLUSTER_LEVEL")
    assert h.paths == [0, 0, 2, 3], h.paths
    for sv in (g, h):
        sv.set_lanes([1] * (sv.nlev - 1))
    rng = np.random.default_rng(SEED + 21)
    for x0 in (np.zeros(s.n), rng.standard_normal(s.n)):
        a = _np(g.vcycle(_t(x0), _t(s.b), fp32=True))
        b = _np(h.vcycle(_t(x0), _t(s.b), fp32=True))
        assert np.array_equal(a, b), f"cluster level differs from the colour launches: {np.abs(a - b).max()}"
        close(a, o.vcycle(x0, s.b), 1e-6, "FP32 cycle with a cluster level", stencil_factor(s.A))
    x, it, rr, _, st = g.solve(_t(s.b), tol=1e-10)
    assert st == 0 and np.linalg.norm(s.b - s.A @ _np(x)) <= 1e-10 * np.linalg.norm(s.b)
    xo, _, _, _ = o.solve(s.b, tol=1e-12, pcg=True)
    close(_np(x), xo, 1e-8, "solve with a cluster level")
    # a numeric refresh re-lays the cluster level's entries
    At = s.A.copy()
    At.data = At.data * 1.5
    g.set_values(At.data)
    h.set_values(At.data)
    assert np.array_equal(_np(g.vcycle(_t(x0), _t(s.b), fp32=True)), _np(h.vcycle(_t(x0), _t(s.b), fp32=True)))
    g.close()
    h.close()


def _reverse_greedy(A):
    n = A.shape[0]
    col = -np.ones(n, np.int64)
    for i in range(n - 1, -1, -1):
        used = {col[j] for j in A.indices[A.indptr[i]:A.indptr[i + 1]] if j != i and col[j] >= 0}
        c = 0
        while c in used:
            c += 1
        col[i] = c
    return col.astype(np.int32)


def test_caller_colouring_matches_oracle_with_it(gmg):
    """gmg_setup with a caller colouring on every level (greedy first fit in
    decreasing row index, unlike the default) against the oracle built with
    the same colouring: identical colourings, bitwise Galerkin levels, FP64 and
    FP32 cycles element by element, a solve to 1e-10.  A colouring that is
    improper on a coarse level (checked after the symbolic product) is
    refused."""
    s = gi.torus_system(250, 122, 1e-4, 11)
    o0 = oracle.Oracle(s.A, s.Ps)
    given = [_reverse_greedy(o0.level(l)[0]) for l in range(o0.nlev)]
    o = oracle.Oracle(s.A, s.Ps, coloring=given)
    g = gmg.Solver(s.A, s.Ps, precision=gmg.GMG_FP32_PCG, coloring=given)
    for l in range(o.nlev):
        Ao, co = o.level(l)
        Ag, cg = g.level(l)
        assert np.array_equal(cg, given[l]) and np.array_equal(co, cg)
        assert np.array_equal(Ag.data, Ao.data)
    rng = np.random.default_rng(SEED + 50)
    x0 = rng.standard_normal(s.n)
    xo = o.vcycle(x0, s.b)
    close(_np(g.vcycle(_t(x0), _t(s.b), fp32=False)), xo, 1e-12, "FP64 cycle, caller colouring")
    close(_np(g.vcycle(_t(x0), _t(s.b), fp32=True)), xo, 1e-6, "FP32 cycle, caller colouring", stencil_factor(s.A))
    x, it, rr, _, st = g.solve(_t(s.b), tol=1e-10)
    assert st == 0 and np.linalg.norm(s.b - s.A @ _np(x)) <= 1e-10 * np.linalg.norm(s.b)
    g.close()
    bad = list(given)
    A1 = o0.level(1)[0]
    c1 = given[1].copy()
    j = next(j for j in A1.indices[A1.indptr[0]:A1.indptr[1]] if j != 0)
    c1[j] = c1[0]
    bad[1] = c1
    with pytest.raises(gmg.GMGError) as e:
        gmg.Solver(s.A, s.Ps, coloring=bad)
    assert e.value.status == gmg.GMG_ERR_INVALID_ARG


@pytest.mark.parametrize("split", [1, 2, 4, 8])
def test_batched_split_rows_match_oracle(gmg, split):
    """The multi-right-hand-side sweeps and residual with every row split over
    1, 2, 4 or 8 warps (the shapes the batched autotuner chooses from) give the
    oracle's cycle per column; the autotuner returns valid splits and a solve
    after it reaches 1e-10."""
    s = gi.torus_system(250, 122, 1e-4, 11)
    o = oracle.Oracle(s.A, s.Ps)
    g = gmg.Solver(s.A, s.Ps)
    rng = np.random.default_rng(SEED + 70 + split)
    X0 = rng.standard_normal((s.n, 5))
    B = rng.standard_normal((s.n, 5)) * s.Mdiag[:, None]
    g.set_lanes_batched(5, [split] * (g.nlev - 1))
    X1 = _np(g.vcycle_batched(_t(X0), _t(B)))
    for c in range(5):
        close(X1[:, c], o.vcycle(X0[:, c], B[:, c]), 1e-6, f"split {split} column {c}", stencil_factor(s.A))
    with pytest.raises(gmg.GMGError):
        g.set_lanes_batched(5, [3] * (g.nlev - 1))
    lanes = g.autotune_batched(5)
    assert all(v in (1, 2, 4, 8) for v in lanes)
    X, it, rr, _, st = g.solve_batched(_t(B), tol=1e-10)
    Xn = _np(X)
    assert st == 0 and max(np.linalg.norm(B - s.A @ Xn, axis=0) / np.linalg.norm(B, axis=0)) <= 1e-10
    g.close()


def test_refresh_defers_the_coarsest_inverse(gmg):
    """A numeric refresh (gmg_set_values) returns once the Galerkin values are
    checked and leaves the coarsest inverse running on its own stream; the next
    solve waits for it right before its first coarse solve.  Refreshed solves
    match the oracle built for the new values, and a refresh whose coarsest
    operator is not positive definite is reported by the solve that follows."""
    import scipy.sparse as sp

    s = gi.icosphere_system(4)
    g = gmg.Solver(s.A, s.Ps, precision=gmg.GMG_FP32_PCG)
    for t in (3e-3, 1e-2):
        At = (sp.diags(s.Mdiag) + t * s.L).tocsr()
        At.sort_indices()
        g.set_values(At.data)
        x, it, rr, _, st = g.solve(_t(s.b), tol=1e-10)
        assert st == 0 and np.linalg.norm(s.b - At @ _np(x)) <= 1e-10 * np.linalg.norm(s.b)
        xo, _, _, ok = oracle.Oracle(At, s.Ps).solve(s.b, tol=1e-12, pcg=True)
        close(_np(x), xo, 1e-8, f"solution after refresh t={t}")
    g.close()
    n = 40
    good = _dense_spd(n, 7)
    g = gmg.Solver(good, [], precision=gmg.GMG_FP64)
    bad = good.copy().tolil()
    bad[3, 4] = bad[4, 3] = 10.0 * good[3, 3]  # symmetric, positive diagonal, not positive definite
    bad = bad.tocsr()
    bad.sort_indices()
    assert np.array_equal(bad.indices, good.indices)
    g.set_values(bad.data)
    with pytest.raises(gmg.GMGError) as e:
        g.solve(_t(np.ones(n)), tol=1e-10)
    assert e.value.status == gmg.GMG_ERR_CHOLESKY
    g.close()
