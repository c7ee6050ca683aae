"""The C ABI: libgmg.so loads without a GPU and exports every function that
include/gmg.h declares; the binding's signature table covers them all."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gmg.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gmg_[A-Za-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import paper_2307_04886_gb300 as g

    try:
        g.build_library()
    except Exception as e:  # pragma: no cover - nvcc missing
        pytest.skip(f"cannot build libgmg: {e}")
    return g


def test_header_declares_core_calls():
    names = declared()
    for core in ("gmg_setup", "gmg_solve", "gmg_destroy", "gmg_solve_batched", "gmg_set_values"):
        assert core in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.check_output(["nm", "-D", "--defined-only", lib.LIB], text=True)
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    missing = [n for n in declared() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_covers_header(lib):
    assert sorted(lib.EXPORTED) == declared()


def test_library_loads_without_gpu(lib):
    h = lib.load_library()
    assert h.gmg_status_string(0) == b"ok"
    assert h.gmg_status_string(3) == b"empty prolongation column"
    opt = lib.gmg_options()
    import ctypes

    h.gmg_default_options(ctypes.byref(opt))
    assert (opt.precision, opt.nu_pre, opt.nu_post, opt.max_iter) == (1, 2, 2, 100)


def test_null_arguments_are_rejected_without_touching_the_device(lib):
    import ctypes

    h = lib.load_library()
    assert h.gmg_setup(None, None, 0, None, None, None, None) == lib.GMG_ERR_INVALID_ARG
    assert h.gmg_solve(None, None, None, 1e-10, 0, None, None) == lib.GMG_ERR_INVALID_ARG
    assert h.gmg_solve_batched(None, 1, None, None, 1e-10, 0, None, None) == lib.GMG_ERR_INVALID_ARG
    assert h.gmg_destroy(None) == lib.GMG_OK
    hh = ctypes.c_void_p()
    assert h.gmg_setup(ctypes.byref(hh), None, 0, None, None, None, None) == lib.GMG_ERR_INVALID_ARG
    assert b"A" in h.gmg_last_error()
    # the warnings query and the wait self-test refuse null arguments before any device work
    assert h.gmg_warnings(None, None, None) == lib.GMG_ERR_INVALID_ARG
    assert h.gmg_wait_selftest(16, None, None, None) == lib.GMG_ERR_INVALID_ARG


def test_hierarchy_checkpoint_format(lib, tmp_path):
    """load_hierarchy reads the .npz layout Solver.save_hierarchy writes
    (prolongations finest first, one colouring per level)."""
    import numpy as np

    rng = np.random.default_rng(0)
    idx0 = rng.integers(0, 5, size=(12, 3)).astype(np.int32)
    w0 = rng.random((12, 3))
    idx1 = rng.integers(0, 2, size=(5, 3)).astype(np.int32)
    w1 = rng.random((5, 3))
    cols = [rng.integers(0, 3, size=n).astype(np.int32) for n in (12, 5, 2)]
    np.savez(tmp_path / "h.npz", nlev=np.array([3]), p0_n_coarse=np.array([5]), p0_idx=idx0, p0_w=w0,
             p1_n_coarse=np.array([2]), p1_idx=idx1, p1_w=w1, colour0=cols[0], colour1=cols[1], colour2=cols[2])
    Ps, cs = lib.load_hierarchy(str(tmp_path / "h.npz"))
    assert [(p.n_fine, p.n_coarse) for p in Ps] == [(12, 5), (5, 2)]
    assert np.array_equal(Ps[0].idx, idx0) and np.array_equal(Ps[1].w, w1)
    assert len(cs) == 3 and all(np.array_equal(a, b) for a, b in zip(cs, cols))
