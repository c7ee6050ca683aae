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
