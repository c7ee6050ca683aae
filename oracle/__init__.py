"""CPU FP64 oracle of the multigrid solve (Alg. 1 and Alg. 2).

TEST INFRASTRUCTURE ONLY: the tests, `__graft_entry__.smoke()` and the
CPU-baseline leg of `bench.py` load it; the product path never does.  The
arithmetic lives in gmg_oracle.c (plain C, FP64, no blocking or fusion);
this module only marshals arrays.  It shares no code with the CUDA library.

Parity pins (see tests/test_oracle_*.py): Galerkin product vs dense brute
force, symmetry and mass conservation; Cholesky vs the defining identity;
multicolour Gauss-Seidel vs the matrix-splitting form (D + L_pi)^-1 (b - U_pi x);
V-cycle symmetry (B = B^T) for the symmetric cycle, exactness with P = I, and
convergence to the dense solution; closed forms for the assembled systems
(constant mode, spherical harmonics).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gmg_oracle.c")
_LIB = os.path.join(_HERE, "_gmg_oracle.so")
_lib = None

OR_OK, OR_ERR_ARG, OR_ERR_NOT_SPD, OR_ERR_EMPTY_COL, OR_ERR_CHOL, OR_ERR_NOT_CONV = range(6)


_LIB_OMP = os.path.join(_HERE, "_gmg_oracle_omp.so")
_FLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-Wno-unknown-pragmas", "-shared", "-fPIC"]


def compile_oracle(force: bool = False) -> str:
    """The single-threaded build (the one every parity test uses)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *_FLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def compile_oracle_threaded(force: bool = False) -> str | None:
    """The same source built with -fopenmp: the row loops run on all host
    cores (OMP_NUM_THREADS to limit them).  Used only for the all-cores CPU
    baseline.  Returns None when the compiler has no OpenMP runtime."""
    if force or not os.path.exists(_LIB_OMP) or os.path.getmtime(_LIB_OMP) < os.path.getmtime(_SRC):
        tmp = _LIB_OMP + f".tmp{os.getpid()}"
        try:
            subprocess.check_call(["gcc", *_FLAGS, "-fopenmp", "-o", tmp, _SRC, "-lm"],
                                  stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (subprocess.CalledProcessError, OSError):
            return None
        os.replace(tmp, _LIB_OMP)
    return _LIB_OMP


def host_cores() -> int:
    """Cores available to this process (what the threaded build uses by default)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def compile_variant(src_text: str, out_path: str) -> str:
    """Compiles a modified copy of the oracle source (used by the tests that
    plant a mistake in the oracle to show that the pins catch it)."""
    c_path = out_path + ".c"
    with open(c_path, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", *_FLAGS, "-o", out_path, c_path, "-lm"])
    return out_path


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _load(path: str | None = None):
    global _lib
    if path is not None or _lib is None:
        lib = ctypes.CDLL(path or compile_oracle())
        V = ctypes.c_void_p
        lib.or_create.restype = ctypes.c_int
        lib.or_create.argtypes = [ctypes.c_int64, V, V, V, ctypes.c_int, V, V, V, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int, V, V]
        lib.or_destroy.argtypes = [V]
        lib.or_nlev.argtypes = [V]
        lib.or_level_dims.argtypes = [V, ctypes.c_int, V, V, V]
        lib.or_level_export.argtypes = [V, ctypes.c_int, V, V, V, V]
        lib.or_chol_export.argtypes = [V, V]
        lib.or_smooth.argtypes = [V, ctypes.c_int, V, V, ctypes.c_int, ctypes.c_int]
        lib.or_residual.argtypes = [V, ctypes.c_int, V, V, V]
        lib.or_apply.argtypes = [V, ctypes.c_int, V, V]
        lib.or_restrict.argtypes = [V, ctypes.c_int, V, V]
        lib.or_prolong_add.argtypes = [V, ctypes.c_int, V, V]
        lib.or_coarse_solve.argtypes = [V, V, V]
        lib.or_mgi.argtypes = [V, ctypes.c_int, V, V]
        lib.or_solve.restype = ctypes.c_int
        lib.or_solve.argtypes = [V, ctypes.c_int, V, V, ctypes.c_double, ctypes.c_int, V, V]
        if path is not None:
            return lib
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__(f"oracle status {code}")
        self.code = code


class Oracle:
    """The multigrid hierarchy of Alg. 1 for A (scipy CSR) and prolongations
    `Ps` (objects with n_coarse, idx [n,3] int32, w [n,3] float64)."""

    def __init__(self, A: sp.csr_matrix, Ps, nu_pre: int = 2, nu_post: int = 2, post_forward: bool = False,
                 lib_path: str | None = None, coloring=None):
        """`coloring`: None (greedy first-fit colouring on every level) or one
        entry per level, each None or an int array of colours."""
        lib = _load(lib_path)
        A = sp.csr_matrix(A)
        A.sort_indices()
        self._keep = []
        rp = np.ascontiguousarray(A.indptr, dtype=np.int64)
        ci = np.ascontiguousarray(A.indices, dtype=np.int32)
        va = _f64(A.data)
        nc = np.array([P.n_coarse for P in Ps] or [0], dtype=np.int64)
        idx = [np.ascontiguousarray(P.idx, dtype=np.int32) for P in Ps]
        w = [_f64(P.w) for P in Ps]
        self._keep += [rp, ci, va, nc] + idx + w
        pidx = (ctypes.c_void_p * max(1, len(Ps)))(*[_p(a).value for a in idx])
        pw = (ctypes.c_void_p * max(1, len(Ps)))(*[_p(a).value for a in w])
        col = None
        if coloring is not None:
            cols = [None if c is None else np.ascontiguousarray(c, dtype=np.int32) for c in coloring]
            self._keep += cols
            col = (ctypes.c_void_p * len(cols))(*[None if c is None else _p(c).value for c in cols])
        h = ctypes.c_void_p()
        st = lib.or_create(A.shape[0], _p(rp), _p(ci), _p(va), len(Ps), _p(nc), ctypes.cast(pidx, ctypes.c_void_p),
                           ctypes.cast(pw, ctypes.c_void_p), nu_pre, nu_post, int(post_forward),
                           None if col is None else ctypes.cast(col, ctypes.c_void_p), ctypes.byref(h))
        if st != OR_OK:
            raise OracleError(st)
        self._h = h
        self._lib = lib
        self.nlev = lib.or_nlev(h)
        self.dims = []
        for l in range(self.nlev):
            n, nnz, ncol = np.zeros(1, np.int64), np.zeros(1, np.int64), np.zeros(1, np.int32)
            lib.or_level_dims(h, l, _p(n), _p(nnz), _p(ncol))
            self.dims.append((int(n[0]), int(nnz[0]), int(ncol[0])))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None:
            self._lib.or_destroy(h)
            self._h = None

    def n(self, l: int = 0) -> int:
        return self.dims[l][0]

    def level(self, l: int):
        """(A_l as scipy CSR, colour of every row)."""
        n, nnz, _ = self.dims[l]
        rp, ci, va, col = np.empty(n + 1, np.int64), np.empty(nnz, np.int32), np.empty(nnz), np.empty(n, np.int32)
        self._lib.or_level_export(self._h, l, _p(rp), _p(ci), _p(va), _p(col))
        return sp.csr_matrix((va, ci, rp), shape=(n, n)), col

    def chol(self):
        n = self.dims[-1][0]
        L = np.empty((n, n))
        self._lib.or_chol_export(self._h, _p(L))
        return L

    def smooth(self, l, x, b, nsweep, descending=False):
        x = _f64(x).copy()
        self._lib.or_smooth(self._h, l, _p(x), _p(_f64(b)), nsweep, int(descending))
        return x

    def residual(self, l, x, b):
        r = np.empty(self.n(l))
        self._lib.or_residual(self._h, l, _p(_f64(x)), _p(_f64(b)), _p(r))
        return r

    def apply(self, l, x):
        y = np.empty(self.n(l))
        self._lib.or_apply(self._h, l, _p(_f64(x)), _p(y))
        return y

    def restrict(self, l, r):
        bc = np.empty(self.n(l + 1))
        self._lib.or_restrict(self._h, l, _p(_f64(r)), _p(bc))
        return bc

    def prolong_add(self, l, u, x):
        x = _f64(x).copy()
        self._lib.or_prolong_add(self._h, l, _p(_f64(u)), _p(x))
        return x

    def coarse_solve(self, b):
        x = np.empty(self.n(self.nlev - 1))
        self._lib.or_coarse_solve(self._h, _p(_f64(b)), _p(x))
        return x

    def vcycle(self, x, b, l: int = 0):
        """One MGI(x, b, l) of Alg. 2."""
        x = _f64(x).copy()
        self._lib.or_mgi(self._h, l, _p(x), _p(_f64(b)))
        return x

    def solve(self, b, x0=None, tol=1e-10, max_iter=100, pcg=False):
        """Alg. 1 (stationary) or PCG with the cycle as preconditioner.
        Returns (x, iterations, relative-residual history, converged)."""
        n = self.n(0)
        x = np.zeros(n) if x0 is None else _f64(x0).copy()
        hist = np.zeros(max_iter + 1)
        it = ctypes.c_int()
        st = self._lib.or_solve(self._h, int(pcg), _p(_f64(b)), _p(x), tol, max_iter, _p(hist), ctypes.byref(it))
        return x, it.value, hist[: it.value + 1], st == OR_OK


def adjoint_gradients(L: sp.csr_matrix, Mdiag, lam, x):
    """For x = A(t)^-1 M u0 with A(t) = M + t L and a loss with dloss/dx = g,
    lam = A^-1 g gives dloss/du0 = M lam and dloss/dt = -lam^T L x (A is
    symmetric, so the adjoint system uses the same matrix)."""
    return np.asarray(Mdiag) * lam, float(-(lam @ (L @ x)))
