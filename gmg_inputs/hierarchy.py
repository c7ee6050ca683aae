"""ctypes front of the host hierarchy builder (builder.cpp, paper Sec. 4).

`build_hierarchy` repeats one coarsening level until at most `stop` points are
left (Sec. 4.2: phi = 1/8, stop at 1000 points) and returns the prolongations
P_l as packed rows of three (int32 coarse index, float64 weight); a weight of 0
marks a padding slot whose index repeats the row's first entry.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "builder.cpp")
_LIB = os.path.join(_HERE, "_builder.so")
_lib = None


def compile_builder(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(compile_builder())
        lib.gb_build_level.restype = ctypes.c_void_p
        lib.gb_build_level.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_double, ctypes.c_int]
        lib.gb_level_sizes.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.gb_level_copy.argtypes = [ctypes.c_void_p] * 6
        lib.gb_level_free.argtypes = [ctypes.c_void_p]
        lib.gb_level_cells.argtypes = [ctypes.c_void_p] * 3
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Prolongation:
    """P_l in R^{n_fine x n_coarse}: row i holds idx[i, s], w[i, s] for s < 3."""
    n_fine: int
    n_coarse: int
    idx: np.ndarray  # int32 [n_fine, 3]
    w: np.ndarray    # float64 [n_fine, 3]
    stats: dict = field(default_factory=dict)

    def to_scipy(self):
        import scipy.sparse as sp

        m = self.w.reshape(-1) != 0
        rows = np.repeat(np.arange(self.n_fine), 3)[m]
        return sp.csr_matrix((self.w.reshape(-1)[m], (rows, self.idx.reshape(-1)[m])),
                             shape=(self.n_fine, self.n_coarse))


def build_level(X: np.ndarray, rowptr: np.ndarray, col: np.ndarray, phi: float = 1.0 / 8.0, shift: bool = True):
    lib = _load()
    X = np.ascontiguousarray(X, dtype=np.float64)
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    n = X.shape[0]
    h = lib.gb_build_level(n, _p(X), _p(rowptr), _p(col), phi, int(shift))
    nc = np.zeros(1, np.int64)
    nnz = np.zeros(1, np.int64)
    st = np.zeros(4, np.int64)
    lib.gb_level_sizes(h, _p(nc), _p(nnz), _p(st))
    nc, nnz = int(nc[0]), int(nnz[0])
    idx = np.empty((n, 3), np.int32)
    w = np.empty((n, 3), np.float64)
    Xc = np.empty((nc, 3), np.float64)
    crp = np.empty(nc + 1, np.int64)
    cci = np.empty(nnz, np.int32)
    lib.gb_level_copy(h, _p(idx), _p(w), _p(Xc), _p(crp), _p(cci))
    samples = np.empty(nc, np.int32)
    seed = np.empty(n, np.int32)
    lib.gb_level_cells(h, _p(samples), _p(seed))
    lib.gb_level_free(h)
    stats = dict(fallback=int(st[0]), repaired=int(st[1]), single=int(st[2]), seeds=int(st[3]))
    P = Prolongation(n, nc, idx, w, stats)
    P.samples, P.seed = samples, seed
    return P, Xc, crp, cci


def build_hierarchy(X, rowptr, col, phi: float = 1.0 / 8.0, stop: int = 1000, max_levels: int = 24,
                    shift: bool = True):
    """Coarsen while the current level has more than `stop` points."""
    Ps = []
    n = X.shape[0]
    while n > stop and len(Ps) < max_levels:
        P, X, rowptr, col = build_level(X, rowptr, col, phi, shift)
        if P.n_coarse >= n or P.n_coarse == 0:
            break
        Ps.append(P)
        n = P.n_coarse
    return Ps
