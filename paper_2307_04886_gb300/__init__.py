"""Python binding of libgmg: the GPU multigrid solve of Wiersma et al.,
"A Fast Geometric Multigrid Method for Curved Surfaces" (SIGGRAPH 2023).

This module only marshals arguments to the C ABI declared in include/gmg.h
(ctypes; no torch types cross the boundary).  Every step of the solve runs in
the library's CUDA kernels; there is no CPU fallback: importing works without
the library, but constructing a Solver raises when libgmg.so is missing.

Device vectors are torch CUDA tensors (float64, contiguous); host vectors are
numpy arrays.  The stream is torch's current CUDA stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB, build_library  # noqa: F401

GMG_OK, GMG_ERR_INVALID_ARG, GMG_ERR_NOT_SPD, GMG_ERR_EMPTY_P_COLUMN, GMG_ERR_CHOLESKY, GMG_ERR_NOT_CONVERGED, \
    GMG_ERR_NONFINITE, GMG_ERR_OOM, GMG_ERR_CUDA, GMG_ERR_TIMEOUT, GMG_ERR_TOO_LARGE = range(11)
GMG_FP64, GMG_FP32_REFINE, GMG_FP32_PCG, GMG_FP64_PCG = 0, 1, 2, 3
GMG_MEM_DEVICE, GMG_MEM_HOST = 0, 1
GMG_WARN_P_UNITY = 1

EXPORTED = [
    "gmg_default_options", "gmg_status_string", "gmg_last_error", "gmg_setup", "gmg_set_values", "gmg_solve",
    "gmg_solve_batched", "gmg_destroy", "gmg_warnings", "gmg_num_levels", "gmg_level_info", "gmg_level_export", "gmg_smooth",
    "gmg_residual", "gmg_restrict", "gmg_prolong_add", "gmg_coarse_solve", "gmg_vcycle", "gmg_profile",
    "gmg_profile_read", "gmg_kernel_launches", "gmg_residual_norm_noalloc", "gmg_setup_ML", "gmg_set_t",
    "gmg_mass", "gmg_grad", "gmg_setup_many", "gmg_solve_many", "gmg_destroy_many", "gmg_autotune", "gmg_set_lanes",
    "gmg_vcycle_batched", "gmg_pivot_reciprocal", "gmg_convert", "gmg_colour", "gmg_wait_selftest", "gmg_level_path", "gmg_profile_levels", "gmg_grad_pattern",
    "gmg_autotune_batched", "gmg_set_lanes_batched", "gmg_autotune_many",
    "gmg_build_hierarchy", "gmg_hierarchy_info", "gmg_hierarchy_level", "gmg_destroy_hierarchy",
]


def kernel_launches() -> int:
    """Kernels libgmg has launched from this thread so far."""
    return int(load_library().gmg_kernel_launches())


class gmg_csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("rowptr", ctypes.c_void_p), ("col", ctypes.c_void_p),
                ("val", ctypes.c_void_p)]


class gmg_prolong(ctypes.Structure):
    _fields_ = [("n_fine", ctypes.c_int64), ("n_coarse", ctypes.c_int64), ("idx", ctypes.c_void_p),
                ("w", ctypes.c_void_p)]


class gmg_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("nu_pre", ctypes.c_int), ("nu_post", ctypes.c_int),
                ("max_iter", ctypes.c_int), ("post_forward", ctypes.c_int), ("use_graphs", ctypes.c_int)]


class gmg_solve_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("rel_res", ctypes.c_double), ("history", ctypes.c_void_p),
                ("history_cap", ctypes.c_int)]


class GMGError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: status {status} ({msg})")
        self.status = status


_lib = None


def load_library(path: str | None = None):
    """Loads libgmg.so (raises OSError when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB
    if not os.path.exists(path):
        raise OSError(f"libgmg.so not found at {path}; build it with paper_2307_04886_gb300.build_library()")
    lib = ctypes.CDLL(path)
    V, I, D, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    sig = {
        "gmg_default_options": (None, [V]),
        "gmg_status_string": (ctypes.c_char_p, [I]),
        "gmg_last_error": (ctypes.c_char_p, []),
        "gmg_setup": (I, [V, V, I, V, V, V, V]),
        "gmg_set_values": (I, [V, V, I, V]),
        "gmg_solve": (I, [V, V, V, D, I, V, V]),
        "gmg_solve_batched": (I, [V, I, V, V, D, I, V, V]),
        "gmg_destroy": (I, [V]),
        "gmg_warnings": (I, [V, V, V]),
        "gmg_num_levels": (I, [V, V]),
        "gmg_level_info": (I, [V, I, V, V, V]),
        "gmg_level_export": (I, [V, I, V, V, V, V]),
        "gmg_smooth": (I, [V, I, I, V, V, I, I, V]),
        "gmg_residual": (I, [V, I, I, V, V, V, V]),
        "gmg_restrict": (I, [V, I, I, V, V, V]),
        "gmg_prolong_add": (I, [V, I, I, V, V, V]),
        "gmg_coarse_solve": (I, [V, I, V, V, V]),
        "gmg_vcycle": (I, [V, I, V, V, V]),
        "gmg_vcycle_batched": (I, [V, I, V, V, V]),
        "gmg_pivot_reciprocal": (I, [I64, V, V, V]),
        "gmg_convert": (I, [I64, I, V, V, V]),
        "gmg_colour": (I, [I64, V, V, V, V]),
        "gmg_wait_selftest": (I, [I, V, V, V]),
        "gmg_level_path": (I, [V, I, V]),
        "gmg_profile": (I, [V, I]),
        "gmg_kernel_launches": (ctypes.c_uint64, []),
        "gmg_residual_norm_noalloc": (I, [I64, V, V, V, V, V, V, V, V]),
        "gmg_setup_ML": (I, [V, V, V, D, I, V, V, V, V]),
        "gmg_grad_pattern": (I, [V, V, V, V, V, V]),
        "gmg_set_t": (I, [V, D, V]),
        "gmg_mass": (I, [V, V, V, V]),
        "gmg_grad": (I, [V, V, V, V, V, V, V]),
        "gmg_setup_many": (I, [V, I, V, V, V, V, V]),
        "gmg_autotune": (I, [V, V, V]),
        "gmg_set_lanes": (I, [V, V]),
        "gmg_autotune_batched": (I, [V, I, V, V]),
        "gmg_set_lanes_batched": (I, [V, I, V]),
        "gmg_autotune_many": (I, [V, I, V]),
        "gmg_build_hierarchy": (I, [V, I64, V, V, V, D, I64, I, V]),
        "gmg_hierarchy_info": (I, [V, V, V]),
        "gmg_hierarchy_level": (I, [V, I, V, V, V, V, V, V, V, V, V, V, V]),
        "gmg_destroy_hierarchy": (I, [V]),
        "gmg_solve_many": (I, [V, I, V, V, D, I, V, V]),
        "gmg_destroy_many": (I, [V]),
        "gmg_profile_read": (I, [V, V]),
        "gmg_profile_levels": (I, [V, V]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(st: int, where: str, ok=(GMG_OK,)):
    if st not in ok:
        raise GMGError(st, where, load_library().gmg_last_error().decode())
    return st


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def colour(A):
    """The library's colouring of the symmetric sparsity pattern of the scipy
    CSR matrix `A` (sorted, unique columns): (colour of every row, number of
    colours).  Host only (`gmg_colour`)."""
    n = A.shape[0]
    rp = np.ascontiguousarray(A.indptr, dtype=np.int64)
    ci = np.ascontiguousarray(A.indices, dtype=np.int32)
    out = np.empty(n, dtype=np.int32)
    nc = ctypes.c_int32(0)
    _check(load_library().gmg_colour(n, _np_ptr(rp), _np_ptr(ci), _np_ptr(out), ctypes.byref(nc)), "gmg_colour")
    return out, int(nc.value)


def load_hierarchy(path: str):
    """(prolongations, per-level colourings) saved by Solver.save_hierarchy:
    pass them as Solver(A, Ps, coloring=colourings)."""
    from types import SimpleNamespace

    z = np.load(path)
    nlev = int(z["nlev"][0])
    Ps = []
    for l in range(nlev - 1):
        idx, w = z[f"p{l}_idx"], z[f"p{l}_w"]
        Ps.append(SimpleNamespace(n_fine=idx.reshape(-1, 3).shape[0], n_coarse=int(z[f"p{l}_n_coarse"][0]),
                                  idx=idx, w=w))
    return Ps, [z[f"colour{l}"] for l in range(nlev)]


def _stream():
    import torch

    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dptr(t, n: int | None = None):
    import torch

    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"expected {n} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


class Solver:
    """A multigrid hierarchy on the GPU (gmg_setup).

    A: scipy sparse matrix (symmetric, sorted CSR with the diagonal present).
    Ps: prolongations, finest first, each with n_coarse, idx [n,3] int32 and
        w [n,3] float64 (three slots per row, weight 0 = unused slot).
    """

    def __init__(self, A, Ps, precision: int = GMG_FP32_REFINE, nu_pre: int = 2, nu_post: int = 2,
                 max_iter: int = 100, post_forward: bool = False, use_graphs: bool = True, ml=None,
                 coloring=None):
        """`ml = (Mdiag, L, t)` builds the hierarchy of A = M + t L with M and L
        kept split (gmg_setup_ML); A is then ignored.  `coloring`: None (the
        library's greedy colouring on every level) or one entry per level,
        each None or an int array of colours in that level's numbering."""
        import scipy.sparse as sp

        lib = load_library()
        if ml is not None:
            Mdiag, A, t = ml
            self._M = np.ascontiguousarray(Mdiag, dtype=np.float64)
            self.t = float(t)
        A = sp.csr_matrix(A)
        A.sort_indices()
        self.n = A.shape[0]
        self._rp = np.ascontiguousarray(A.indptr, dtype=np.int64)
        self._ci = np.ascontiguousarray(A.indices, dtype=np.int32)
        self._va = np.ascontiguousarray(A.data, dtype=np.float64)
        csr = gmg_csr(self.n, _np_ptr(self._rp).value, _np_ptr(self._ci).value, _np_ptr(self._va).value)
        keep, arr = [], (gmg_prolong * max(1, len(Ps)))()
        nf = self.n
        for l, P in enumerate(Ps):
            idx = np.ascontiguousarray(P.idx, dtype=np.int32)
            w = np.ascontiguousarray(P.w, dtype=np.float64)
            keep += [idx, w]
            arr[l] = gmg_prolong(nf, P.n_coarse, _np_ptr(idx).value, _np_ptr(w).value)
            nf = P.n_coarse
        opt = gmg_options(precision, nu_pre, nu_post, max_iter, int(post_forward), int(use_graphs))
        self._opt = opt
        col = None
        if coloring is not None:
            if len(coloring) != len(Ps) + 1:
                raise ValueError("coloring needs one entry per level")
            self._col = [None if c is None else np.ascontiguousarray(c, dtype=np.int32) for c in coloring]
            col = (ctypes.c_void_p * len(self._col))(*[None if c is None else _np_ptr(c).value for c in self._col])
        h = ctypes.c_void_p()
        if ml is not None:
            _check(lib.gmg_setup_ML(ctypes.byref(h), _np_ptr(self._M), ctypes.byref(csr), self.t, len(Ps), arr, col,
                                    ctypes.byref(opt), _stream()), "gmg_setup_ML")
        else:
            _check(lib.gmg_setup(ctypes.byref(h), ctypes.byref(csr), len(Ps), arr, col, ctypes.byref(opt),
                                 _stream()), "gmg_setup")
        self._h = h
        self._lib = lib
        self._Ps = [(int(P.n_coarse), np.asarray(P.idx, dtype=np.int32), np.asarray(P.w, dtype=np.float64)) for P in Ps]
        nl = ctypes.c_int()
        lib.gmg_num_levels(h, ctypes.byref(nl))
        self.nlev = nl.value
        self.dims = []
        for l in range(self.nlev):
            n, nnz, nc = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
            lib.gmg_level_info(h, l, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(nc))
            self.dims.append((n.value, nnz.value, nc.value))
        self.paths = []  # per level, how the FP32 cycle runs it (gmg_level_path)
        for l in range(self.nlev):
            p = ctypes.c_int()
            lib.gmg_level_path(h, l, ctypes.byref(p))
            self.paths.append(p.value)
        fl, dev = ctypes.c_uint32(0), ctypes.c_double(0.0)
        _check(lib.gmg_warnings(h, ctypes.byref(fl), ctypes.byref(dev)), "gmg_warnings")
        self.warnings = fl.value  # GMG_WARN_P_UNITY: some P_l row's weights do not sum to 1 within 1e-12
        self.p_unity_dev = dev.value  # largest |sum_k w_ik - 1| over every P_l

    def close(self):
        if getattr(self, "_h", None) is not None:
            self._lib.gmg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # ---- whole solves ----
    def solve(self, b, x=None, tol: float = 1e-10, history: int = 0, raise_on_fail: bool = True):
        """Solves A x = b.  b/x: CUDA float64 tensors (device path) or numpy
        arrays (host path).  Returns (x, iters, rel_res, history, status)."""
        import torch

        hist = np.zeros(max(1, history))
        info = gmg_solve_info(0, 0.0, _np_ptr(hist).value if history else None, history)
        if isinstance(b, torch.Tensor):
            xx = torch.zeros_like(b) if x is None else x
            st = self._lib.gmg_solve(self._h, _dptr(b, self.n), _dptr(xx, self.n), tol, GMG_MEM_DEVICE,
                                     ctypes.byref(info), _stream())
        else:
            bb = np.ascontiguousarray(b, dtype=np.float64)
            xx = np.zeros(self.n) if x is None else np.ascontiguousarray(x, dtype=np.float64).copy()
            st = self._lib.gmg_solve(self._h, _np_ptr(bb), _np_ptr(xx), tol, GMG_MEM_HOST, ctypes.byref(info),
                                     _stream())
        if raise_on_fail:
            _check(st, "gmg_solve")
        return xx, info.iters, info.rel_res, hist[: min(history, info.iters + 1)], st

    def solve_batched(self, B, X=None, tol: float = 1e-10, history: int = 0, raise_on_fail: bool = True):
        import torch

        hist = np.zeros(max(1, history))
        info = gmg_solve_info(0, 0.0, _np_ptr(hist).value if history else None, history)
        if isinstance(B, torch.Tensor):
            nrhs = B.shape[1]
            XX = torch.zeros_like(B) if X is None else X
            st = self._lib.gmg_solve_batched(self._h, nrhs, _dptr(B), _dptr(XX), tol, GMG_MEM_DEVICE,
                                             ctypes.byref(info), _stream())
        else:
            BB = np.ascontiguousarray(B, dtype=np.float64)
            nrhs = BB.shape[1]
            XX = np.zeros_like(BB) if X is None else np.ascontiguousarray(X, dtype=np.float64).copy()
            st = self._lib.gmg_solve_batched(self._h, nrhs, _np_ptr(BB), _np_ptr(XX), tol, GMG_MEM_HOST,
                                             ctypes.byref(info), _stream())
        if raise_on_fail:
            _check(st, "gmg_solve_batched")
        return XX, info.iters, info.rel_res, hist[: min(history, info.iters + 1)], st

    def set_values(self, val):
        import torch

        if isinstance(val, torch.Tensor):
            _check(self._lib.gmg_set_values(self._h, _dptr(val), GMG_MEM_DEVICE, _stream()), "gmg_set_values")
        else:
            v = np.ascontiguousarray(val, dtype=np.float64)
            _check(self._lib.gmg_set_values(self._h, _np_ptr(v), GMG_MEM_HOST, _stream()), "gmg_set_values")

    # ---- A(t) = M + t L and gradients (handles built with ml=...) ----
    def set_t(self, t: float):
        _check(self._lib.gmg_set_t(self._h, float(t), _stream()), "gmg_set_t")
        self.t = float(t)

    def mass(self, u, out=None):
        import torch

        out = torch.empty_like(u) if out is None else out
        _check(self._lib.gmg_mass(self._h, _dptr(u, self.n), _dptr(out, self.n), _stream()), "gmg_mass")
        return out

    def grad(self, lam, x, pattern: bool = False):
        """(M lam, -lam^T L x as a 0-d tensor, -lam_i x_j on the pattern or None)."""
        import torch

        g_u0 = torch.empty_like(lam)
        dldt = torch.zeros((), dtype=torch.float64, device=lam.device)
        G = torch.empty(self._va.size, dtype=torch.float64, device=lam.device) if pattern else None
        _check(self._lib.gmg_grad(self._h, _dptr(lam, self.n), _dptr(x, self.n), _dptr(g_u0),
                                  ctypes.c_void_p(dldt.data_ptr()), _dptr(G) if pattern else None, _stream()),
               "gmg_grad")
        return g_u0, dldt, G

    def autotune(self):
        """Picks the warps-per-row split of every level by timing (gmg_autotune)."""
        lanes = (ctypes.c_int * max(1, self.nlev - 1))()
        _check(self._lib.gmg_autotune(self._h, lanes, _stream()), "gmg_autotune")
        return list(lanes)[: self.nlev - 1]

    def set_lanes(self, lanes):
        """Fixes the warps-per-row split of every smoothed level (gmg_set_lanes)."""
        arr = (ctypes.c_int * max(1, self.nlev - 1))(*[int(v) for v in lanes])
        _check(self._lib.gmg_set_lanes(self._h, arr), "gmg_set_lanes")

    def autotune_batched(self, nrhs: int):
        """Picks the multi-right-hand-side kernels' split per level for nrhs columns."""
        lanes = (ctypes.c_int * max(1, self.nlev - 1))()
        _check(self._lib.gmg_autotune_batched(self._h, int(nrhs), lanes, _stream()), "gmg_autotune_batched")
        return list(lanes)[: self.nlev - 1]

    def set_lanes_batched(self, nrhs: int, lanes):
        arr = (ctypes.c_int * max(1, self.nlev - 1))(*[int(v) for v in lanes])
        _check(self._lib.gmg_set_lanes_batched(self._h, int(nrhs), arr), "gmg_set_lanes_batched")

    def profile(self, enable: bool = True):
        _check(self._lib.gmg_profile(self._h, int(enable)), "gmg_profile")

    def profile_read(self):
        """(finest smoothing ms, GS launches, V-cycle ms, V-cycles) since the last read."""
        out = np.zeros(4)
        _check(self._lib.gmg_profile_read(self._h, _np_ptr(out)), "gmg_profile_read")
        return tuple(float(v) for v in out)

    def profile_levels(self):
        """Per level: (smoothing ms, GS launches, transfer ms, whole-level ms) since the last read."""
        out = np.zeros(4 * self.nlev)
        _check(self._lib.gmg_profile_levels(self._h, _np_ptr(out)), "gmg_profile_levels")
        return [tuple(float(v) for v in out[4 * l: 4 * l + 4]) for l in range(self.nlev)]

    # ---- introspection ----
    def level(self, l: int):
        """(A_l as scipy CSR in caller numbering, colour of every row)."""
        import scipy.sparse as sp

        n, nnz, _ = self.dims[l]
        rp, ci, va, col = np.empty(n + 1, np.int64), np.empty(nnz, np.int32), np.empty(nnz), np.empty(n, np.int32)
        _check(self._lib.gmg_level_export(self._h, l, _np_ptr(rp), _np_ptr(ci), _np_ptr(va), _np_ptr(col)),
               "gmg_level_export")
        return sp.csr_matrix((va, ci, rp), shape=(n, n)), col

    def save_hierarchy(self, path: str):
        """Writes the prolongations and every level's colouring to an .npz file;
        `load_hierarchy` returns them so that a later Solver on the same system
        skips the colouring (its caller-colouring path) and starts from them."""
        arrs = {"nlev": np.array([self.nlev])}
        for l, (nc, idx, w) in enumerate(self._Ps):
            arrs[f"p{l}_n_coarse"] = np.array([nc])
            arrs[f"p{l}_idx"] = idx
            arrs[f"p{l}_w"] = w
        for l in range(self.nlev):
            arrs[f"colour{l}"] = self.level(l)[1]
        np.savez(path, **arrs)

    # ---- single steps of Alg. 2 (device tensors, caller numbering) ----
    def smooth(self, l, x, b, nsweep, descending=False, fp32=False):
        _check(self._lib.gmg_smooth(self._h, l, int(fp32), _dptr(b), _dptr(x), nsweep, int(descending), _stream()),
               "gmg_smooth")
        return x

    def residual(self, l, x, b, r, fp32=False):
        _check(self._lib.gmg_residual(self._h, l, int(fp32), _dptr(x), _dptr(b), _dptr(r), _stream()),
               "gmg_residual")
        return r

    def restrict(self, l, r, bc, fp32=False):
        _check(self._lib.gmg_restrict(self._h, l, int(fp32), _dptr(r), _dptr(bc), _stream()), "gmg_restrict")
        return bc

    def prolong_add(self, l, u, x, fp32=False):
        _check(self._lib.gmg_prolong_add(self._h, l, int(fp32), _dptr(u), _dptr(x), _stream()), "gmg_prolong_add")
        return x

    def coarse_solve(self, b, x, fp32=False):
        _check(self._lib.gmg_coarse_solve(self._h, int(fp32), _dptr(b), _dptr(x), _stream()), "gmg_coarse_solve")
        return x

    def vcycle(self, x, b, fp32=False):
        _check(self._lib.gmg_vcycle(self._h, int(fp32), _dptr(b), _dptr(x), _stream()), "gmg_vcycle")
        return x

    def vcycle_batched(self, X, B):
        """One FP32 V-cycle on every column of the [n, nrhs] blocks (X in place)."""
        if B.dim() != 2 or X.shape != B.shape or B.shape[0] != self.n:
            raise ValueError("expected X and B of shape [n, nrhs]")
        _check(self._lib.gmg_vcycle_batched(self._h, B.shape[1], _dptr(B), _dptr(X), _stream()), "gmg_vcycle_batched")
        return X


class SolverMany:
    """A batch of independent systems (gmg_setup_many): `systems` is a list
    of (A, Ps) pairs.  solve() takes one [n_k, nrhs] CUDA float64 tensor per
    system and solves them all together (one graph launch per iteration)."""

    def __init__(self, systems, precision: int = GMG_FP32_REFINE, nu_pre: int = 2, nu_post: int = 2,
                 max_iter: int = 100):
        import scipy.sparse as sp

        lib = load_library()
        K = len(systems)
        self._keep = []
        self.sizes = []
        csrs = (gmg_csr * K)()
        nps = (ctypes.c_int * K)()
        plists = (ctypes.c_void_p * K)()
        for k, (A, Ps) in enumerate(systems):
            A = sp.csr_matrix(A)
            A.sort_indices()
            rp = np.ascontiguousarray(A.indptr, dtype=np.int64)
            ci = np.ascontiguousarray(A.indices, dtype=np.int32)
            va = np.ascontiguousarray(A.data, dtype=np.float64)
            csrs[k] = gmg_csr(A.shape[0], _np_ptr(rp).value, _np_ptr(ci).value, _np_ptr(va).value)
            arr = (gmg_prolong * max(1, len(Ps)))()
            nf = A.shape[0]
            for l, P in enumerate(Ps):
                idx = np.ascontiguousarray(P.idx, dtype=np.int32)
                w = np.ascontiguousarray(P.w, dtype=np.float64)
                self._keep += [idx, w]
                arr[l] = gmg_prolong(nf, P.n_coarse, _np_ptr(idx).value, _np_ptr(w).value)
                nf = P.n_coarse
            self._keep += [rp, ci, va, arr]
            nps[k] = len(Ps)
            plists[k] = ctypes.cast(arr, ctypes.c_void_p).value
            self.sizes.append(A.shape[0])
        opt = gmg_options(precision, nu_pre, nu_post, max_iter, 0, 1)
        h = ctypes.c_void_p()
        _check(lib.gmg_setup_many(ctypes.byref(h), K, csrs, nps, plists, ctypes.byref(opt), _stream()),
               "gmg_setup_many")
        self._h, self._lib, self.K = h, lib, K

    def solve(self, Bs, Xs=None, tol: float = 1e-10, raise_on_fail: bool = True):
        """Returns (Xs, per-system iterations, per-system relative residual, status)."""
        import torch

        nrhs = Bs[0].shape[1]
        Xs = [torch.zeros_like(b) for b in Bs] if Xs is None else Xs
        bp = (ctypes.c_void_p * self.K)(*[_dptr(b).value for b in Bs])
        xp = (ctypes.c_void_p * self.K)(*[_dptr(x).value for x in Xs])
        info = (gmg_solve_info * self.K)()
        st = self._lib.gmg_solve_many(self._h, nrhs, bp, xp, tol, GMG_MEM_DEVICE, info, _stream())
        if raise_on_fail:
            _check(st, "gmg_solve_many")
        return Xs, [i.iters for i in info], [i.rel_res for i in info], st

    def autotune(self, nrhs: int):
        """Autotunes every mesh's multi-right-hand-side kernels for nrhs columns."""
        _check(self._lib.gmg_autotune_many(self._h, int(nrhs), _stream()), "gmg_autotune_many")

    def close(self):
        if getattr(self, "_h", None) is not None:
            self._lib.gmg_destroy_many(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BuiltLevel:
    """One level of a hierarchy built on the GPU (gmg_build_hierarchy): the
    prolongation in the layout Solver takes (n_coarse, idx [n, 3], w [n, 3])
    and the construction's by-products."""

    def __init__(self, n_fine, n_coarse, idx, w, samples, cell, Xc, graph_rowptr, graph_col, stats):
        self.n_fine, self.n_coarse = n_fine, n_coarse
        self.idx, self.w = idx, w
        self.samples, self.cell, self.Xc = samples, cell, Xc
        self.graph_rowptr, self.graph_col = graph_rowptr, graph_col
        self.stats = dict(fallback=int(stats[0]), repaired=int(stats[1]), single=int(stats[2]), seeds=int(stats[3]))


def build_hierarchy(X, rowptr, col, phi: float = 1.0 / 8.0, stop: int = 1000, max_levels: int = 24):
    """The hierarchy construction of Sec. 4 on the GPU.  X: [n, 3] points;
    (rowptr, col): the symmetric neighbour graph.  Returns (levels, GPU ms)."""
    lib = load_library()
    X = np.ascontiguousarray(X, dtype=np.float64)
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(col, dtype=np.int32)
    h = ctypes.c_void_p()
    _check(lib.gmg_build_hierarchy(ctypes.byref(h), X.shape[0], _np_ptr(X), _np_ptr(rp), _np_ptr(ci), float(phi),
                                   int(stop), int(max_levels), _stream()), "gmg_build_hierarchy")
    try:
        nP, ms = ctypes.c_int(), ctypes.c_double()
        _check(lib.gmg_hierarchy_info(h, ctypes.byref(nP), ctypes.byref(ms)), "gmg_hierarchy_info")
        out = []
        for l in range(nP.value):
            nf, nc, nnz = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
            _check(lib.gmg_hierarchy_level(h, l, ctypes.byref(nf), ctypes.byref(nc), ctypes.byref(nnz), None, None,
                                           None, None, None, None, None, None), "gmg_hierarchy_level")
            nf, nc, nnz = nf.value, nc.value, nnz.value
            idx, w = np.empty((nf, 3), np.int32), np.empty((nf, 3))
            samples, cell, Xc = np.empty(nc, np.int32), np.empty(nf, np.int32), np.empty((nc, 3))
            grp, gcol, st = np.empty(nc + 1, np.int64), np.empty(nnz, np.int32), np.empty(4, np.int64)
            _check(lib.gmg_hierarchy_level(h, l, None, None, None, _np_ptr(idx), _np_ptr(w), _np_ptr(samples),
                                           _np_ptr(cell), _np_ptr(Xc), _np_ptr(grp), _np_ptr(gcol), _np_ptr(st)),
                   "gmg_hierarchy_level")
            out.append(BuiltLevel(nf, nc, idx, w, samples, cell, Xc, grp, gcol, st))
        return out, ms.value
    finally:
        lib.gmg_destroy_hierarchy(h)
