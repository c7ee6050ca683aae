"""Comparison of a GPU result with the oracle's, used by every GPU parity test.

A result passes when BOTH hold:
  * normwise:     ||gpu - ref||_2 / ||ref||_2 <= tol
  * element-wise: max_i |gpu_i - ref_i| <= tol * max_i |ref_i|
The normwise bound alone dilutes a few wrong rows by about 1/sqrt(n) on the
million-row workloads; the element-wise bound catches a single bad row (a
padding slot, the last partial slice of a colour, a colour boundary).  Every
entry must also be finite.

For FP32 results the element-wise bound is the normwise one times
stencil_factor(A): rounding in one Gauss-Seidel update or residual row grows
with the row's length z (about sqrt(z) for independent roundings) and with its
cancellation, gamma = sum_j |a_ij| / a_ii (the row's terms are gamma times
larger than its result).  The FP32 tolerance 1e-6 is stated for Laplace-type
rows (z = 7, gamma <= 2, factor 1); rows with obtuse-angle cotan weights
(gamma up to 5 on the jittered 1M torus) or two-ring stencils (z = 19) may
round more in their worst entry.  FP64 bounds need no factor: they sit about
four orders above the FP64 rounding level.
"""
from __future__ import annotations

import numpy as np


def errors(got, ref):
    """(normwise relative error, element-wise max error relative to max|ref|, index of the worst entry)."""
    g = np.asarray(got, dtype=np.float64).ravel()
    r = np.asarray(ref, dtype=np.float64).ravel()
    assert g.shape == r.shape, f"shape {g.shape} != {r.shape}"
    d = np.abs(g - r)
    nr = float(np.linalg.norm(r))
    mr = float(np.abs(r).max()) if r.size else 0.0
    norm_err = float(np.linalg.norm(g - r)) / max(nr, 1e-300)
    k = int(d.argmax()) if d.size else 0
    elem_err = float(d[k]) / max(mr, 1e-300) if d.size else 0.0
    return norm_err, elem_err, k


def stencil_factor(A) -> float:
    """max(1, sqrt(z_max / 7) * gamma_max / 2) of the operator A (scipy CSR),
    z_max its longest row, gamma_max the largest sum_j |a_ij| / a_ii."""
    d = A.diagonal()
    gamma = float(((abs(A) @ np.ones(A.shape[0])) / d).max())
    zmax = int(np.diff(A.indptr).max())
    return max(1.0, np.sqrt(zmax / 7.0) * gamma / 2.0)


def assert_close(got, ref, tol: float, what: str = "", elem_factor: float = 1.0):
    g = np.asarray(got, dtype=np.float64)
    assert np.all(np.isfinite(g)), f"{what}: non-finite entries"
    ne, ee, k = errors(g, ref)
    et = tol * elem_factor
    assert ne <= tol, f"{what}: normwise relative error {ne:.3e} > {tol:.1e}"
    assert ee <= et, f"{what}: element-wise error {ee:.3e} (entry {k}) > {et:.2e} of max|ref|"
    return ne, ee
