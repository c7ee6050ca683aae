"""Comparison of a GPU result with the oracle's, used by every GPU parity test.

A result passes when BOTH hold:
  * normwise:     ||gpu - ref||_2 / ||ref||_2 <= tol
  * element-wise: max_i |gpu_i - ref_i| <= tol * max_i |ref_i|
The normwise bound alone dilutes a few wrong rows by about 1/sqrt(n) on the
million-row workloads; the element-wise bound catches a single bad row (a
padding slot, the last partial slice of a colour, a colour boundary).  Every
entry must also be finite.
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


def assert_close(got, ref, tol: float, what: str = ""):
    g = np.asarray(got, dtype=np.float64)
    assert np.all(np.isfinite(g)), f"{what}: non-finite entries"
    ne, ee, k = errors(g, ref)
    assert ne <= tol, f"{what}: normwise relative error {ne:.3e} > {tol:.1e}"
    assert ee <= tol, f"{what}: element-wise error {ee:.3e} (entry {k}) > {tol:.1e} of max|ref|"
    return ne, ee
