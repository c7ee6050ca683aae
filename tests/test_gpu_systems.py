"""GPU parity on the further systems of the paper: Eq. (Poisson) of Sec. 5.2
with eta = 1e-6 (nearly singular), the bi-Laplacian smoothing of Sec. 5.5
(two-ring stencil, wider Galerkin rows, more colours), and data smoothing on a
non-manifold mesh (Sec. 5.4: sheets sharing a spine whose edges border three
triangles), at 14,240 vertices and at the full 149,200-vertex workload.

Tolerances: Galerkin levels and colourings bit-exact.  One V-cycle against
the oracle (normwise and element-wise relative to the largest entry): the coarse solves differ in rounding (explicit
inverse vs Cholesky), which the coarsest operator amplifies by its condition
number kappa, so the bound is max(1e-12, 10 kappa 2^-53) in FP64 and
max(1e-6, 10 kappa 2^-24) in FP32 (1e-12 and 1e-6 for the bi-Laplacian,
kappa = 3.9).  The Poisson coarsest operator has kappa = 3.2e8: its FP64 bound
is 3.5e-7, and an FP32 cycle carries no accuracy in the near-constant mode
(kappa 2^-24 > 1), so only its use as a preconditioner is tested (the solves).
Element-wise, the FP32 bound scales with the stencil (parity_util.stencil_factor):
the bi-Laplacian's 19-entry rows carry off-diagonal mass up to 5.5 times their
diagonal, so one FP32 Gauss-Seidel update may round several times more than on
the 7-entry Laplace-type rows for which 1e-6 is stated.
Solves reach the stated residual in every precision.  The Poisson system
stalls near a 1e-8 relative residual in FP64 (a direct solve's own residual is
2.5e-8 on this mesh), so it is solved to 1e-7, still above the paper's 1e-4,
and compared with a direct solve within 1e-6."""
import numpy as np
import pytest
import scipy.sparse.linalg as sla

import gmg_inputs as gi
import oracle
from parity_util import assert_close as close
from parity_util import stencil_factor

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gmg(cuda):
    import paper_2307_04886_gb300 as g

    g.load_library()
    return g


def _t(x):
    import torch

    return torch.tensor(np.asarray(x, dtype=np.float64), device="cuda")


@pytest.fixture(scope="module", params=["poisson", "bilaplacian", "book"])
def system(request):
    if request.param == "poisson":
        return request.param, gi.workloads.poisson_system(), 1e-7
    if request.param == "book":  # non-manifold: 3 sheets sharing a spine, 14,240 vertices
        return request.param, gi.nonmanifold_system(3, 60, 80), 1e-10
    return request.param, gi.workloads.bilaplacian_system(), 1e-10


def test_levels_and_cycles_match(gmg, system):
    name, s, _ = system
    o = oracle.Oracle(s.A, s.Ps)
    g = gmg.Solver(s.A, s.Ps)
    assert g.nlev == o.nlev
    for l in range(o.nlev):
        Ao, co = o.level(l)
        Ag, cg = g.level(l)
        assert np.array_equal(Ao.indices, Ag.indices) and np.array_equal(co, cg)
        assert np.array_equal(Ao.data, Ag.data), f"{name}: Galerkin level {l}"
    Ac, _ = o.level(o.nlev - 1)
    ev = np.linalg.eigvalsh(Ac.toarray())
    kappa = ev[-1] / ev[0]
    rng = np.random.default_rng(21)
    x0 = rng.standard_normal(s.n)
    xo = o.vcycle(x0, s.b)
    close(g.vcycle(_t(x0), _t(s.b), fp32=False).cpu().numpy(), xo, max(1e-12, 10 * kappa * 2.0**-53), "FP64 cycle")
    if kappa * 2.0**-24 < 1e-3:
        close(g.vcycle(_t(x0), _t(s.b), fp32=True).cpu().numpy(), xo, max(1e-6, 10 * kappa * 2.0**-24),
              "FP32 cycle", stencil_factor(s.A))
    g.close()


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_solves(gmg, system, precision):
    name, s, tol = system
    g = gmg.Solver(s.A, s.Ps, precision=precision)
    x, it, rr, _, st = g.solve(_t(s.b), tol=tol)
    xn = x.cpu().numpy()
    assert st == 0
    assert np.linalg.norm(s.b - s.A @ xn) <= tol * np.linalg.norm(s.b)
    xe = sla.spsolve(s.A.tocsc(), s.b)
    close(xn, xe, 1e-6 if name == "poisson" else 1e-8, "solution vs direct solve")
    g.close()


@pytest.mark.slow
def test_book_full_size(gmg):
    """The full non-manifold workload (5 sheets, 149,200 vertices): Galerkin
    levels and colourings bitwise, one FP64 and one FP32 cycle element-wise
    (bounds scaled by the coarsest operator's condition number, as for the
    other systems of this file), and FP32-preconditioned CG to 1e-10 against a
    direct solve."""
    s = gi.workload("book5")
    o = oracle.Oracle(s.A, s.Ps)
    g = gmg.Solver(s.A, s.Ps, precision=gmg.GMG_FP32_PCG)
    for l in range(o.nlev):
        Ao, co = o.level(l)
        Ag, cg = g.level(l)
        assert np.array_equal(Ao.indices, Ag.indices) and np.array_equal(co, cg)
        assert np.array_equal(Ao.data, Ag.data)
    Ac, _ = o.level(o.nlev - 1)
    ev = np.linalg.eigvalsh(Ac.toarray())
    kappa = ev[-1] / ev[0]
    rng = np.random.default_rng(31)
    x0 = rng.standard_normal(s.n)
    xo = o.vcycle(x0, s.b)
    close(g.vcycle(_t(x0), _t(s.b), fp32=False).cpu().numpy(), xo, max(1e-12, 10 * kappa * 2.0**-53), "FP64 cycle")
    close(g.vcycle(_t(x0), _t(s.b), fp32=True).cpu().numpy(), xo, max(1e-6, 10 * kappa * 2.0**-24), "FP32 cycle",
          stencil_factor(s.A))
    x, it, rr, _, st = g.solve(_t(s.b), tol=1e-10)
    xn = x.cpu().numpy()
    assert st == 0 and np.linalg.norm(s.b - s.A @ xn) <= 1e-10 * np.linalg.norm(s.b)
    close(xn, sla.spsolve(s.A.tocsc(), s.b), 1e-8, "solution vs direct solve")
    g.close()
