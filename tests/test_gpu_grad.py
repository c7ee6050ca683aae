"""GPU gradients of loss = ||x - x_target||^2 with x = (M + t L)^-1 M u0
(heat diffusion, adjoint solve with the same hierarchy):

* gmg_grad against the oracle's adjoint formulas on the oracle's solves
  (1e-8 relative: both sides solve to 1e-13);
* the pattern gradient G_ij = -lambda_i x_j exactly (one product per entry);
* gmg_set_t levels against the oracle built for A(t) (bitwise: the same
  products in the same order);
* the torch.autograd wrapper against central finite differences with step
  1e-6 on t and on 32 sampled entries of u0 (16 hot, 16 random), on the
  524,288-vertex torus, at 1e-4 relative (the finite-difference error of
  solves to 1e-13 is about 1e-13 / 1e-6 of the perturbed solution).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import gmg_inputs as gi
import oracle
from parity_util import assert_close as close

pytestmark = pytest.mark.gpu
TOL = 1e-13


@pytest.fixture(scope="module")
def gmg(cuda):
    import paper_2307_04886_gb300 as g

    g.load_library()
    return g


def _t(x):
    import torch

    return torch.tensor(np.asarray(x, dtype=np.float64), device="cuda")


def _oracle_solve(s, t, rhs):
    A = (sp.diags(s.Mdiag) + t * s.L).tocsr()
    A.sort_indices()
    x, _, _, ok = oracle.Oracle(A, s.Ps).solve(rhs, tol=TOL, max_iter=300)
    assert ok
    return x


@pytest.mark.parametrize("precision", [1, 2])
def test_grad_matches_oracle(gmg, precision):
    import torch

    t = 1e-3
    s = gi.heat_system(96, 40, t=t, hot=16)
    solver = gmg.Solver(None, s.Ps, precision=precision, ml=(s.Mdiag, s.L, t))
    u0, xt = _t(s.extra["u0"]), _t(s.extra["x_target"])
    b = solver.mass(u0)
    assert np.array_equal(b.cpu().numpy(), s.Mdiag * s.extra["u0"])
    x = torch.zeros_like(b)
    solver.solve(b, x, tol=TOL)
    lam = torch.zeros_like(b)
    solver.solve(2.0 * (x - xt), lam, tol=TOL)
    g_u0, dldt, G = solver.grad(lam, x, pattern=True)
    xo = _oracle_solve(s, t, s.Mdiag * s.extra["u0"])
    lo = _oracle_solve(s, t, 2.0 * (xo - s.extra["x_target"]))
    go_u0, go_t = oracle.adjoint_gradients(s.L, s.Mdiag, lo, xo)
    close(g_u0.cpu().numpy(), go_u0, 1e-8, "dloss/du0")
    assert abs(dldt.item() - go_t) <= 1e-8 * abs(go_t)
    Lc = s.L.tocsr()
    rows = np.repeat(np.arange(s.n), np.diff(Lc.indptr))
    ln, xn = lam.cpu().numpy(), x.cpu().numpy()
    assert np.array_equal(G.cpu().numpy(), -ln[rows] * xn[Lc.indices])
    solver.close()


def test_set_t_refresh_matches_oracle(gmg):
    s = gi.heat_system(64, 24, t=1e-3, hot=4, stop=200)
    solver = gmg.Solver(None, s.Ps, ml=(s.Mdiag, s.L, 1e-3))
    for t in (5e-3, 2e-4):
        solver.set_t(t)
        A = (sp.diags(s.Mdiag) + t * s.L).tocsr()
        A.sort_indices()
        o = oracle.Oracle(A, s.Ps)
        for l in range(o.nlev):
            assert np.array_equal(solver.level(l)[0].data, o.level(l)[0].data), f"level {l} at t={t}"
    solver.close()


@pytest.mark.slow
def test_autograd_finite_differences_full_size(gmg):
    import torch

    from paper_2307_04886_gb300.autograd import smooth

    s = gi.workload("heat512k")
    t0 = float(s.t)
    solver = gmg.Solver(None, s.Ps, precision=gmg.GMG_FP32_REFINE, ml=(s.Mdiag, s.L, t0))
    xt = _t(s.extra["x_target"])
    u0 = _t(s.extra["u0"]).requires_grad_(True)
    t = torch.tensor(t0, dtype=torch.float64, requires_grad=True)
    x = smooth(t, u0, solver, TOL)
    loss = ((x - xt) ** 2).sum()
    loss.backward()
    g_t, g_u0 = t.grad.item(), u0.grad.detach().cpu().numpy()

    def forward(tv, u):
        with torch.no_grad():
            return smooth(torch.tensor(tv, dtype=torch.float64), u, solver, TOL)

    def dloss(xp, xm):
        return float(((xp - xm) * (xp + xm - 2.0 * xt)).sum().item())

    h = 1e-6
    u = u0.detach()
    fd_t = dloss(forward(t0 + h, u), forward(t0 - h, u)) / (2 * h)
    assert abs(fd_t - g_t) <= 1e-4 * abs(g_t)
    rng = np.random.default_rng(4)
    idx = np.concatenate([s.extra["hot"], rng.choice(s.n, 16, replace=False)])
    for k in idx:
        e = torch.zeros_like(u)
        e[int(k)] = h
        fd = dloss(forward(t0, u + e), forward(t0, u - e)) / (2 * h)
        assert abs(fd - g_u0[k]) <= 1e-4 * abs(g_u0[k]) + 1e-12, f"entry {k}"
    solver.close()


def test_autograd_interleaved_forwards_use_their_own_t(gmg):
    """Two forwards on one solver at different t, then both backwards: each
    backward must solve the adjoint system of its own forward's A(t) (the
    shared solver is left at the second t by the second forward).  Every
    gradient is checked against the oracle's adjoint formulas at its t."""
    import torch

    from paper_2307_04886_gb300.autograd import smooth

    s = gi.heat_system(96, 40, t=1e-3, hot=16)
    solver = gmg.Solver(None, s.Ps, precision=gmg.GMG_FP32_PCG, ml=(s.Mdiag, s.L, 1e-3))
    xt = _t(s.extra["x_target"])
    res = []
    for tv in (1e-3, 4e-3):
        t = torch.tensor(tv, dtype=torch.float64, requires_grad=True)
        u0 = _t(s.extra["u0"]).requires_grad_(True)
        x = smooth(t, u0, solver, TOL)
        res.append((tv, t, u0, ((x - xt) ** 2).sum()))
    for tv, t, u0, loss in res:  # backwards after both forwards, first t first
        loss.backward()
        xo = _oracle_solve(s, tv, s.Mdiag * s.extra["u0"])
        lo = _oracle_solve(s, tv, 2.0 * (xo - s.extra["x_target"]))
        go_u0, go_t = oracle.adjoint_gradients(s.L, s.Mdiag, lo, xo)
        close(u0.grad.detach().cpu().numpy(), go_u0, 1e-8, f"dloss/du0 at t={tv}")
        assert abs(t.grad.item() - go_t) <= 1e-8 * abs(go_t), f"dloss/dt at t={tv}"
    solver.close()
