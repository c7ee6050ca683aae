"""Pins of the oracle's adjoint gradients (adjoint_gradients) for
x = (M + t L)^-1 M u0 and loss = ||x - x_target||^2, against central finite
differences with step 1e-6 computed from the oracle's own solves.

The loss difference is formed as (x+ - x-) . (x+ + x- - 2 x_target), which
equals loss(+) - loss(-) exactly in real arithmetic and avoids cancelling two
large numbers.  With solves to 1e-14 the finite-difference error is about
1e-14 / 1e-6 relative to the perturbation, far below the 1e-5 used here."""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import gmg_inputs as gi
import oracle

H = 1e-6
TOL = 1e-14


def _system(t):
    s = gi.heat_system(48, 20, t=t, hot=8, stop=100)
    return s


def _solve(s, t, rhs):
    A = (sp.diags(s.Mdiag) + t * s.L).tocsr()
    A.sort_indices()
    o = oracle.Oracle(A, s.Ps)
    x, it, hist, ok = o.solve(rhs, tol=TOL, max_iter=300)
    assert ok
    return x


def test_adjoint_identity():
    s = _system(1e-2)
    rng = np.random.default_rng(0)
    u, v = rng.standard_normal(s.n), rng.standard_normal(s.n)
    a = _solve(s, 1e-2, u) @ v
    b = u @ _solve(s, 1e-2, v)
    assert abs(a - b) <= 1e-12 * abs(a)


def test_gradients_match_finite_differences():
    t = 1e-2
    s = _system(t)
    u0, xt = s.extra["u0"], s.extra["x_target"]
    x = _solve(s, t, s.Mdiag * u0)
    lam = _solve(s, t, 2.0 * (x - xt))
    g_u0, g_t = oracle.adjoint_gradients(s.L, s.Mdiag, lam, x)

    def dloss(xp, xm):
        return (xp - xm) @ (xp + xm - 2.0 * xt)

    xp, xm = _solve(s, t + H, s.Mdiag * u0), _solve(s, t - H, s.Mdiag * u0)
    fd_t = dloss(xp, xm) / (2 * H)
    assert abs(fd_t - g_t) <= 1e-5 * abs(g_t)
    rng = np.random.default_rng(1)
    idx = np.concatenate([s.extra["hot"][:4], rng.choice(s.n, 4, replace=False)])
    for k in idx:
        e = np.zeros(s.n)
        e[k] = H
        xp, xm = _solve(s, t, s.Mdiag * (u0 + e)), _solve(s, t, s.Mdiag * (u0 - e))
        fd = dloss(xp, xm) / (2 * H)
        assert abs(fd - g_u0[k]) <= 1e-5 * abs(g_u0[k]) + 1e-12
