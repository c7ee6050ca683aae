"""Planted mistakes: each test compiles a copy of the oracle with one
plausible error and checks that the corresponding pin of test_oracle.py
rejects it.  The mistakes are planted in the oracle, on the CPU."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import gmg_inputs as gi
import oracle

MUTATIONS = {
    # a dropped term in the Galerkin product (the first entry of every row of A)
    "galerkin_dropped_term": ("        double a = F->val[k];",
                              "        double a = F->val[k];\n        if (k == F->rowptr[i]) continue;"),
    # Gauss-Seidel subtracting the diagonal term as well
    "gs_includes_diagonal": ("          else sum -= L->val[k] * x[j];", "          sum -= L->val[k] * x[j];"),
    # post-relaxation in the same colour order as the pre-relaxation
    "post_order_forward": ("or_smooth(c, l, x, b, c->nu_post, !c->post_forward);",
                           "or_smooth(c, l, x, b, c->nu_post, c->post_forward);"),
    # restriction with the squared weights
    "restriction_weight": ("bc[L->pidx[3 * i + s]] += L->pw[3 * i + s] * r[i];",
                           "bc[L->pidx[3 * i + s]] += L->pw[3 * i + s] * L->pw[3 * i + s] * r[i];"),
    # transposed operand in the back substitution L^T x = y
    "cholesky_transposed": ("s -= Lf[k * n + i] * x[k];", "s -= Lf[i * n + k] * x[k];"),
    # coarse correction from the pre-relaxation input x instead of y: undo
    # the pre-smoothing before adding P u
    "correction_from_x": ("  or_smooth(c, l, x, b, c->nu_pre, 0);                 /* y = Relax(A_l, x, b) */",
                          "  double *x_in = (double *)malloc(sizeof(double) * (size_t)L->n);\n"
                          "  memcpy(x_in, x, sizeof(double) * (size_t)L->n);\n"
                          "  or_smooth(c, l, x, b, c->nu_pre, 0);\n"),
}


def _variant(name, tmp_path):
    src = oracle.source_text()
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, f"mutation site of {name} not found exactly once"
    src = src.replace(old, new)
    if name == "correction_from_x":
        site = "  or_prolong_add(c, l, C->x, x);                       /* y + P_l u            */"
        assert src.count(site) == 1
        src = src.replace(site, "  memcpy(x, x_in, sizeof(double) * (size_t)L->n);\n  free(x_in);\n" + site)
    return oracle.compile_variant(src, str(tmp_path / f"{name}.so"))


@pytest.fixture(scope="module")
def system():
    return gi.icosphere_system(3, stop=100)


def _galerkin_pin(o, s):
    for l in range(o.nlev - 1):
        Al, _ = o.level(l)
        Ac, _ = o.level(l + 1)
        Pd = s.Ps[l].to_scipy().toarray()
        D = Pd.T @ Al.toarray() @ Pd
        if np.abs(Ac.toarray() - D).max() > 1e-14 * np.abs(D).max():
            return False
    return True


def _symmetry_pin(o, n):
    B = np.empty((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        B[:, j] = o.vcycle(np.zeros(n), e)
    return np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max(), B


def test_unmodified_oracle_passes_every_pin(system, tmp_path):
    s = system
    path = oracle.compile_variant(oracle.source_text(), str(tmp_path / "plain.so"))
    o = oracle.Oracle(s.A, s.Ps, lib_path=path)
    assert _galerkin_pin(o, s)
    assert _symmetry_pin(o, s.n)[0]


def test_dropped_galerkin_term_is_caught(system, tmp_path):
    s = system
    o = oracle.Oracle(s.A, s.Ps, lib_path=_variant("galerkin_dropped_term", tmp_path))
    assert not _galerkin_pin(o, s)


def test_gs_with_diagonal_is_caught(system, tmp_path):
    from test_oracle import _gs_splitting

    s = system
    o = oracle.Oracle(s.A, s.Ps, lib_path=_variant("gs_includes_diagonal", tmp_path))
    A, col = o.level(0)
    rng = np.random.default_rng(5)
    x, b = rng.standard_normal(s.n), rng.standard_normal(s.n)
    got = o.smooth(0, x, b, 1, False)
    ref = _gs_splitting(A, col, x, b, False)
    assert np.linalg.norm(got - ref) > 1e-6 * np.linalg.norm(ref)


def test_forward_post_relaxation_is_caught(system, tmp_path):
    s = system
    o = oracle.Oracle(s.A, s.Ps, lib_path=_variant("post_order_forward", tmp_path))
    assert not _symmetry_pin(o, s.n)[0]


def test_squared_restriction_weight_is_caught(system, tmp_path):
    s = system
    o = oracle.Oracle(s.A, s.Ps, lib_path=_variant("restriction_weight", tmp_path))
    r = np.random.default_rng(6).standard_normal(s.n)
    P = s.Ps[0].to_scipy()
    assert np.linalg.norm(o.restrict(0, r) - P.T @ r) > 1e-6 * np.linalg.norm(P.T @ r)


def test_transposed_back_substitution_is_caught(system, tmp_path):
    s = system
    o = oracle.Oracle(s.A, s.Ps, lib_path=_variant("cholesky_transposed", tmp_path))
    C, _ = o.level(o.nlev - 1)
    b = np.random.default_rng(3).standard_normal(C.shape[0])
    x = o.coarse_solve(b)
    assert np.linalg.norm(C @ x - b) > 1e-6 * np.linalg.norm(b)


def test_correction_from_unsmoothed_iterate_is_caught(system, tmp_path):
    """Alg. 2 as printed (x + P u, discarding the pre-relaxed y): the cycle is
    no longer the affine map x + B (b - A x) with the symmetric B of the
    correct cycle."""
    s = system
    good = oracle.Oracle(s.A, s.Ps)
    ok, B = _symmetry_pin(good, s.n)
    assert ok
    o = oracle.Oracle(s.A, s.Ps, lib_path=_variant("correction_from_x", tmp_path))
    x = np.random.default_rng(2).standard_normal(s.n)
    lhs = o.vcycle(x, s.b)
    rhs = x + B @ (s.b - s.A @ x)
    assert np.linalg.norm(lhs - rhs) > 1e-6 * np.linalg.norm(rhs)
    # and the oracle's solve still reaches the direct solution only with the reading y + P u
    xs = spla.spsolve(s.A.tocsc(), s.b)
    xg, _, _, ok = good.solve(s.b, tol=1e-12)
    assert ok and np.linalg.norm(xg - xs) <= 1e-9 * np.linalg.norm(xs)
