"""Many meshes of uneven size in one batch (gmg_solve_many): every mesh's
columns reach 1e-10, and the solutions agree with the single-system batched
solve (identical kernels per mesh and, since every mesh stops at its own
convergence in the device-side loop, the same iteration count: identical
bits) and with the oracle (1e-8 relative).  The full-size case is the
64-sphere workload (sizes log-uniform in [5e3, 2e5], 8 right-hand sides
each)."""
import numpy as np
import pytest

import gmg_inputs as gi
import oracle
from parity_util import assert_close as close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gmg(cuda):
    import paper_2307_04886_gb300 as g

    g.load_library()
    return g


def _t(x):
    import torch

    return torch.tensor(np.ascontiguousarray(x, dtype=np.float64), device="cuda")


def test_small_batch_matches_single_and_oracle(gmg):
    systems = gi.spheres_batch(count=6, lo=800, hi=6000, nrhs=3, seed=8, stop=200)
    many = gmg.SolverMany([(s.A, s.Ps) for s in systems])
    Xs, its, rels, st = many.solve([_t(s.b) for s in systems], tol=1e-10)
    assert st == 0 and max(rels) <= 1e-10
    for s, X in zip(systems, Xs):
        Xn = X.cpu().numpy()
        for c in range(3):
            assert np.linalg.norm(s.b[:, c] - s.A @ Xn[:, c]) <= 1e-10 * np.linalg.norm(s.b[:, c])
        one = gmg.Solver(s.A, s.Ps)
        Xb, itb, _, _, _ = one.solve_batched(_t(s.b), tol=1e-10)
        assert itb == its[systems.index(s)], "a mesh must stop at its own convergence"
        assert np.array_equal(Xb.cpu().numpy(), Xn), "same kernels, same iterations: same bits"
        o = oracle.Oracle(s.A, s.Ps)
        for c in range(3):
            xo, _, _, ok = o.solve(s.b[:, c].copy(), tol=1e-12)
            close(Xn[:, c], xo, 1e-8, f"mesh n={s.n} column {c}")
        one.close()
    many.close()


@pytest.mark.slow
def test_sixty_four_spheres(gmg):
    systems = gi.spheres_batch()  # seed 3: 64 jittered spheres, about 3.2M vertices
    assert len(systems) == 64
    many = gmg.SolverMany([(s.A, s.Ps) for s in systems])
    Xs, its, rels, st = many.solve([_t(s.b) for s in systems], tol=1e-10)
    assert st == 0 and max(rels) <= 1e-10
    assert min(its) >= 1 and max(its) <= 100
    for k in (0, 31, 63):
        s, Xn = systems[k], Xs[k].cpu().numpy()
        r = np.linalg.norm(s.b - s.A @ Xn, axis=0) / np.linalg.norm(s.b, axis=0)
        assert r.max() <= 1e-10
    many.close()


def test_device_loop_matches_host_loop(gmg, monkeypatch):
    """The device-side loop (one graph launch, per-mesh IF nodes) and the
    host-driven form (GMG_NO_DEVICE_LOOP=1: one graph per iteration, every mesh
    runs until all have converged) report the same per-mesh iteration counts
    and residuals; meshes that stop early in the device loop keep their
    converged iterate."""
    systems = gi.spheres_batch(count=5, lo=600, hi=9000, nrhs=2, seed=12, stop=200)
    out = {}
    for dev in (True, False):
        if dev:
            monkeypatch.delenv("GMG_NO_DEVICE_LOOP", raising=False)
        else:
            monkeypatch.setenv("GMG_NO_DEVICE_LOOP", "1")
        many = gmg.SolverMany([(s.A, s.Ps) for s in systems])
        Xs, its, rels, st = many.solve([_t(s.b) for s in systems], tol=1e-10)
        assert st == 0
        out[dev] = ([X.cpu().numpy() for X in Xs], its, rels)
        many.close()
    assert out[True][1] == out[False][1]
    assert np.allclose(out[True][2], out[False][2], rtol=1e-12, atol=0)
    for s, Xd in zip(systems, out[True][0]):
        r = np.linalg.norm(s.b - s.A @ Xd, axis=0) / np.linalg.norm(s.b, axis=0)
        assert r.max() <= 1e-10
