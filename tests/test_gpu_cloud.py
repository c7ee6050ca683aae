"""Point-cloud workload (k = 30 Gaussian kNN Laplacian, A = I + 1e-3 L, about
33 entries per row and 26 colours on the finest level): Galerkin levels and
colourings against the oracle, one FP32 V-cycle at 1e-6 and FP64 at 1e-12
(normwise and element-wise),
and a solve to 1e-10, on a 262,144-point cloud and on the full
4,194,304-point workload."""
import numpy as np
import pytest

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


def _check(gmg, s, full_levels=True):
    o = oracle.Oracle(s.A, s.Ps)
    g = gmg.Solver(s.A, s.Ps, precision=gmg.GMG_FP32_PCG)
    assert g.nlev == o.nlev
    for l in range(o.nlev):
        Ao, co = o.level(l)
        Ag, cg = g.level(l)
        assert np.array_equal(Ao.indices, Ag.indices) and np.array_equal(co, cg)
        assert np.array_equal(Ao.data, Ag.data), f"Galerkin level {l}"
    rng = np.random.default_rng(9)
    x0 = rng.standard_normal(s.n)
    xo = o.vcycle(x0, s.b)
    close(g.vcycle(_t(x0), _t(s.b), fp32=True).cpu().numpy(), xo, 1e-6, "FP32 V-cycle", stencil_factor(s.A))
    close(g.vcycle(_t(x0), _t(s.b), fp32=False).cpu().numpy(), xo, 1e-12, "FP64 V-cycle")
    x, it, rr, _, _ = g.solve(_t(s.b), tol=1e-10)
    xn = x.cpu().numpy()
    assert np.linalg.norm(s.b - s.A @ xn) <= 1e-10 * np.linalg.norm(s.b)
    xr, _, _, ok = o.solve(s.b, tol=1e-12, pcg=True)
    assert ok
    close(xn, xr, 1e-8, "solution")
    g.close()


def test_cloud_262k(gmg):
    _check(gmg, gi.cached("cloud262k", gi.cloud_system, 262144))


@pytest.mark.slow
def test_cloud_full_size(gmg):
    _check(gmg, gi.workload("cloud4m"))
