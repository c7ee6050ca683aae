"""Pins of the host hierarchy builder (Sec. 4) against its defining rules,
checked with independent routines (scipy's graph Dijkstra, brute force):

* sampling (Sec. 4.2): a point is sampled iff no earlier sample reaches it
  within r = phi^(-1/3) * mean edge length inside the sample's 2-ring;
* graph Voronoi cells (Sec. 4.3): every point belongs to a seed at minimum
  graph distance;
* coarse edges: cells i, j are adjacent iff a fine edge joins them;
* shift (Sec. 4.4): coarse positions are the cell means;
* prolongation (Sec. 4.4): rows are barycentric coordinates of the closest
  point on the best candidate triangle of the point's seed (<= 3 entries,
  non-negative, summing to one), no coarse column is empty.
"""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import dijkstra

from gmg_inputs import build_level, meshes, operators


def _level(V, F):
    rp, ci = operators.edges_to_adjacency(V.shape[0], meshes.mesh_edges(F))
    P, Xc, crp, cci = build_level(V, rp, ci)
    return rp, ci, P, Xc, crp, cci


@pytest.fixture(scope="module")
def ico3():
    V, F = meshes.icosphere(3)
    return (V, F) + _level(V, F)


@pytest.fixture(scope="module")
def torus():
    V, F, _ = meshes.jittered_torus(64, 24, 5)
    return (V, F) + _level(V, F)


def _graph(V, rp, ci):
    n = V.shape[0]
    rows = np.repeat(np.arange(n), np.diff(rp))
    w = np.linalg.norm(V[rows] - V[ci], axis=1)
    return sp.csr_matrix((w, ci, rp), shape=(n, n))


@pytest.mark.parametrize("fx", ["ico3", "torus"])
def test_prolongation_rows(fx, request):
    V, F, rp, ci, P, Xc, crp, cci = request.getfixturevalue(fx)
    w, idx = P.w, P.idx
    assert np.all(w >= 0)
    assert np.abs(w.sum(axis=1) - 1.0).max() <= 1e-14
    for i in range(P.n_fine):  # non-zero slots name distinct coarse points, padding repeats slot 0
        nz = idx[i][w[i] != 0]
        assert len(set(nz.tolist())) == nz.size and nz.size >= 1
        assert np.all(idx[i][w[i] == 0] == idx[i][0])
    S = P.to_scipy()
    assert np.all(np.diff(S.tocsc().indptr) > 0), "empty coarse column"
    assert P.stats["repaired"] == 0


@pytest.mark.parametrize("fx", ["ico3", "torus"])
def test_voronoi_cells_are_nearest_seeds(fx, request):
    V, F, rp, ci, P, Xc, crp, cci = request.getfixturevalue(fx)
    G = _graph(V, rp, ci)
    D = dijkstra(G, directed=False, indices=P.samples)  # [nc, n]
    dmin = D.min(axis=0)
    dseed = D[P.seed, np.arange(V.shape[0])]
    assert np.abs(dseed - dmin).max() <= 1e-12
    assert np.array_equal(P.seed[P.samples], np.arange(P.n_coarse))


@pytest.mark.parametrize("fx", ["ico3", "torus"])
def test_coarse_edges_and_shift(fx, request):
    V, F, rp, ci, P, Xc, crp, cci = request.getfixturevalue(fx)
    n, nc = V.shape[0], P.n_coarse
    rows = np.repeat(np.arange(n), np.diff(rp))
    a, b = P.seed[rows], P.seed[ci]
    m = a != b
    expect = np.unique(a[m].astype(np.int64) * nc + b[m])
    got = np.repeat(np.arange(nc), np.diff(crp)).astype(np.int64) * nc + cci
    assert np.array_equal(np.sort(got), expect)
    for c in range(nc):
        assert np.allclose(Xc[c], V[P.seed == c].mean(axis=0), atol=1e-15)


def test_sampling_rule(ico3):
    V, F, rp, ci, P, Xc, crp, cci = ico3
    n = V.shape[0]
    G = _graph(V, rp, ci)
    E = meshes.mesh_edges(F)
    r = 8.0 ** (1.0 / 3.0) * np.linalg.norm(V[E[:, 0]] - V[E[:, 1]], axis=1).mean()
    covered = np.full(n, -1)  # first sample (in sweep order) reaching each point
    for s in P.samples:
        ring1 = ci[rp[s]:rp[s + 1]]
        ring = np.unique(np.concatenate([[s], ring1] + [ci[rp[a]:rp[a + 1]] for a in ring1]))
        sub = G[ring][:, ring]
        d = dijkstra(sub, directed=False, indices=int(np.searchsorted(ring, s)))
        reach = ring[d <= r]
        assert covered[s] == -1, "a sample lies within r of an earlier sample"
        covered[reach] = np.where(covered[reach] == -1, s, covered[reach])
    assert np.all(covered >= 0), "a point is reached by no sample"
    # sweep order: a point not sampled was reached by an earlier sample
    nonsample = np.setdiff1d(np.arange(n), P.samples)
    assert np.all(covered[nonsample] < nonsample)


_K = 240  # brute-force grid: k subdivisions per barycentric axis


def _closest_on_triangle_brute(p, tri, k=_K):
    u = np.linspace(0.0, 1.0, k + 1)
    U, W = np.meshgrid(u, u)
    m = U + W <= 1.0 + 1e-15
    bary = np.stack([1 - U[m] - W[m], U[m], W[m]], axis=1)
    pts = bary @ tri
    return np.min(np.linalg.norm(pts - p, axis=1))


def test_projection_is_closest_candidate(torus):
    V, F, rp, ci, P, Xc, crp, cci = torus
    rng = np.random.default_rng(0)
    adj = [set(cci[crp[c]:crp[c + 1]].tolist()) for c in range(P.n_coarse)]
    checked = 0
    for i in rng.choice(V.shape[0], 60, replace=False):
        c = P.seed[i]
        q = P.w[i] @ Xc[P.idx[i]]  # interpolated point
        dq = np.linalg.norm(V[i] - q)
        nb = sorted(adj[c])
        best, hmax = np.inf, 0.0
        for x in range(len(nb)):
            for y in range(x + 1, len(nb)):
                a, b = nb[x], nb[y]
                if b in adj[a]:
                    tri = Xc[[c, a, b]]
                    best = min(best, _closest_on_triangle_brute(V[i], tri))
                    hmax = max(hmax, np.linalg.norm(tri - np.roll(tri, 1, axis=0), axis=1).max())
        if np.isfinite(best):
            # the exact closest point is never farther than a sampled point, and
            # the sampled minimum is within a grid step of the exact one
            assert dq <= best + 1e-12, "a candidate triangle is closer than the chosen projection"
            assert dq >= best - 2.0 * hmax / _K
            checked += 1
    assert checked > 50


def test_coarsening_ratio_and_fallback_rate():
    s_levels = []
    V, F, _ = meshes.jittered_torus(256, 96, 9)
    rp, ci, P, Xc, crp, cci = _level(V, F)
    ratio = P.n_coarse / P.n_fine
    assert 1 / 12 < ratio < 1 / 4  # the paper aims at 1/8 (Sec. 4.2)
    assert P.stats["fallback"] / P.n_fine < 0.01  # the paper reports about 0.25% (Sec. 4.4)
    assert 3 * np.count_nonzero(P.w) / P.n_fine / 3 <= 3
