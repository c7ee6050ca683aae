"""Hierarchy construction of Sec. 4 on the GPU (gmg_build_hierarchy) against
the host builder that produces every workload's prolongations: on every level
the samples, the Voronoi cells, the coarse points, the coarse neighbour graph
and the prolongation (indices and weights) are bit-identical, on meshes with
index orders that make the sampling sweep's dependencies short (icosphere)
and long (row-major tori), a non-manifold mesh, a point cloud's
nearest-neighbour graph, and the full 1M-vertex torus.
The GPU takes the sweep's exact decisions (a propagation over the relation
"t < s and s within r of t"), the Voronoi labels of multi-source Dijkstra
(Jacobi rounds of lexicographic minimisation), and the host builder's
arithmetic operation by operation."""
import numpy as np
import pytest

from gmg_inputs import meshes, operators
from gmg_inputs.hierarchy import build_level

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gmg(cuda):
    import paper_2307_04886_gb300 as g

    g.load_library()
    return g


def _mesh(name):
    if name == "ico5":
        V, F = meshes.icosphere(5)
    elif name == "torus":
        V, F, _ = meshes.jittered_torus(256, 120, 7)
    elif name == "book":
        V, F, _ = meshes.book(3, 60, 80, seed=7)
    elif name == "cloud":  # the point-cloud neighbourhood graph (union of 6 nearest neighbours)
        V = meshes.noisy_sphere_cloud(65536, np.random.default_rng(2))
        E, _ = operators.knn_graph(V, 6)
        rp, ci = operators.edges_to_adjacency(V.shape[0], E)
        return V, rp, ci
    else:
        V, F, _ = meshes.jittered_torus(2048, 512, 1)
    rp, ci = operators.edges_to_adjacency(V.shape[0], meshes.mesh_edges(F))
    return V, rp, ci


def _compare(gmg, V, rp, ci, stop=200):
    levels, ms = gmg.build_hierarchy(V, rp, ci, stop=stop)
    X, r, c = V, rp, ci
    n = V.shape[0]
    k = 0
    while n > stop:
        P, Xc, crp, cci = build_level(X, r, c)
        if P.n_coarse >= n or P.n_coarse == 0:
            break
        assert k < len(levels), "the GPU hierarchy stopped early"
        G = levels[k]
        assert G.n_fine == n and G.n_coarse == P.n_coarse, f"level {k}: sizes"
        assert np.array_equal(G.samples, P.samples), f"level {k}: samples"
        assert np.array_equal(G.cell, P.seed), f"level {k}: Voronoi cells"
        assert np.array_equal(G.Xc, Xc), f"level {k}: coarse points"
        assert np.array_equal(G.graph_rowptr, crp) and np.array_equal(G.graph_col, cci), f"level {k}: coarse graph"
        assert np.array_equal(G.idx, P.idx) and np.array_equal(G.w, P.w), f"level {k}: prolongation"
        assert G.stats == P.stats, f"level {k}: statistics"
        X, r, c, n = Xc, crp, cci, P.n_coarse
        k += 1
    assert k == len(levels) and k >= 2
    return ms


@pytest.mark.parametrize("name", ["ico5", "torus", "book", "cloud"])
def test_gpu_hierarchy_is_the_host_builders(gmg, name):
    _compare(gmg, *_mesh(name))


@pytest.mark.slow
def test_gpu_hierarchy_full_torus(gmg):
    ms = _compare(gmg, *_mesh("torus1m"), stop=1000)
    assert ms > 0


def test_gpu_hierarchy_rejects_bad_graphs(gmg):
    V, rp, ci = _mesh("ico5")
    bad = ci.copy()
    bad[rp[5]] = 5  # a self loop in row 5
    with pytest.raises(gmg.GMGError) as e:
        gmg.build_hierarchy(V, rp, bad)
    assert e.value.status == gmg.GMG_ERR_INVALID_ARG
    Vn = V.copy()
    Vn[3, 1] = np.nan
    with pytest.raises(gmg.GMGError) as e:
        gmg.build_hierarchy(Vn, rp, ci)
    assert e.value.status == gmg.GMG_ERR_NONFINITE
