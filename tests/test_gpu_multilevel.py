"""GPU parity of the multilevel layout (Algorithm 3, Sec. 2.3) through the
C-ABI: every level of the coarsening hierarchy (grouping, adjacency, merged
edge costs, summed vertex weights), the prolongation with its jitter, and one
layout step on coarse levels, where vertex weights and edge costs are not 1
(the weighted near field and the costed attraction of the step kernel).

Bars: groupings, adjacency and costs (integer sums) bit-exact; weights equal
to the oracle's FP64 sums rounded to fp32 (exact for unit level-0 weights,
within one fp32 rounding per level otherwise); prolonged points within fp32
rounding of the FP64 formula; one step within 1e-4 normwise."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

Y_TOL = 1e-4


@pytest.fixture(scope="module")
def V():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1105_4490_gb300 as P
    assert torch.cuda.is_available()
    return P


@pytest.fixture(scope="module")
def O():
    import oracle
    oracle.build()
    return oracle


def _np(t):
    return t.detach().cpu().numpy()


def _connected_powerlaw(n, seed):
    """The largest connected component of a power-law pattern (the layout
    treats every component as its own problem; the hierarchy entry points
    coarsen the whole graph, which is the same for a connected one)."""
    from scipy import sparse
    from scipy.sparse import csgraph
    A = W.powerlaw_symmetric(n, seed=seed)
    M = sparse.csr_matrix((np.ones(len(A.colidx)), A.colidx, A.rowptr), shape=(A.m, A.m))
    _, lab = csgraph.connected_components(M, directed=False)
    big = np.flatnonzero(lab == np.bincount(lab).argmax())
    S = M[big][:, big].tocsr()
    S.sort_indices()
    return W.Matrix(f"powerlaw{n}_cc", len(big), len(big), S.indptr.astype(np.int32), S.indices.astype(np.int32))


CASES = [("grid2d_64", lambda: W.grid_laplacian_2d(64)), ("powerlaw_20k", lambda: _connected_powerlaw(20000, 3)),
         ("grid3d_24", lambda: W.grid_laplacian_3d(24))]


def _weights(k, seed):
    return np.random.default_rng(seed).uniform(0.5, 3.0, k).astype(np.float32)


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("name,make", CASES)
def test_hierarchy_levels_bit_exact(V, O, name, make, weighted):
    A = make()
    w = _weights(A.m, 4) if weighted else None
    hg = V.Hypergraph.from_matrix(A, weights=None if w is None else torch.as_tensor(w))
    ref = O.build_from_matrix("symmetric", A)
    p = V.Params(seed=21)
    sizes = hg.coarsen(p)[3]
    assert sizes == O.hierarchy(ref, 21)
    assert len(sizes) >= 4, sizes
    for j in range(len(sizes)):
        g = hg.hierarchy_level(j, p)
        o = O.hierarchy_level(ref, j, seed=21, w=None if w is None else w.astype(np.float64))
        assert g["k"] == o["k"] == sizes[j]
        assert np.array_equal(_np(g["adj_ptr"]), o["adj_ptr"]), (name, j)
        assert np.array_equal(_np(g["adj"]), o["adj"]), (name, j)
        assert np.array_equal(_np(g["acost"]).astype(np.float64), o["acost"]), (name, j)
        gw = _np(g["weight"])
        if w is None:
            assert np.array_equal(gw.astype(np.float64), o["w"]), (name, j)
        else:
            assert np.allclose(gw, o["w"], rtol=(j + 1) * 2.0 ** -23, atol=0), (name, j)
        if j > 0:
            assert np.array_equal(_np(g["pi"]), o["pi"]), (name, j)


@pytest.mark.parametrize("d", [2, 3, 4])
@pytest.mark.parametrize("name,make", CASES[:2])
def test_prolongation_matches_oracle(V, O, name, make, d):
    A = make()
    hg = V.Hypergraph.from_matrix(A)
    ref = O.build_from_matrix("symmetric", A)
    p = V.Params(d=d, seed=8)
    sizes = hg.coarsen(p)[3]
    rng = np.random.default_rng(d)
    for j in (1, len(sizes) // 2, len(sizes) - 1):
        kc, kf = sizes[j], sizes[j - 1]
        xc = np.zeros((kc, 4), dtype=np.float32)
        xc[:, :d] = rng.uniform(-30.0, 30.0, (kc, d)).astype(np.float32)
        xg = _np(hg.hierarchy_prolong(j, torch.as_tensor(xc).cuda(), kf, p)).astype(np.float64)
        pi = O.hierarchy_level(ref, j, seed=8)["pi"]
        xo = O.prolong(kf, kc, d, 8, j, pi, xc.astype(np.float64))
        # fp32 evaluation of f * x + 0.1 (u - 1/2): a few roundings of |f x| + 0.05
        bound = 4 * 2.0 ** -24 * (np.abs(xo) + 0.1)
        assert np.all(np.abs(xg - xo) <= bound), (name, j, np.abs(xg - xo).max())
        assert np.all(xg[:, d:] == 0.0)


def _level_graph(O, o):
    return O.graph_nets(o["k"], o["adj_ptr"], o["adj"], o["acost"])


@pytest.mark.parametrize("d", [2, 3, 4])
@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("name,make", CASES[:2])
def test_coarse_level_step_weighted_costed(V, O, name, make, weighted, d):
    """One step on coarse levels (non-unit vertex weights and edge costs): the
    weighted near field, the far-field charges of weighted points and the
    costed attraction, against the oracle's step on its own coarse graph."""
    A = make()
    w = _weights(A.m, 9) if weighted else None
    hg = V.Hypergraph.from_matrix(A, weights=None if w is None else torch.as_tensor(w))
    ref = O.build_from_matrix("symmetric", A)
    p = V.Params(d=d, seed=13)
    sizes = hg.coarsen(p)[3]
    for j in (1, 2, len(sizes) // 2):
        o = O.hierarchy_level(ref, j, seed=13, w=None if w is None else w.astype(np.float64))
        g = hg.hierarchy_level(j, p)
        gw = _np(g["weight"]).astype(np.float64)
        assert gw.max() > 1.0 and o["acost"].max() > 1.0
        og, oc = _level_graph(O, o)
        x0 = O.init_coords(o["k"], d, 100 + j)
        step = 0.29
        xg, yg = hg.hierarchy_step(j, torch.as_tensor(x0).cuda(), step, p)
        # the oracle on the GPU's fp32 weights (equal to its own up to rounding)
        xo, yo, _, _ = O.layout_step(og, d, x0.astype(np.float64), step, w=gw, c=oc)
        yg, xg = _np(yg).astype(np.float64), _np(xg).astype(np.float64)
        ey = np.linalg.norm(yg[:, :d] - yo[:, :d]) / np.linalg.norm(yo[:, :d])
        dx = xo[:, :d] - x0[:, :d]
        ex = np.linalg.norm((xg[:, :d] - x0[:, :d]) - dx) / np.linalg.norm(dx)
        assert ey <= Y_TOL and ex <= Y_TOL, (name, j, ey, ex)


@pytest.mark.parametrize("d", [2, 3])
def test_level0_step_with_vertex_weights(V, O, d):
    """Hypergraph(weights=...) at level 0 (the finest level of a weighted
    layout): one step against the oracle's weighted step."""
    A = _connected_powerlaw(12000, 5)
    w = _weights(A.m, 2)
    hg = V.Hypergraph.from_matrix(A, weights=torch.as_tensor(w))
    ref = O.build_from_matrix("symmetric", A)
    x0 = O.init_coords(ref.k, d, 7)
    step = 0.41
    xg, yg, kg, L = hg.layout_step(torch.as_tensor(x0).cuda(), step, V.Params(d=d))
    xo, yo, ko, Lo = O.layout_step(ref, d, x0.astype(np.float64), step, w=w.astype(np.float64))
    assert L == Lo and np.array_equal(_np(kg).view(np.uint32), ko)
    yg, xg = _np(yg).astype(np.float64), _np(xg).astype(np.float64)
    ey = np.linalg.norm(yg[:, :d] - yo[:, :d]) / np.linalg.norm(yo[:, :d])
    dx = xo[:, :d] - x0[:, :d]
    ex = np.linalg.norm((xg[:, :d] - x0[:, :d]) - dx) / np.linalg.norm(dx)
    assert ey <= Y_TOL and ex <= Y_TOL, (ey, ex)


def test_hierarchy_level_zero_and_errors(V):
    A = W.grid_laplacian_2d(20)
    hg = V.Hypergraph.from_matrix(A)
    g = hg.hierarchy_level(0)
    assert g["k"] == A.m and g["pi"] is None
    assert np.array_equal(_np(g["adj_ptr"]), hg.arrays()["adj_ptr"].cpu().numpy())
    assert torch.all(g["acost"] == 1.0) and torch.all(g["weight"] == 1.0)
    n = len(hg.coarsen()[3])
    with pytest.raises(V.VmoError):
        hg.hierarchy_level(n)
    with pytest.raises(V.VmoError):
        hg.hierarchy_prolong(0, torch.zeros((A.m, 4), device="cuda"), A.m)
    rn = V.Hypergraph.from_matrix(W.powerlaw_rectangular(300, 200, seed=1), "rownet")
    with pytest.raises(V.VmoError):
        rn.hierarchy_level(0)
