"""Pins of the oracle's hypergraph models, duality and connected components
against the paper's worked example and independent constructions."""
import json
import os

import numpy as np
import pytest
from scipy import sparse
from scipy.sparse import csgraph

import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _nets(ptr, pins):
    return [sorted(pins[ptr[j]:ptr[j + 1]].tolist()) for j in range(len(ptr) - 1)]


def _matrix_from_nets(k, nets):
    """k x len(nets) pattern whose column j holds the pins of net j, so that the
    column-net model reproduces the nets."""
    rows, cols = [], []
    for j, e in enumerate(nets):
        for v in e:
            rows.append(v)
            cols.append(j)
    return W.csr_from_coo(k, len(nets), np.array(rows), np.array(cols), "nets")


def test_hgexample_colnet_dual_and_components(oracle_mod):
    O = oracle_mod
    g = json.load(open(os.path.join(GOLD, "hgexample.json")))
    nets = [[v - 1 for v in e] for e in g["nets_1based"]]
    A = _matrix_from_nets(g["vertices"], nets)
    hg = O.build_from_matrix("colnet", A)
    assert hg.k == 5 and hg.l == 4
    assert _nets(hg.net_ptr, hg.pins) == nets
    dptr, dpins = O.dual(hg.k, hg.l, hg.net_ptr, hg.pins)
    assert _nets(dptr, dpins) == [[e - 1 for e in n] for n in g["dual_nets_1based"]]
    # row-net and column-net models are each other's dual (Sec. 1.1, observation 4)
    rn = O.build_from_matrix("rownet", A)
    assert _nets(rn.net_ptr, rn.pins) == _nets(dptr, dpins)
    lab = O.components(hg)
    comps = {}
    for v, p in enumerate(lab):
        comps.setdefault(int(p), []).append(v + 1)
    assert sorted(comps.values()) == g["components_1based"]
    assert lab.tolist() == [0, 0, 0, 0, 4]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_dual_of_dual_is_identity(oracle_mod, seed):
    O = oracle_mod
    A = W.random_pattern(37, 23, 120, seed)
    for model in ("rownet", "colnet", "symmetric", "bipartite"):
        if model == "symmetric":
            A2 = W.random_pattern(31, 31, 100, seed)
            hg = O.build_from_matrix(model, A2)
        else:
            hg = O.build_from_matrix(model, A)
        p1, q1 = O.dual(hg.k, hg.l, hg.net_ptr, hg.pins)
        p2, q2 = O.dual(hg.l, hg.k, p1, q1)
        assert _nets(p2, q2) == _nets(hg.net_ptr, hg.pins)


def test_bipartite_is_dual_of_finegrain(oracle_mod):
    """Finegrain and bipartite models are each other's dual (Sec. 1.1, obs. 5):
    the dual of the finegrain hypergraph (built here independently) has one
    net {r_i, c_j} per nonzero, which is exactly the bipartite edge set."""
    O = oracle_mod
    A = W.random_pattern(19, 29, 90, 7)
    m, n = A.m, A.n
    rows = np.repeat(np.arange(m), np.diff(A.rowptr))
    cols = A.colidx
    nz = len(cols)
    # finegrain: vertices = nonzeros, nets = m row nets then n column nets
    fg = [[t for t in range(nz) if rows[t] == i] for i in range(m)] + \
         [[t for t in range(nz) if cols[t] == j] for j in range(n)]
    ptr = np.zeros(len(fg) + 1, dtype=np.int32)
    ptr[1:] = np.cumsum([len(e) for e in fg])
    pins = np.array([v for e in fg for v in e], dtype=np.int32)
    dptr, dpins = O.dual(nz, len(fg), ptr, pins)
    dual_edges = sorted(tuple(e) for e in _nets(dptr, dpins))
    bp = O.build_from_matrix("bipartite", A)
    bip_edges = sorted(tuple(e) for e in _nets(bp.net_ptr, bp.pins))
    assert dual_edges == bip_edges
    assert bp.k == m + n


@pytest.mark.parametrize("seed", [1, 5])
def test_symmetric_model_definition(oracle_mod, seed):
    """Symmetric model (Table 1): nets {i, j} for a_ij != 0, i != j, as a set;
    checked against a plain Python set construction on unsymmetric input with
    duplicates and diagonal entries."""
    O = oracle_mod
    n = 41
    A = W.random_pattern(n, n, 200, seed)
    # add duplicates and the diagonal
    rows = np.concatenate([np.repeat(np.arange(n), np.diff(A.rowptr)), np.arange(n), [3, 3]])
    cols = np.concatenate([A.colidx, np.arange(n), [5, 5]])
    rp = np.zeros(n + 1, dtype=np.int32)
    order = np.argsort(rows, kind="stable")
    rows, cols = rows[order], cols[order]
    rp[1:] = np.cumsum(np.bincount(rows, minlength=n))
    hg = O.build_hypergraph("symmetric", n, n, rp, cols.astype(np.int32))
    expect = sorted({(min(i, j), max(i, j)) for i, j in zip(rows.tolist(), cols.tolist()) if i != j})
    got = [tuple(e) for e in _nets(hg.net_ptr, hg.pins)]
    assert got == expect
    adj = {v: set() for v in range(n)}
    for a, b in expect:
        adj[a].add(b)
        adj[b].add(a)
    for v in range(n):
        assert hg.adj[hg.adj_ptr[v]:hg.adj_ptr[v + 1]].tolist() == sorted(adj[v])
        nets_v = [j for j, e in enumerate(expect) if v in e]
        assert hg.vnets[hg.vtx_ptr[v]:hg.vtx_ptr[v + 1]].tolist() == nets_v


@pytest.mark.parametrize("side", [2, 5, 16])
def test_grid_edge_counts_closed_form(oracle_mod, side):
    O = oracle_mod
    g2 = O.build_from_matrix("symmetric", W.grid_laplacian_2d(side))
    assert g2.l == 2 * side * (side - 1)
    g3 = O.build_from_matrix("symmetric", W.grid_laplacian_3d(side))
    assert g3.l == 3 * side * side * (side - 1)


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_components_match_bfs(oracle_mod, seed):
    """Algorithm 1 labels every vertex with the smallest id of its component;
    compared with scipy's breadth-first components."""
    O = oracle_mod
    n = 300
    A = W.random_symmetric(n, 1.8, seed)  # sparse: many components
    hg = O.build_from_matrix("symmetric", A)
    lab = O.components(hg)
    M = sparse.csr_matrix((np.ones(A.nnz), A.colidx, A.rowptr), shape=(n, n))
    nc, comp = csgraph.connected_components(M, directed=False)
    canon = np.full(nc, n)
    for v in range(n):
        canon[comp[v]] = min(canon[comp[v]], v)
    assert (lab == canon[comp]).all()
    assert nc > 1


def test_components_hypergraph_nets(oracle_mod):
    O = oracle_mod
    A = W.random_pattern(60, 25, 40, 3)
    hg = O.build_from_matrix("colnet", A)   # vertices = rows, nets = columns
    lab = O.components(hg)
    # rows connected iff they share a column, transitively
    B = sparse.csr_matrix((np.ones(A.nnz), A.colidx, A.rowptr), shape=(A.m, A.n))
    G = (B @ B.T) > 0
    nc, comp = csgraph.connected_components(G, directed=False)
    canon = np.full(nc, A.m)
    for v in range(A.m):
        canon[comp[v]] = min(canon[comp[v]], v)
    assert (lab == canon[comp]).all()


def test_finegrain_model_definition(oracle_mod):
    """Finegrain model (Table 1): one vertex per distinct entry (row-major),
    the m row nets then the n column nets; equal to a plain construction from
    a pattern with duplicate entries, every vertex on exactly its row's and
    its column's net, and the dual is the bipartite graph (one net
    {r_i, c_j} per entry)."""
    O = oracle_mod
    A = W.random_pattern(23, 31, 140, 9)
    m, n = A.m, A.n
    rows = np.repeat(np.arange(m), np.diff(A.rowptr))
    cols = A.colidx
    # the same pattern given with every entry twice, rows reversed in order
    rr = np.concatenate([rows[::-1], rows])
    cc = np.concatenate([cols[::-1], cols])
    o = np.lexsort((np.arange(len(rr)), rr))
    rp = np.zeros(m + 1, dtype=np.int32)
    rp[1:] = np.cumsum(np.bincount(rr, minlength=m))
    fg = O.build_hypergraph("finegrain", m, n, rp, cc[o])
    entries = sorted(set(zip(rows.tolist(), cols.tolist())))
    assert fg.k == len(entries) and fg.l == m + n
    want = [[t for t, (i, _) in enumerate(entries) if i == r] for r in range(m)] + \
           [[t for t, (_, j) in enumerate(entries) if j == c] for c in range(n)]
    assert _nets(fg.net_ptr, fg.pins) == [list(e) for e in want]
    for t, (i, j) in enumerate(entries):
        assert fg.vnets[fg.vtx_ptr[t]:fg.vtx_ptr[t + 1]].tolist() == [i, m + j]
    dptr, dpins = O.dual(fg.k, fg.l, fg.net_ptr, fg.pins)
    bp = O.build_from_matrix("bipartite", A)
    assert sorted(tuple(e) for e in _nets(dptr, dpins)) == sorted(tuple(e) for e in _nets(bp.net_ptr, bp.pins))


def test_finegrain_coords_are_edge_midpoints(oracle_mod):
    """Finegrain layout from the bipartite one (Sec. 4.2): entry t lies at the
    midpoint of the bipartite edge it is dual to (the bipartite nets are listed
    in the same row-major order); an entry whose row and column share a point
    lies on it."""
    O = oracle_mod
    A = W.random_pattern(40, 35, 300, 4)
    bp = O.build_from_matrix("bipartite", A)
    fg = O.build_from_matrix("finegrain", A)
    xb = O.init_coords(bp.k, 3, 4)
    xf = O.finegrain_coords(fg, xb)
    ends = bp.pins.reshape(-1, 2)
    mid = 0.5 * (xb[ends[:, 0]].astype(np.float64) + xb[ends[:, 1]].astype(np.float64))
    assert np.array_equal(xf, mid)
    xb2 = xb.copy()
    xb2[A.m:] = xb2[np.arange(A.n) % A.m]  # column j at row j's point (j < m)
    xf2 = O.finegrain_coords(fg, xb2)
    same = fg.vnets[0::2] == (fg.vnets[1::2] - A.m)
    assert same.any()
    assert np.array_equal(xf2[same], xb2[fg.vnets[0::2][same]].astype(np.float64))
