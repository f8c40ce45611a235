"""Pins of the oracle's layout (Sec. 2): gradient against finite differences of
the energy and against an all-pairs sum, closed forms of the attraction term,
the grid-pyramid bookkeeping, the step rule and the multilevel coarsening."""
import numpy as np
import pytest
from scipy import sparse

import workloads as W


def _hg(O, A, model="symmetric"):
    return O.build_from_matrix(model, A)


def _exact_repulsion(x, d, w=None):
    """All-pairs repulsion part of eq. graphenergygradientsimple (kappa = d-2,
    1 for the d = 2 logarithmic reading), written with numpy broadcasting."""
    k = x.shape[0]
    w = np.ones(k) if w is None else w
    D = x[None, :, :d] - x[:, None, :d]          # D[n, i] = x_i - x_n
    r2 = (D ** 2).sum(-1)
    np.fill_diagonal(r2, np.inf)
    kap = 1.0 if d == 2 else d - 2.0
    g = kap * w[None, :] * w[:, None] * r2 ** (-0.5 * d)
    out = np.zeros((k, 4))
    out[:, :d] = (g[:, :, None] * D).sum(1)
    return out


@pytest.mark.parametrize("d", [2, 3, 4])
def test_gradient_matches_finite_differences(oracle_mod, d):
    O = oracle_mod
    A = W.grid_laplacian_2d(6)
    hg = _hg(O, A)
    x = O.init_coords(hg.k, d, 11).astype(np.float64)
    y, _, L, _, _ = O.gradient(hg, d, x, occ=10 ** 6)
    assert L == 1
    h = 1e-6
    for n in range(0, hg.k, 5):
        for m in range(d):
            xp = x.copy(); xp[n, m] += h
            xm = x.copy(); xm[n, m] -= h
            fd = (O.energy(hg, d, xp) - O.energy(hg, d, xm)) / (2 * h)
            assert abs(fd - y[n, m]) <= 1e-5 * (1 + abs(y[n, m]))


@pytest.mark.parametrize("d", [2, 3, 4])
def test_single_level_grid_equals_all_pairs(oracle_mod, d):
    """With L = 1 every cell is adjacent to every other, so the approximation
    reduces to the exact O(k^2) sum; the attraction of 2-pin nets is half the
    graph Laplacian times x."""
    O = oracle_mod
    A = W.random_symmetric(50, 5, 3)
    hg = _hg(O, A)
    rng = np.random.default_rng(0)
    x = np.zeros((hg.k, 4)); x[:, :d] = rng.standard_normal((hg.k, d)) * 3
    w = rng.uniform(0.5, 2.0, hg.k)
    y, _, L, _, _ = O.gradient(hg, d, x, occ=10 ** 6, w=w)
    assert L == 1
    Adj = sparse.csr_matrix((np.ones(len(hg.adj)), hg.adj, hg.adj_ptr), shape=(hg.k, hg.k))
    Lap = sparse.diags(np.asarray(Adj.sum(1)).ravel()) - Adj
    att = 0.5 * (Lap @ x)
    expect = att + _exact_repulsion(x, d, w)
    assert np.allclose(y, expect, rtol=1e-10, atol=1e-10)


def test_two_points_closed_form(oracle_mod):
    O = oracle_mod
    for d in (2, 3, 4):
        A = W.csr_from_coo(2, 2, np.array([0, 1]), np.array([0, 1]), "two")
        hg = _hg(O, A)      # no edges: repulsion only
        x = np.zeros((2, 4)); x[1, :d] = 2.0
        y, *_ = O.gradient(hg, d, x, occ=1)
        r = 2.0 * np.sqrt(d)
        kap = 1.0 if d == 2 else d - 2.0
        mag = kap * r ** (-d) * 2.0   # |x_1 - x_0|_m = 2
        assert np.allclose(y[0, :d], mag) and np.allclose(y[1, :d], -mag)


def test_gamma2_cancellation_hypergraph_nets(oracle_mod):
    """gamma = 2 (Sec. 2.1): the attraction on vertex n is sum_j c_j (x_n - z_j);
    for a linear coordinate field on a grid it vanishes at interior vertices,
    and summed over all vertices it vanishes (sum_{i in e} (x_i - z_e) = 0)."""
    O = oracle_mod
    s = 9
    A = W.grid_laplacian_2d(s)
    hg = _hg(O, A)
    ij = np.indices((s, s)).reshape(2, -1).T.astype(np.float64)
    x = np.zeros((hg.k, 4)); x[:, :2] = ij * np.array([1.5, -0.5])
    # far apart copy to isolate attraction: compare gradient with and without nets
    empty = O.build_from_matrix("symmetric", W.csr_from_coo(hg.k, hg.k, np.arange(hg.k), np.arange(hg.k), "diag"))
    y, *_ = O.gradient(hg, 2, x)
    y0, *_ = O.gradient(empty, 2, x)
    att = y - y0
    interior = [(i * s + j) for i in range(1, s - 1) for j in range(1, s - 1)]
    assert np.abs(att[interior]).max() < 1e-12
    assert np.abs(att.sum(0)).max() < 1e-10
    # general hypergraph nets (column-net model): sum over vertices is zero too
    B = W.random_pattern(30, 12, 80, 4)
    hc = O.build_from_matrix("colnet", B)
    xr = np.random.default_rng(1).standard_normal((hc.k, 4)); xr[:, 3] = 0
    e0 = O.build_from_matrix("colnet", W.csr_from_coo(30, 1, np.array([], int), np.array([], int), "e"))
    ya, *_ = O.gradient(hc, 3, xr)
    yb, *_ = O.gradient(e0, 3, xr)
    assert np.abs((ya - yb).sum(0)).max() < 1e-10


@pytest.mark.parametrize("d,k", [(2, 3000), (3, 3000), (4, 2500)])
def test_every_source_counted_once(oracle_mod, d, k):
    """Near field plus far-field charges cover every other vertex exactly once:
    the source weight seen by each target equals sum(w) - w_n."""
    O = oracle_mod
    A = W.csr_from_coo(k, k, np.arange(k), np.arange(k), "iso")
    hg = _hg(O, A)
    rng = np.random.default_rng(d)
    x = np.zeros((k, 4)); x[:, :d] = rng.standard_normal((k, d)) ** 3  # clustered, uneven
    w = rng.integers(1, 4, k).astype(np.float64)
    y, keys, L, ninter, wseen = O.gradient(hg, d, x, w=w)
    assert L >= 3
    assert np.array_equal(wseen, w.sum() - w)
    assert (ninter < k - 1).all()       # the far field really groups sources


@pytest.mark.parametrize("d", [2, 3])
def test_far_field_error_small_and_translation_invariant(oracle_mod, d):
    O = oracle_mod
    k = 2000
    A = W.csr_from_coo(k, k, np.arange(k), np.arange(k), "iso")
    hg = _hg(O, A)
    rng = np.random.default_rng(7)
    x = np.zeros((k, 4)); x[:, :d] = rng.uniform(0, 20, (k, d))
    y, _, L, _, _ = O.gradient(hg, d, x)
    ex = _exact_repulsion(x, d)
    rel = np.linalg.norm(y - ex) / np.linalg.norm(ex)
    assert L >= 3 and rel < 0.05
    # translation invariance (Sec. 2.1 observation 3); cells are relative to the box
    shift = np.zeros(4); shift[:d] = 2.0 ** 5  # exact in fp32, so the cells do not move
    y2, *_ = O.gradient(hg, d, x + shift)
    assert np.allclose(y2, y, rtol=1e-9, atol=1e-9)
    # axis permutation permutes the gradient
    if d == 3:
        p = [1, 2, 0, 3]
        y3, *_ = O.gradient(hg, d, x[:, p])
        assert np.allclose(y3, y[:, p], rtol=1e-9, atol=1e-9)


def test_keys_locate_points(oracle_mod):
    """The level-L key of a vertex (row-major cell index) decodes to the fp32
    cell containing it."""
    O = oracle_mod
    k, d = 5000, 3
    A = W.csr_from_coo(k, k, np.arange(k), np.arange(k), "iso")
    hg = _hg(O, A)
    x = np.zeros((k, 4)); x[:, :d] = np.random.default_rng(2).uniform(-3, 9, (k, d))
    _, keys, L, _, _ = O.gradient(hg, d, x)
    assert L == O.levels(k, d)
    assert 8 * 2 ** (d * L) >= k > 8 * 2 ** (d * (L - 1))
    xf = x.astype(np.float32)[:, :d]
    lo, hi = xf.min(0), xf.max(0)
    E = float((hi - lo).max())
    c = np.zeros((k, d), dtype=np.int64)
    for m in range(d):
        c[:, m] = (keys.astype(np.int64) >> (L * m)) & ((1 << L) - 1)
    cell = E / 2 ** L
    pos = (xf.astype(np.float64) - lo) / cell
    assert (c <= np.floor(pos) + 1e-6).all() and (pos - c < 1 + 1e-5).all()
    assert c.max() == 2 ** L - 1 and c.min() == 0


def test_step_rule_moves_each_vertex_by_step(oracle_mod):
    O = oracle_mod
    A = W.grid_laplacian_2d(12)
    hg = _hg(O, A)
    x = O.init_coords(hg.k, 2, 5).astype(np.float64)
    s0 = O.step0(hg.k, 2, x)
    lo, hi = x[:, :2].min(0), x[:, :2].max(0)
    assert np.isclose(s0, np.sqrt(np.prod(hi - lo)) / np.sqrt(hg.k))
    xn, y, keys, L = O.layout_step(hg, 2, x, 0.25)
    disp = np.linalg.norm((xn - x)[:, :2], axis=1)
    assert np.allclose(disp, 0.25)
    # moves are along -y
    cos = ((x - xn)[:, :2] * y[:, :2]).sum(1) / (disp * np.linalg.norm(y[:, :2], axis=1))
    assert np.allclose(cos, 1.0)


@pytest.mark.parametrize("d", [2, 3])
def test_small_step_decreases_energy(oracle_mod, d):
    """Steepest descent (Sec. 2.3): a small step along -y lowers the energy."""
    O = oracle_mod
    A = W.grid_laplacian_2d(7)
    hg = _hg(O, A)
    x = O.init_coords(hg.k, d, 2).astype(np.float64)
    f0 = O.energy(hg, d, x)
    y, *_ = O.gradient(hg, d, x, occ=10 ** 6)
    f1 = O.energy(hg, d, x - 1e-4 * y)
    assert f1 < f0


def test_matching_structure(oracle_mod):
    """Coarsening groups (Algorithm 3): matched pairs are edges and mutual; every
    unmatched single-neighbour vertex shares its neighbour's group; coarse ids
    follow the anchors; every group is connected."""
    O = oracle_mod
    A = W.powerlaw_symmetric(2000, seed=4)
    hg = _hg(O, A)
    cost = np.ones(len(hg.adj))
    kc, mate, pi = O.match(hg.k, hg.adj_ptr, hg.adj, cost, seed=3)
    k = hg.k
    assert kc == pi.max() + 1 and set(np.unique(pi)) == set(range(kc))
    nbrs = [set(hg.adj[hg.adj_ptr[v]:hg.adj_ptr[v + 1]].tolist()) for v in range(k)]
    for v in range(k):
        if mate[v] >= 0:
            assert mate[mate[v]] == v and mate[v] in nbrs[v] and pi[v] == pi[mate[v]]
        elif len(nbrs[v]) == 1:
            (u,) = nbrs[v]
            assert pi[v] == pi[u]
    anchors = []
    for g in range(kc):
        mem = np.flatnonzero(pi == g)
        sub = sparse.csr_matrix((np.ones(len(hg.adj)), hg.adj, hg.adj_ptr), shape=(k, k))[mem][:, mem]
        from scipy.sparse import csgraph
        assert csgraph.connected_components(sub, directed=False)[0] == 1
        paired = [v for v in mem if mate[v] >= 0]
        anchors.append(min(paired) if paired else (mem[0] if len(mem) == 1 else
                                                     [v for v in mem if len(nbrs[v]) != 1 or mate[v] >= 0][0]))
    assert anchors == sorted(anchors)
    assert kc < 0.7 * k


def test_matching_prefers_heavy_edges(oracle_mod):
    """A vertex whose heaviest edge leads to a vertex that also prefers it is
    matched along that edge."""
    O = oracle_mod
    # path 0-1-2-3 with costs 1, 5, 1: 1 and 2 must match
    ptr = np.array([0, 1, 3, 5, 6]); adj = np.array([1, 0, 2, 1, 3, 2])
    cost = np.array([1.0, 1.0, 5.0, 5.0, 1.0, 1.0])
    kc, mate, pi = O.match(4, ptr, adj, cost, seed=1)
    assert mate[1] == 2 and mate[2] == 1
    # 0 and 3 are single-neighbour vertices: they join their neighbours' group
    assert kc == 1 and (pi == 0).all()


def test_hierarchy_shrinks(oracle_mod):
    O = oracle_mod
    hg = _hg(O, W.grid_laplacian_2d(64))
    ks = O.hierarchy(hg, 1)
    assert ks[0] == 4096 and ks[-1] <= 64
    assert all(b <= 0.95 * a for a, b in zip(ks, ks[1:]))


def test_threads_do_not_change_results(oracle_mod):
    """The per-vertex gradient loop runs on several threads when the oracle is
    built with OpenMP; every vertex's sums stay one thread's, in order, so a
    layout is bit-identical for 1 and 4 threads."""
    O = oracle_mod
    A = W.powerlaw_symmetric(3000, seed=5)
    hg = _hg(O, A)
    before = O.threads()
    try:
        O.set_threads(1)
        x1 = O.layout_multilevel(hg, 3, seed=2, iters=10)
        O.set_threads(4)
        x4 = O.layout_multilevel(hg, 3, seed=2, iters=10)
    finally:
        O.set_threads(before)
    assert np.array_equal(x1.view(np.uint64), x4.view(np.uint64))
