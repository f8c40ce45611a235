"""Pins of the oracle's partitioning and ordering (Sec. 3 and 4): exhaustive
2-means optima, k-means++ sampling, the separator postconditions of Algorithm 7
and its order-free equivalent, the recursive BBD/SBD structure, brute-force cut
counts and the fill-in example."""
import itertools
import json
import os

import numpy as np
import pytest

import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _x4(pts):
    x = np.zeros((len(pts), 4), dtype=np.float32)
    x[:, :pts.shape[1]] = pts
    return x


def _kmeans_cost(pts, lab):
    c = 0.0
    for s in (1, 2):
        p = pts[lab == s]
        if len(p):
            c += ((p - p.mean(0)) ** 2).sum()
    return c


def _best_split(pts):
    k = len(pts)
    best, arg = np.inf, None
    for mask in range(1, 2 ** (k - 1)):
        lab = np.array([1 + ((mask >> i) & 1) for i in range(k)])
        c = _kmeans_cost(pts, lab)
        if c < best:
            best, arg = c, lab
    return best, arg


@pytest.mark.parametrize("seed", range(6))
def test_two_means_optimal_on_separated_clusters(oracle_mod, seed):
    """eq. kmeans: on two well separated clusters (k <= 14) the oracle's 2-means
    finds the exhaustive optimum."""
    O = oracle_mod
    rng = np.random.default_rng(seed)
    d = 2 + seed % 3
    k1 = rng.integers(2, 8)
    k2 = rng.integers(2, 7)
    pts = np.concatenate([rng.normal(0, 1, (k1, d)), rng.normal(12, 1, (k2, d))]).astype(np.float32)
    best, lab_opt = _best_split(pts.astype(np.float64))
    ok, lab, z1, z2 = O.bisect(d, _x4(pts), np.arange(len(pts)), seed=seed, key=1)
    assert ok
    same = np.array_equal(lab, lab_opt) or np.array_equal(lab, 3 - lab_opt)
    assert same
    assert np.isclose(_kmeans_cost(pts.astype(np.float64), lab), best, rtol=1e-6)


@pytest.mark.parametrize("seed", range(8))
def test_two_means_lloyd_fixed_point_and_bound(oracle_mod, seed):
    """On arbitrary points: the result is never better than the exhaustive
    optimum, its labels are nearest-centre labels of its centres, and (when
    converged) the centres are the means of their clusters."""
    O = oracle_mod
    rng = np.random.default_rng(100 + seed)
    d = 2 + seed % 3
    pts = rng.uniform(0, 10, (12, d)).astype(np.float32)
    best, _ = _best_split(pts.astype(np.float64))
    ok, lab, z1, z2 = O.bisect(d, _x4(pts), np.arange(12), seed=seed, key=1, km_iters=50)
    assert ok
    assert _kmeans_cost(pts.astype(np.float64), lab) >= best * (1 - 1e-9)
    d1 = ((pts - z1[:d]) ** 2).sum(1)
    d2 = ((pts - z2[:d]) ** 2).sum(1)
    assert np.array_equal(lab == 1, d1 <= d2)
    assert np.allclose(z1[:d], pts[lab == 1].mean(0), atol=1e-5)
    assert np.allclose(z2[:d], pts[lab == 2].mean(0), atol=1e-5)


def test_two_means_collinear_matches_sorted_scan(oracle_mod):
    """1-D inputs: the optimal 2-split is a threshold in sorted order."""
    O = oracle_mod
    rng = np.random.default_rng(3)
    for _ in range(5):
        v = np.concatenate([rng.normal(0, 1, 30), rng.normal(8, 1, 25)]).astype(np.float32)
        s = np.sort(v.astype(np.float64))
        costs = [((s[:i] - s[:i].mean()) ** 2).sum() + ((s[i:] - s[i:].mean()) ** 2).sum()
                 for i in range(1, len(s))]
        best = min(costs)
        pts = v[:, None]
        ok, lab, *_ = O.bisect(2, _x4(np.concatenate([pts, np.zeros_like(pts)], 1)),
                               np.arange(len(v)), seed=1)
        assert ok and np.isclose(_kmeans_cost(v[:, None].astype(np.float64), lab), best, rtol=1e-9)


def test_kmeanspp_second_centre_distribution(oracle_mod):
    """Algorithm 5: z2 = x_i with probability d_i / sum d.  Over many draws (node
    keys) the empirical frequencies match the D^2 weights."""
    O = oracle_mod
    pts = np.array([[0, 0], [1, 0], [3, 0], [0, 2], [4, 4]], dtype=np.float32)
    x4 = _x4(pts)
    counts = np.zeros((5, 5))
    N = 20000
    for key in range(N):
        _, _, z1, z2 = O.bisect(2, x4, np.arange(5), seed=9, key=key, km_iters=0)
        i0 = int(np.flatnonzero((pts == z1[:2]).all(1))[0])
        i1 = int(np.flatnonzero((pts == z2[:2]).all(1))[0])
        counts[i0, i1] += 1
    first = counts.sum(1) / N
    assert np.allclose(first, 0.2, atol=0.02)
    for i0 in range(5):
        dd = ((pts - pts[i0]) ** 2).sum(1).astype(np.float64)
        p = dd / dd.sum()
        emp = counts[i0] / counts[i0].sum()
        assert np.abs(emp - p).max() < 0.04


def test_kmeanspp_expected_cost_bound(oracle_mod):
    """k-means++ seeding is O(log m)-competitive in expectation (Sec. 3): the mean
    seeding cost over many draws stays below 8 (ln 2 + 2) times the optimum."""
    O = oracle_mod
    rng = np.random.default_rng(5)
    pts = rng.uniform(0, 1, (12, 2)).astype(np.float32)
    best, _ = _best_split(pts.astype(np.float64))
    costs = []
    for key in range(400):
        _, lab, z1, z2 = O.bisect(2, _x4(pts), np.arange(12), seed=2, key=key, km_iters=0)
        d1 = ((pts - z1[:2]) ** 2).sum(1)
        d2 = ((pts - z2[:2]) ** 2).sum(1)
        costs.append(np.minimum(d1, d2).sum())
    assert np.mean(costs) <= 8 * (np.log(2) + 2) * best


def _ancestor(h1, d1, h2, d2):
    return d1 <= d2 and (int(h2) >> (d2 - d1)) == int(h1)


def _owner_info(k, perm, tree, sbd):
    """owner index, heap and depth of every vertex."""
    part = np.full(k, -1)
    for idx in range(len(tree["heap"])):
        o, n1, n2, ns = (int(tree[f][idx]) for f in ("offset", "n1", "n2", "nsep"))
        if n2 == 0 and ns == 0:
            part[perm[o:o + n1]] = idx
        else:
            so = o + n1 if sbd else o + n1 + n2
            part[perm[so:so + ns]] = idx
    return part


def _check_ordering(O, A, hg, perm, tree, sbd, d=None, x4=None, min_part=64, max_depth=62):
    k = hg.k
    assert sorted(perm.tolist()) == list(range(k))
    key = [(int(c), int(h)) for c, h in zip(tree["comp"], tree["heap"])]
    assert key == sorted(key) and len(set(key)) == len(key)
    part = _owner_info(k, perm, tree, sbd)
    assert (part >= 0).all()
    H, D = tree["heap"], tree["depth"]
    # every edge lies in a diagonal block or a border: owners are nested
    for v in range(k):
        for u in hg.adj[hg.adj_ptr[v]:hg.adj_ptr[v + 1]]:
            a, b = part[v], part[u]
            assert _ancestor(H[a], D[a], H[b], D[b]) or _ancestor(H[b], D[b], H[a], D[a])
    # tree bookkeeping: children of node h are 2h / 2h+1 at the right offsets
    idx = {(int(c), int(h)): i for i, (c, h) in enumerate(zip(tree["comp"], H))}
    for i, h in enumerate(H):
        cmp_ = int(tree["comp"][i])
        o, n1, n2, ns, dp = (int(tree[f][i]) for f in ("offset", "n1", "n2", "nsep", "depth"))
        leaf = n2 == 0 and ns == 0
        if leaf:
            continue
        if n1:
            c = idx[(cmp_, 2 * int(h))]
            assert tree["offset"][c] == o and tree["depth"][c] == dp + 1
        if n2:
            c = idx[(cmp_, 2 * int(h) + 1)]
            assert tree["offset"][c] == (o + n1 + ns if sbd else o + n1)
        assert dp < max_depth
    # leaves are small, deep or unsplittable
    return part


@pytest.mark.parametrize("sbd", [False, True])
def test_order_true_grid_coordinates(oracle_mod, sbd):
    """With the grid's own coordinates (Example pothen: given geometry) the root
    separator of a 64x64 grid is one grid line of 64 vertices."""
    O = oracle_mod
    A = W.grid_laplacian_2d(64)
    hg = O.build_from_matrix("symmetric", A)
    ij = np.indices((64, 64)).reshape(2, -1).T
    x4 = _x4(ij.astype(np.float32))
    perm, tree = O.order(hg, 2, x4, seed=1, sbd=sbd)
    assert tree["heap"][0] == 1 and tree["nsep"][0] == 64
    assert tree["n1"][0] + tree["n2"][0] + tree["nsep"][0] == 4096
    _check_ordering(O, A, hg, perm, tree, sbd)
    if not sbd:
        assert O.fill_in(A, perm) < 0.5 * O.fill_in(A, np.arange(A.n, dtype=np.int32))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_order_random_structure(oracle_mod, seed):
    O = oracle_mod
    A = W.powerlaw_symmetric(1500, seed=seed)
    hg = O.build_from_matrix("symmetric", A)
    x4 = O.init_coords(hg.k, 3, seed)
    for sbd in (False, True):
        perm, tree = O.order(hg, 3, x4, seed=seed, min_part=16, sbd=sbd)
        _check_ordering(O, A, hg, perm, tree, sbd)
        leaves = (tree["n2"] == 0) & (tree["nsep"] == 0)
        assert leaves.sum() >= 2


def test_order_depth_limit_and_bipartite_sbd(oracle_mod):
    """SBD on the bipartite model to 2^depth parts: no nonzero in the blocks
    (R1, C2) and (R2, C1) of any split."""
    O = oracle_mod
    A = W.powerlaw_rectangular(300, 200, seed=3)
    hg = O.build_from_matrix("bipartite", A)
    x4 = O.init_coords(hg.k, 2, 4)
    perm, tree = O.order(hg, 2, x4, seed=4, min_part=1, max_depth=3, sbd=True)
    assert tree["depth"].max() <= 3
    part = _check_ordering(O, A, hg, perm, tree, True, max_depth=3)
    assert ((tree["depth"] < 3) | ((tree["n2"] == 0) & (tree["nsep"] == 0))).all()


def _separator_order_free(hg, d, x4, verts, lab, z1, z2):
    """Order-free rule: v joins the separator iff a neighbour w in the node has
    the other label and (s(v), v) < (s(w), w), s from the fp32 plane."""
    f = np.float32
    r = (z2 - z1).astype(np.float32)
    delta = f(0)
    for m in range(d):
        delta = f(delta + f(f(f(0.5) * f(z1[m] + z2[m])) * r[m]))

    def s(v):
        acc = f(0)
        for m in range(d):
            acc = f(acc + f(x4[v, m] * r[m]))
        return abs(f(acc - delta))

    innode = {int(v): int(l) for v, l in zip(verts, lab)}
    out = dict(innode)
    for v, lv in innode.items():
        for w in hg.adj[hg.adj_ptr[v]:hg.adj_ptr[v + 1]]:
            w = int(w)
            if w in innode and innode[w] != lv and (s(v), v) < (s(w), w):
                out[v] = 3
                break
    return out


@pytest.mark.parametrize("seed", range(5))
def test_separator_sequential_equals_order_free(oracle_mod, seed):
    """The oracle runs Algorithm 7's edge loop in the canonical order; the
    parallel rule the GPU uses gives the same separator, and the result has no
    edge between V1 and V2 (Algorithm 7 postcondition)."""
    O = oracle_mod
    A = W.random_symmetric(400, 9, seed)
    hg = O.build_from_matrix("symmetric", A)
    x4 = O.init_coords(hg.k, 3, seed)
    # root only: redo its 2-means, then compare the separator
    ok, lab, z1, z2 = O.bisect(3, x4, np.arange(hg.k), seed=seed, key=1)
    assert ok
    perm, tree = O.order(hg, 3, x4, seed=seed, min_part=1, max_depth=1)
    n1, n2, ns = int(tree["n1"][0]), int(tree["n2"][0]), int(tree["nsep"][0])
    V1, V2, V3 = set(perm[:n1].tolist()), set(perm[n1:n1 + n2].tolist()), set(perm[n1 + n2:].tolist())
    rule = _separator_order_free(hg, 3, x4, np.arange(hg.k), lab, z1, z2)
    assert {v for v, l in rule.items() if l == 3} == V3
    assert {v for v, l in rule.items() if l == 1} == V1
    for v in V1:
        assert not (set(hg.adj[hg.adj_ptr[v]:hg.adj_ptr[v + 1]].tolist()) & V2)
    # the stable partition keeps the original relative order
    assert (np.diff(perm[:n1]) > 0).all() and (np.diff(perm[n1:n1 + n2]) > 0).all()


def test_separator_replay_matches_bisect(oracle_mod):
    """Each split of the ordering equals a standalone 2-means of the node's
    vertices (in node order, keyed by the node's heap number)."""
    O = oracle_mod
    A = W.grid_laplacian_3d(12)
    hg = O.build_from_matrix("symmetric", A)
    x4 = O.init_coords(hg.k, 3, 8)
    perm, tree = O.order(hg, 3, x4, seed=8, min_part=32, max_depth=4)
    # the child 2 of the root holds V2 in node order; its own split is replayed
    assert (tree["comp"] == 0).all()
    idx = {int(h): i for i, h in enumerate(tree["heap"])}
    i2 = idx[3]
    o, n1, n2, ns = (int(tree[f][i2]) for f in ("offset", "n1", "n2", "nsep"))
    size = n1 + n2 + ns
    # node vertices in the order they had when the node was split = stable
    # partition of the root's V2 list, which is ascending in vertex id
    verts = np.sort(perm[o:o + size])
    ok, lab, z1, z2 = O.bisect(3, x4, verts, seed=8, key=3)
    assert ok
    assert set(perm[o:o + n1].tolist()) <= set(verts[lab == 1].tolist())
    assert set(perm[o + n1:o + n1 + n2].tolist()) <= set(verts[lab == 2].tolist())


@pytest.mark.parametrize("seed", range(4))
def test_cut_size_brute_force(oracle_mod, seed):
    O = oracle_mod
    rng = np.random.default_rng(seed)
    A = W.random_pattern(25, 17, 90, seed)
    for model in ("rownet", "colnet", "bipartite", "symmetric"):
        B = A if model != "symmetric" else W.random_pattern(25, 25, 90, seed)
        hg = O.build_from_matrix(model, B)
        nparts = int(rng.integers(2, 90))
        part = rng.integers(0, nparts, hg.k).astype(np.int32)
        cn, l1 = O.cut_size(hg.net_ptr, hg.pins, part)
        lam = [len({int(part[v]) for v in hg.pins[hg.net_ptr[j]:hg.net_ptr[j + 1]]}) for j in range(hg.l)]
        assert cn == sum(1 for x in lam if x > 1)
        assert l1 == sum(max(x - 1, 0) for x in lam)


def _dense_fill(P):
    """Symbolic LU of a dense boolean pattern without pivoting: new nonzeros."""
    n = len(P)
    F = P.copy()
    for k in range(n):
        rows = np.flatnonzero(F[k + 1:, k]) + k + 1
        cols = np.flatnonzero(F[k, k + 1:]) + k + 1
        for i in rows:
            F[i, cols] = True
    return int(F.sum() - P.sum())


def test_fill_in_example(oracle_mod):
    """Example fillin: six new nonzeros in the original order, none after
    swapping the first and last rows and columns."""
    O = oracle_mod
    g = json.load(open(os.path.join(GOLD, "fillin.json")))
    M = np.array(g["matrix"])
    r, c = np.nonzero(M)
    A = W.csr_from_coo(4, 4, r, c, "arrow")
    ident = np.arange(4, dtype=np.int32)
    nzl = O.cholesky_nnz(4, A.rowptr, A.colidx, ident)
    assert 2 * nzl - 4 - A.nnz == g["new_nonzeros_original_order"]
    sw = np.array(g["swap"], dtype=np.int32)
    nzl2 = O.cholesky_nnz(4, A.rowptr, A.colidx, sw)
    assert 2 * nzl2 - 4 - A.nnz == g["new_nonzeros_after_swap"]
    assert _dense_fill(M != 0) == g["new_nonzeros_original_order"]


@pytest.mark.parametrize("seed", range(4))
def test_cholesky_count_matches_dense_elimination(oracle_mod, seed):
    O = oracle_mod
    A = W.random_symmetric(40, 4, seed)
    perm = np.random.default_rng(seed).permutation(40).astype(np.int32)
    P = np.zeros((40, 40), dtype=bool)
    rows = np.repeat(np.arange(40), np.diff(A.rowptr))
    P[rows, A.colidx] = True
    Pp = P[np.ix_(perm, perm)]
    nzl = O.cholesky_nnz(40, A.rowptr, A.colidx, perm)
    assert 2 * nzl - 40 == Pp.sum() + _dense_fill(Pp)


def test_order_components_block_diagonal(oracle_mod):
    """A disconnected graph (Sec. 2.2: components are treated separately) is
    ordered component after component, in order of smallest vertex id, each by
    its own recursion; isolated vertices are single-vertex leaves."""
    O = oracle_mod
    A = W.powerlaw_symmetric(3000, seed=1)
    hg = O.build_from_matrix("symmetric", A)
    lab = O.components(hg)
    comps = np.unique(lab)
    assert len(comps) > 1
    x4 = O.init_coords(hg.k, 3, 2)
    perm, tree = O.order(hg, 3, x4, seed=2, min_part=16)
    part = _check_ordering(O, A, hg, perm, tree, False)
    # component blocks are contiguous and in order of their smallest vertex
    assert (np.diff(lab[perm]) >= 0).all()
    roots = tree["heap"] == 1
    assert roots.sum() == len(comps)
    sizes = np.bincount(np.searchsorted(comps, lab))
    assert np.array_equal(np.sort(tree["n1"][roots & (tree["n2"] == 0) & (tree["nsep"] == 0)]),
                          np.sort(sizes[sizes <= 16]))


def test_multilevel_layout_of_components_is_independent(oracle_mod):
    """Each component is laid out on its own: adding an isolated vertex with a
    larger id leaves the layout of the rest unchanged."""
    O = oracle_mod
    A = W.grid_laplacian_2d(12)
    rows = np.repeat(np.arange(A.m), np.diff(A.rowptr))
    B = W.csr_from_coo(A.m + 1, A.n + 1, np.concatenate([rows, [A.m]]), np.concatenate([A.colidx, [A.m]]), "iso")
    ha = O.build_from_matrix("symmetric", A)
    hb = O.build_from_matrix("symmetric", B)
    xa = O.layout_multilevel(ha, 2, 5)
    xb = O.layout_multilevel(hb, 2, 5)
    assert np.array_equal(xa, xb[:A.m])


def _parent3(h):
    return (int(h) + 1) // 3


def _branch3(h):
    """0, 1, 2 for the V1, V2, V3 child of its parent (keys 3p-1, 3p, 3p+1)."""
    return int(h) - (3 * _parent3(h) - 1)


@pytest.mark.parametrize("sbd", [False, True])
def test_sep_recursion_separator_of_grid_separator(oracle_mod, sbd):
    """Separator recursion (the additional freedom of Sec. 4.2) on a 64x64 grid
    with its own coordinates: the root separator is one grid line, a path of
    64 vertices, and the separator of a path is a single vertex: the V3 child
    of the root (key 4) splits 32 / 31 / 1, at the offset of the separator
    block (after V1 and V2 in BBD, between them in SBD)."""
    O = oracle_mod
    A = W.grid_laplacian_2d(64)
    hg = O.build_from_matrix("symmetric", A)
    ij = np.indices((64, 64)).reshape(2, -1).T
    perm, tree = O.order(hg, 2, _x4(ij.astype(np.float32)), seed=1, sbd=sbd, sep_rec=True, min_part=8)
    H = [int(h) for h in tree["heap"]]
    n1, n2, ns = (int(tree[f][0]) for f in ("n1", "n2", "nsep"))
    assert H[0] == 1 and ns == 64 and n1 + n2 + ns == 4096
    j = H.index(4)
    assert tree["offset"][j] == (n1 if sbd else n1 + n2)
    assert sorted((int(tree["n1"][j]), int(tree["n2"][j]))) == [31, 32] and tree["nsep"][j] == 1
    # its three children are there too (keys 11, 12, 13)
    assert {11, 12, 13} <= set(H)


def test_sep_recursion_nesting(oracle_mod):
    """Separator recursion on a power-law graph: a permutation; every split
    node's three children at the right keys, offsets and sizes; and every edge
    lies in a diagonal block or a border: below the lowest common node of its
    two ends' owners, the ends are never one in the V1 branch and one in the V2
    branch."""
    O = oracle_mod
    A = W.powerlaw_symmetric(3000, seed=21)
    hg = O.build_from_matrix("symmetric", A)
    x4 = O.init_coords(hg.k, 2, 21)
    for sbd in (False, True):
        perm, tree = O.order(hg, 2, x4, seed=3, sbd=sbd, sep_rec=True, min_part=4)
        k = hg.k
        assert sorted(perm.tolist()) == list(range(k))
        idx = {(int(c), int(h)): i for i, (c, h) in enumerate(zip(tree["comp"], tree["heap"]))}
        owner = np.full(k, -1)
        for i in range(len(tree["heap"])):
            o, n1, n2, ns, dp = (int(tree[f][i]) for f in ("offset", "n1", "n2", "nsep", "depth"))
            c, h = int(tree["comp"][i]), int(tree["heap"][i])
            if n2 == 0 and ns == 0:
                owner[perm[o:o + n1]] = i
                continue
            for side, (size, off) in enumerate(((n1, o), (n2, o + n1 + ns if sbd else o + n1),
                                                 (ns, o + n1 if sbd else o + n1 + n2))):
                if size:
                    ch = idx[(c, 3 * h - 1 + side)]
                    assert tree["offset"][ch] == off and tree["depth"][ch] == dp + 1
                    cs = int(tree["n1"][ch]) + int(tree["n2"][ch]) + int(tree["nsep"][ch])
                    assert cs == size
        assert (owner >= 0).all()
        H, D, Cm = tree["heap"], tree["depth"], tree["comp"]

        def path(i):
            h, d, out = int(H[i]), int(D[i]), []
            while d > 0:
                out.append(h)
                h, d = _parent3(h), d - 1
            return out[::-1]  # keys from depth 1 down

        for v in range(k):
            for u in hg.adj[hg.adj_ptr[v]:hg.adj_ptr[v + 1]]:
                a, b = owner[v], owner[u]
                assert Cm[a] == Cm[b]
                pa, pb = path(a), path(b)
                m = 0
                while m < min(len(pa), len(pb)) and pa[m] == pb[m]:
                    m += 1
                if m < len(pa) and m < len(pb):
                    assert {_branch3(pa[m]), _branch3(pb[m])} != {0, 1}


# ---------------------------------------------------------------- m-way k-means++ (Algorithm 5, m centres)
def _best_mway(pts, m):
    """Exhaustive minimum of eq. kmeans over all m-labelings (small k)."""
    k = len(pts)
    best = np.inf
    for lab in itertools.product(range(m), repeat=k):
        lab = np.array(lab)
        if len(set(lab.tolist())) < m:
            continue
        c = sum(((pts[lab == j] - pts[lab == j].mean(0)) ** 2).sum() for j in range(m))
        best = min(best, c)
    return best


def _cost_m(pts, lab, m):
    return sum(((pts[lab == j] - pts[lab == j].mean(0)) ** 2).sum() for j in range(m) if (lab == j).any())


@pytest.mark.parametrize("seed", range(12))
def test_kmeans_m2_equals_two_means(oracle_mod, seed):
    """For m = 2 the m-way k-means++ is exactly the pinned 2-means (same draws,
    same Lloyd rounds): labels 0 / 1 for 1 / 2 and the same centres."""
    O = oracle_mod
    rng = np.random.default_rng(300 + seed)
    d = 2 + seed % 3
    n = int(rng.integers(2, 400))
    pts = (rng.normal(0, 1, (n, d)) * rng.uniform(0.1, 50)).astype(np.float32)
    verts = rng.permutation(n)[: max(2, n - 3)].astype(np.int32)
    for km in (0, 3, 20):
        ok, lab2, z1, z2 = O.bisect(d, _x4(pts), verts, seed=seed, key=7 + seed, km_iters=km)
        labm, zm, ne = O.kmeans(d, _x4(pts), verts, 2, seed=seed, key=7 + seed, km_iters=km)
        assert np.array_equal(labm, lab2.astype(np.int32) - 1)
        if ok:
            assert ne == 2
            assert np.array_equal(zm[0].view(np.uint32), z1.view(np.uint32))
            assert np.array_equal(zm[1].view(np.uint32), z2.view(np.uint32))


@pytest.mark.parametrize("seed", range(6))
def test_kmeans_m3_optimal_on_separated_clusters(oracle_mod, seed):
    """Three well separated clusters (k <= 8): k-means++ finds the exhaustive
    optimum of eq. kmeans (every cluster gets a seed with high probability by
    D^2 sampling, and Lloyd keeps the clusters)."""
    O = oracle_mod
    rng = np.random.default_rng(40 + seed)
    d = 2 + seed % 3
    sizes = rng.integers(2, 4, 3)
    pts = np.concatenate([rng.normal(c * 30.0, 0.5, (s, d)) for c, s in enumerate(sizes)]).astype(np.float32)
    best = _best_mway(pts.astype(np.float64), 3)
    lab, z, ne = O.kmeans(d, _x4(pts), np.arange(len(pts)), 3, seed=seed, key=1)
    assert ne == 3
    assert np.isclose(_cost_m(pts.astype(np.float64), lab, 3), best, rtol=1e-6)


@pytest.mark.parametrize("seed", range(8))
def test_kmeans_m_lloyd_fixed_point_and_bound(oracle_mod, seed):
    """Arbitrary points, m = 3 or 4: never better than the exhaustive optimum;
    labels are the nearest centres (ties to the smaller index); converged
    centres are the means of their clusters; m = 1 gives one cluster at the
    mean."""
    O = oracle_mod
    rng = np.random.default_rng(500 + seed)
    d = 2 + seed % 3
    m = 3 + seed % 2
    k = 8 if m == 3 else 7
    pts = rng.uniform(0, 10, (k, d)).astype(np.float32)
    best = _best_mway(pts.astype(np.float64), m)
    lab, z, ne = O.kmeans(d, _x4(pts), np.arange(k), m, seed=seed, key=2, km_iters=60)
    assert _cost_m(pts.astype(np.float64), lab, m) >= best * (1 - 1e-9)
    dist = ((pts[:, None, :] - z[None, :, :d]) ** 2).sum(2)
    assert np.array_equal(lab, dist.argmin(1))
    for j in range(m):
        if (lab == j).any():
            assert np.allclose(z[j, :d], pts[lab == j].mean(0), atol=1e-5)
    lab1, z1, ne1 = O.kmeans(d, _x4(pts), np.arange(k), 1, seed=seed, key=2)
    assert ne1 == 1 and (lab1 == 0).all() and np.allclose(z1[0, :d], pts.mean(0), atol=1e-5)


def test_kmeanspp_m_expected_cost_bound(oracle_mod):
    """Arthur and Vassilvitskii: the seeding alone (0 Lloyd rounds) costs at most
    8 (ln m + 2) times the optimum in expectation; checked over many keys."""
    O = oracle_mod
    rng = np.random.default_rng(77)
    for m in (3, 4):
        pts = np.concatenate([rng.normal(c * 5.0, 1.0, (3, 2)) for c in range(m)]).astype(np.float32)[:8]
        best = _best_mway(pts.astype(np.float64), m)
        costs = []
        for key in range(400):
            lab, z, _ = O.kmeans(2, _x4(pts), np.arange(len(pts)), m, seed=5, key=key, km_iters=0)
            dist = ((pts[:, None, :] - z[None, :, :2]) ** 2).sum(2).min(1)
            costs.append(dist.sum())
        assert np.mean(costs) <= 8 * (np.log(m) + 2) * best


# ---------------------------------------------------------------- cut-row/column ordering (Sec. 4.2)
def _records(tree):
    return {(int(c), int(h)): i for i, (c, h) in enumerate(zip(tree["comp"], tree["heap"]))}


def _split_ranges(tree, i, sbd):
    """(V1, V2, V3) position ranges of split node i."""
    o, n1, n2, ns = (int(tree[f][i]) for f in ("offset", "n1", "n2", "nsep"))
    v2 = (o + n1 + ns, o + n1 + ns + n2) if sbd else (o + n1, o + n1 + n2)
    v3 = (o + n1, o + n1 + ns) if sbd else (o + n1 + n2, o + n1 + n2 + ns)
    return (o, o + n1), v2, v3


def _is_split(tree, i):
    return not (tree["n2"][i] == 0 and tree["nsep"][i] == 0)


@pytest.mark.parametrize("sbd", [False, True])
def test_cut_order_grid_line_runs(oracle_mod, sbd):
    """64x64 grid with its own coordinates: the root separator is one grid
    line; the root's two children split their halves along the other axis.
    With the cut rows ordered, the root separator is three runs of the line:
    the vertices beside the children's separators (linked to no part of
    either child's split), and the two halves of the line beside the
    children's first and second parts.  BBD puts the first run first; SBD
    puts it between the two halves, in the middle of the line."""
    O = oracle_mod
    A = W.grid_laplacian_2d(64)
    hg = O.build_from_matrix("symmetric", A)
    ij = np.indices((64, 64)).reshape(2, -1).T
    x4 = _x4(ij.astype(np.float32))
    plain, tree0 = O.order(hg, 2, x4, seed=1, sbd=sbd)
    perm, tree = O.order(hg, 2, x4, seed=1, sbd=sbd, cut_order=True)
    for f in tree0:
        assert np.array_equal(tree[f], tree0[f]), f
    rec = _records(tree)
    (a, b) = _split_ranges(tree, rec[(0, 1)], sbd)[2]
    line = ij[perm[a:b]]
    assert sorted(map(tuple, ij[plain[a:b]])) == sorted(map(tuple, line))
    axis = 0 if len(set(line[:, 0])) == 1 else 1
    along = line[:, 1 - axis]
    # the coordinates, along the root line, of the children's separator lines
    cut = set()
    for c in (2, 3):
        lo, hi = _split_ranges(tree, rec[(0, c)], sbd)[2]
        cut |= set(int(v) for v in ij[perm[lo:hi]][:, 1 - axis])
    assert len(cut) >= 1
    on = np.array([int(t) in cut for t in along])
    below = ~on & (along < min(cut))
    above = ~on & (along > max(cut))
    assert (on | below | above).all()
    cls = np.where(on, 0, np.where(below, 1, 2))
    runs = [cls[0]] + [cls[t] for t in range(1, len(cls)) if cls[t] != cls[t - 1]]
    assert sorted(runs) == [0, 1, 2]  # three contiguous runs
    if sbd:
        assert runs[1] == 0
    else:
        assert runs[0] == 0


@pytest.mark.parametrize("seed", [5, 6])
def test_cut_order_zero_blocks(oracle_mod, seed):
    """Power-law graph: the ordering differs from the plain one only inside the
    separator ranges (same sets, same tree), and every separator V3 of a node
    whose children split into (V11, V12) and (V21, V22) falls into four
    consecutive runs R0..R3 (BBD; SBD: R1, R0, R3, R2) with the zero blocks of
    the recursive form: rows of R0 meet none of V11, V12, V21, V22; rows of R1
    meet V11 or V21 but neither V12 nor V22; R2 the reverse; R3 both.  Inside
    every run the plain order is kept."""
    O = oracle_mod
    A = W.powerlaw_symmetric(2500, seed=seed)
    hg = O.build_from_matrix("symmetric", A)
    x4 = O.init_coords(hg.k, 3, seed)
    for sbd in (False, True):
        plain, tree0 = O.order(hg, 3, x4, seed=seed, min_part=8, sbd=sbd)
        perm, tree = O.order(hg, 3, x4, seed=seed, min_part=8, sbd=sbd, cut_order=True)
        for f in tree0:
            assert np.array_equal(tree[f], tree0[f]), f
        _check_ordering(O, A, hg, perm, tree, sbd)
        pos = np.empty(hg.k, dtype=np.int64)
        pos[perm] = np.arange(hg.k)
        pos0 = np.empty(hg.k, dtype=np.int64)
        pos0[plain] = np.arange(hg.k)
        inside = np.zeros(hg.k, dtype=bool)
        rec = _records(tree)
        moved = 0
        for i in range(len(tree["heap"])):
            if not _is_split(tree, i):
                continue
            c, h = int(tree["comp"][i]), int(tree["heap"][i])
            a, b = _split_ranges(tree, i, sbd)[2]
            inside[a:b] = True
            assert set(perm[a:b]) == set(plain[a:b])
            firsts, seconds = [], []
            for ch in (2 * h, 2 * h + 1):
                j = rec.get((c, ch))
                if j is not None and _is_split(tree, j):
                    r1, r2, _ = _split_ranges(tree, j, sbd)
                    firsts.append(r1)
                    seconds.append(r2)

            def meets(v, ranges):
                return any(lo <= pos[u] < hi for u in hg.adj[hg.adj_ptr[v]:hg.adj_ptr[v + 1]] for lo, hi in ranges)

            cls = np.array([int(meets(v, firsts)) + 2 * int(meets(v, seconds)) for v in perm[a:b]])
            order = [1, 0, 3, 2] if sbd else [0, 1, 2, 3]
            rank = np.array([order.index(t) for t in cls])
            assert (np.diff(rank) >= 0).all()
            for t in range(4):
                sel = perm[a:b][cls == t]
                assert (np.diff(pos0[sel]) > 0).all()
            moved += int((perm[a:b] != plain[a:b]).sum())
        assert np.array_equal(perm[~inside], plain[~inside])
        assert moved > 0


def test_cut_order_special_cases(oracle_mod):
    """Depth 1 (leaf children: every separator row has code 00) and separator
    recursion (the cut ordering is then not applied) leave the ordering as it
    is."""
    O = oracle_mod
    A = W.powerlaw_symmetric(1200, seed=9)
    hg = O.build_from_matrix("symmetric", A)
    x4 = O.init_coords(hg.k, 2, 9)
    for sbd in (False, True):
        for kw in ({"max_depth": 1}, {"sep_rec": True, "min_part": 8}):
            p0, t0 = O.order(hg, 2, x4, seed=2, sbd=sbd, **kw)
            p1, t1 = O.order(hg, 2, x4, seed=2, sbd=sbd, cut_order=True, **kw)
            assert np.array_equal(p0, p1)
            for f in t0:
                assert np.array_equal(t0[f], t1[f]), f


# ---------------------------------------------------------------- strengthened diagonal mu (Sec. 4.2, Alg. 7)
def _matched_rows(perm, m, match):
    rp = perm[perm < m].astype(np.int64)
    return rp, np.asarray(match, dtype=np.int64)[rp]


def _owners_of_pairs_agree(k, m, perm, tree, sbd, match):
    part = _owner_info(k, perm, tree, sbd)
    return np.array_equal(part[:m], part[m + np.asarray(match)])


def test_matched_luproblem_example(oracle_mod):
    """Ex. luproblem: with its diagonal as the matching and every row placed
    on its column (rows and columns of B at the left, of C at the right, row
    and column 4 between), one split gives the example's BBD form: blocks of
    b = 2 and c = 2 pairs and a border of d = 1 pair, the matrix unchanged up
    to the order of the two blocks."""
    O = oracle_mod
    g = json.load(open(os.path.join(GOLD, "luproblem.json")))
    M = np.array(g["matrix"])
    a = g["a"]
    assert abs(round(np.linalg.det(M)) - g["det_A"]) == 0
    r, c = np.nonzero(M)
    A = W.csr_from_coo(a, a, r, c, "luproblem")
    hg = O.build_from_matrix("bipartite", A)
    pts = np.array([[0, 0], [0, 1], [10, 0], [10, 1], [5, 0.5]], dtype=np.float32)
    x4 = _x4(np.concatenate([pts, pts]))
    match = np.arange(a)
    for sbd in (False, True):
        perm, tree = O.order(hg, 2, x4, seed=1, min_part=1, max_depth=1, sbd=sbd, match=match)
        n1, n2, ns = (int(tree[f][0]) for f in ("n1", "n2", "nsep"))
        assert sorted([n1 // 2, n2 // 2]) == [g["b"], g["c"]] and ns // 2 == g["d"]
        rp, cp = _matched_rows(perm, a, match)
        assert np.array_equal(rp, cp)
        blocks = [set(rp[:2]), set(rp[2:4]) if not sbd else set(rp[3:5])]
        assert sorted(map(sorted, blocks)) == [[0, 1], [2, 3]]
        assert rp[4 if not sbd else 2] == 4
        B = M[np.ix_(rp, cp)]
        lo, hi = (slice(0, 2), slice(2, 4)) if not sbd else (slice(0, 2), slice(3, 5))
        assert not B[lo, hi].any() and not B[hi, lo].any()


@pytest.mark.parametrize("cut_order", [False, True])
@pytest.mark.parametrize("sbd", [False, True])
@pytest.mark.parametrize("seed", [1, 2])
def test_matched_square_blocks(oracle_mod, sbd, seed, cut_order):
    """Unsymmetric mesh pattern with a strengthened diagonal, random
    coordinates (many matching edges cut): every matched pair (row i, column
    mu(i)) has one owner (no matching edge leaves the diagonal blocks and
    separators); the rows with their matched columns give square diagonal
    blocks: with the column order mu(row order) the diagonal is full and, at
    every split, the blocks (R1, C2) and (R2, C1) are empty.  Without the
    matching, separators split pairs.  The cut-row ordering (pairs sorted by
    the two-bit numbers of row and column together) keeps all of this."""
    O = oracle_mod
    A = W.with_strengthened_diagonal(W.grid_laplacian_2d(36), 0.7, seed)
    match = A.meta["match"]
    m = A.m
    hg = O.build_from_matrix("bipartite", A)
    x4 = O.init_coords(hg.k, 2, seed)
    perm, tree = O.order(hg, 2, x4, seed=seed, min_part=6, sbd=sbd, match=match, cut_order=cut_order)
    _check_ordering(O, A, hg, perm, tree, sbd)
    assert _owners_of_pairs_agree(hg.k, m, perm, tree, sbd, match)
    rp, cp = _matched_rows(perm, m, match)
    assert sorted(rp.tolist()) == list(range(m)) and sorted(cp.tolist()) == list(range(m))
    dense = np.zeros((m, m), dtype=bool)
    r = np.repeat(np.arange(m), np.diff(A.rowptr))
    dense[r, A.colidx] = True
    B = dense[np.ix_(rp, cp)]
    assert B.diagonal().all()
    for i in range(len(tree["heap"])):
        o, n1, n2, ns = (int(tree[f][i]) for f in ("offset", "n1", "n2", "nsep"))
        if n2 == 0 and ns == 0:
            continue
        assert o % 2 == 0 and n1 % 2 == 0 and n2 % 2 == 0 and ns % 2 == 0
        p0, p1, p2 = o // 2, n1 // 2, n2 // 2
        r1 = slice(p0, p0 + p1)
        r2 = slice(p0 + p1 + ns // 2, p0 + p1 + ns // 2 + p2) if sbd else slice(p0 + p1, p0 + p1 + p2)
        assert not B[r1, r2].any() and not B[r2, r1].any()
    plain, tree0 = O.order(hg, 2, x4, seed=seed, min_part=6, sbd=sbd)
    assert not _owners_of_pairs_agree(hg.k, m, plain, tree0, sbd, match)


def _root_separator_case(O, order_free):
    A = W.with_strengthened_diagonal(W.powerlaw_symmetric(800, seed=4), 0.6, 4)
    match = A.meta["match"]
    hg = O.build_from_matrix("bipartite", A)
    x4 = O.init_coords(hg.k, 3, 4)
    comps = O.components(hg)
    root = np.flatnonzero(comps == comps[0]).astype(np.int32)
    perm, tree = O.order(hg, 3, x4, seed=4, max_depth=1, match=match, min_part=1, order_free=order_free)
    # the first component's root node; its vertices in their initial order
    j = [i for i in range(len(tree["heap"])) if tree["comp"][i] == 0 and tree["heap"][i] == 1][0]
    o, n1, n2, ns = (int(tree[f][j]) for f in ("offset", "n1", "n2", "nsep"))
    assert np.array_equal(np.sort(perm[o:o + n1 + n2 + ns]), root)
    verts = root  # the root's order before its split: ascending vertex ids
    ok, lab, z1, z2 = O.bisect(3, x4, verts, seed=4, key=1)
    assert ok
    r = (z2[:3] - z1[:3]).astype(np.float32)
    mid = (np.float32(0.5) * (z1[:3] + z2[:3])).astype(np.float32)
    delta = np.float32(0)
    for t in range(3):
        delta = np.float32(delta + np.float32(mid[t] * r[t]))

    def s(v):
        acc = np.float32(0)
        for t in range(3):
            acc = np.float32(acc + np.float32(np.float32(x4[v, t]) * r[t]))
        return abs(np.float32(acc - delta))

    L = dict(zip(verts.tolist(), lab.tolist()))
    mu = O.mu_from_match(hg, match)
    # cut edges (2-means labels), as (key of the selected end, selected end, other end)
    cut = []
    for v in verts.tolist():
        for w in hg.adj[hg.adj_ptr[v]:hg.adj_ptr[v + 1]].tolist():
            if w > v and w in L and L[v] != L[w]:
                a, b = sorted([(s(v), v), (s(w), w)])
                cut.append((a[0], a[1], b[1]))
    got = set(perm[o + n1 + n2:o + n1 + n2 + ns].tolist())
    side1 = set(perm[o:o + n1].tolist())
    assert all(L[v] == L[next(iter(side1))] for v in side1)
    return got, cut, L, mu


def test_matched_separator_order_free(oracle_mod):
    """The separator with a matching in its order-free reading: at the root,
    V3 is exactly the set of ends with the smaller (|x.r - delta|, id) of the
    edges cut by the 2-means labels, with their partners; V1 and V2 keep the
    2-means labels."""
    got, cut, L, mu = _root_separator_case(oracle_mod, True)
    sel = {v for _, v, _ in cut}
    assert got == sel | {int(mu[v]) for v in sel}


def test_matched_separator_literal_loop(oracle_mod):
    """The default reading: Algorithm 7's loop itself over the cut edges in the
    canonical order (ascending key of the selected end, then the other end);
    an edge still cut when reached moves its selected end and that end's
    partner into V3, an edge with an end (or through it a partner) already
    moved is skipped.  Restated here as a plain loop on the root's data; it
    gives a subset of the order-free separator, strictly smaller here."""
    got, cut, L, mu = _root_separator_case(oracle_mod, False)
    lab = dict(L)
    for _, v, w in sorted(cut):
        if lab[v] != 3 and lab[w] != 3:
            lab[v] = 3
            lab[int(mu[v])] = 3
    assert got == {v for v, l in lab.items() if l == 3}
    free, _, _, _ = _root_separator_case(oracle_mod, True)
    assert got < free


def _heap_path_codes(hg, perm, tree, sbd, b, owner):
    """Pairs 1..b of every separator vertex, from the owners' heap numbers:
    a neighbour owned by a node D levels below the separator's node d lies in
    the first (second) part of the split of its ancestor at depth d + l when
    D >= d + l + 1 and the branch taken at depth d + l + 1 is 2h (2h + 1)."""
    H, Dp = tree["heap"], tree["depth"]
    codes = {}
    for i in range(len(H)):
        o, n1, n2, ns = (int(tree[f][i]) for f in ("offset", "n1", "n2", "nsep"))
        if ns == 0:
            continue
        a = o + n1 if sbd else o + n1 + n2
        h, d = int(H[i]), int(Dp[i])
        for w in perm[a:a + ns].tolist():
            c = 0
            for u in hg.adj[hg.adj_ptr[w]:hg.adj_ptr[w + 1]].tolist():
                j = owner[u]
                hu, du = int(H[j]), int(Dp[j])
                if du <= d or (hu >> (du - d)) != h or tree["comp"][j] != tree["comp"][i]:
                    continue
                for l in range(1, b + 1):
                    if du >= d + l + 1:
                        c |= (2 if (hu >> (du - d - l - 1)) & 1 else 1) << (2 * (b - l))
            codes[w] = c
    return codes


@pytest.mark.parametrize("b", [2, 3])
def test_cut_order_levels(oracle_mod, b):
    """Cut ordering to b levels: every separator is sorted by its vertices'
    pairs 1..b in turn (rank per pair: BBD 00, 01, 10, 11; SBD 01, 00, 11, 10),
    the pairs recomputed from the tree's heap numbers (the branch a neighbour's
    owner takes below the separator's node), the plain order kept within
    equal pairs; the ordering differs from one level's; b beyond the depth of
    the tree changes nothing more."""
    O = oracle_mod
    A = W.grid_laplacian_3d(14)
    hg = O.build_from_matrix("symmetric", A)
    x4 = O.init_coords(hg.k, 3, 8)
    for sbd in (False, True):
        plain, _ = O.order(hg, 3, x4, seed=8, min_part=4, sbd=sbd)
        one, _ = O.order(hg, 3, x4, seed=8, min_part=4, sbd=sbd, cut_order=1)
        perm, tree = O.order(hg, 3, x4, seed=8, min_part=4, sbd=sbd, cut_order=b)
        _check_ordering(O, A, hg, perm, tree, sbd)
        owner = _owner_info(hg.k, perm, tree, sbd)
        codes = _heap_path_codes(hg, perm, tree, sbd, b, owner)
        rank1 = [1, 0, 3, 2] if sbd else [0, 1, 2, 3]
        pos0 = np.empty(hg.k, dtype=np.int64)
        pos0[plain] = np.arange(hg.k)
        for i in range(len(tree["heap"])):
            o, n1, n2, ns = (int(tree[f][i]) for f in ("offset", "n1", "n2", "nsep"))
            if ns == 0:
                continue
            a = o + n1 if sbd else o + n1 + n2
            seg = perm[a:a + ns]
            assert set(seg.tolist()) == set(plain[a:a + ns].tolist())
            key = [tuple(rank1[(codes[w] >> (2 * (b - l))) & 3] for l in range(1, b + 1)) + (int(pos0[w]),)
                   for w in seg.tolist()]
            assert key == sorted(key)
        assert not np.array_equal(perm, one)
    # the tree is 3 levels deep: pairs beyond the deepest split are 00
    p3, _ = O.order(hg, 3, x4, seed=8, min_part=4, max_depth=3, cut_order=2)
    for bb in (3, 8):
        pb, _ = O.order(hg, 3, x4, seed=8, min_part=4, max_depth=3, cut_order=bb)
        assert np.array_equal(pb, p3)


def test_mu_from_match_checks_the_matching(oracle_mod):
    """mu of a perfect matching pairs row i with column match[i] both ways;
    a non-permutation, an entry outside the pattern, a non-bipartite model and
    a rectangular pattern are refused."""
    O = oracle_mod
    A = W.with_strengthened_diagonal(W.grid_laplacian_2d(12), 0.6, 4)
    m = A.m
    bp = O.build_from_matrix("bipartite", A)
    match = A.meta["match"].astype(np.int64)
    mu = O.mu_from_match(bp, match)
    assert np.array_equal(mu[:m], m + match) and np.array_equal(mu[m + match], np.arange(m))
    assert np.array_equal(mu[mu], np.arange(2 * m))
    dup = match.copy()
    dup[1] = dup[0]
    dense = np.zeros((m, m), dtype=bool)
    dense[np.repeat(np.arange(m), np.diff(A.rowptr)), A.colidx] = True
    i, j = np.argwhere(~dense)[0]
    off = match.copy()
    k = int(np.flatnonzero(match == j)[0])
    off[i], off[k] = j, match[i]
    for bad in (dup, off):
        with pytest.raises(ValueError):
            O.mu_from_match(bp, bad)
    with pytest.raises(ValueError):
        O.mu_from_match(O.build_from_matrix("symmetric", A), match)
    R = W.powerlaw_rectangular(30, 20, seed=1)
    with pytest.raises(ValueError):
        O.mu_from_match(O.build_from_matrix("bipartite", R), np.arange(25))
