"""Pins of the oracle's multilevel layout (Algorithm 3, Sec. 2.3): the coarse
graphs of the hierarchy against the quotient P^T A P of the grouping (scipy
sparse products), the vertex weights against P^T w, the prolongation against
the properties the paper asks of it (unit point density kept, members of a
group started apart by a small jitter keyed by the fine vertex), and the
weighted, costed gradient against finite differences of the energy."""
import numpy as np
import pytest
from scipy import sparse, stats

import workloads as W


def _graphs():
    return [("grid2d_24", W.grid_laplacian_2d(24)), ("powerlaw_1500", W.powerlaw_symmetric(1500, seed=3)),
            ("grid3d_9", W.grid_laplacian_3d(9))]


def _adj_matrix(k, adj_ptr, adj, val):
    return sparse.csr_matrix((np.asarray(val, dtype=np.float64), np.asarray(adj), np.asarray(adj_ptr)),
                             shape=(k, k))


def _group_matrix(pi, kc):
    kf = len(pi)
    return sparse.csr_matrix((np.ones(kf), (np.arange(kf), pi)), shape=(kf, kc))


@pytest.mark.parametrize("name,A", _graphs())
def test_contraction_is_the_quotient_graph(oracle_mod, name, A):
    """Every coarse level j: costs = P^T A_{j-1} P off the diagonal (merged
    parallel edges add, edges inside a group vanish), weights = P^T w_{j-1};
    and against level 0 directly: the cost between two coarse vertices is the
    number of fine edges between the vertex sets they stand for, the weight
    their total fine weight."""
    O = oracle_mod
    hg = O.build_from_matrix("symmetric", A)
    rng = np.random.default_rng(7)
    w0 = rng.uniform(0.25, 4.0, hg.k)
    lv0 = O.hierarchy_level(hg, 0, seed=5, w=w0)
    assert lv0["nlevels"] >= 3, name
    A0 = _adj_matrix(hg.k, hg.adj_ptr, hg.adj, np.ones(len(hg.adj)))
    assert np.array_equal(lv0["acost"], np.ones(len(hg.adj)))
    assert np.array_equal(lv0["w"], w0)
    prev, Ptot = lv0, sparse.identity(hg.k, format="csr")
    for j in range(1, lv0["nlevels"]):
        cur = O.hierarchy_level(hg, j, seed=5, w=w0)
        kc, pi = cur["k"], cur["pi"]
        assert len(pi) == prev["k"] and pi.min() == 0 and pi.max() == kc - 1
        assert len(np.unique(pi)) == kc  # every coarse vertex stands for a group
        P = _group_matrix(pi, kc)
        Ap = _adj_matrix(prev["k"], prev["adj_ptr"], prev["adj"], prev["acost"])
        Q = (P.T @ Ap @ P).tolil()
        Q.setdiag(0)
        Q = Q.tocsr()
        Q.eliminate_zeros()
        Q.sort_indices()
        assert np.array_equal(Q.indptr, cur["adj_ptr"]), (name, j)
        assert np.array_equal(Q.indices, cur["adj"]), (name, j)
        assert np.array_equal(Q.data, cur["acost"]), (name, j)
        assert np.allclose(P.T @ prev["w"], cur["w"], rtol=1e-14, atol=0)
        # straight from level 0
        Ptot = Ptot @ P
        Q0 = (Ptot.T @ A0 @ Ptot).tolil()
        Q0.setdiag(0)
        Q0 = Q0.tocsr()
        Q0.eliminate_zeros()
        Q0.sort_indices()
        assert np.array_equal(Q0.data, cur["acost"]) and np.array_equal(Q0.indices, cur["adj"])
        assert np.allclose(Ptot.T @ w0, cur["w"], rtol=1e-13, atol=0)
        assert np.isclose(cur["w"].sum(), w0.sum(), rtol=1e-13)
        # symmetric adjacency, no self-loops, neighbours ascending
        rows = np.repeat(np.arange(kc), np.diff(cur["adj_ptr"]))
        assert not np.any(rows == cur["adj"])
        assert all(np.all(np.diff(cur["adj"][a:b]) > 0) for a, b in zip(cur["adj_ptr"][:-1], cur["adj_ptr"][1:]))
        prev = cur
    assert O.hierarchy_level(hg, lv0["nlevels"], seed=5) is None


def test_hierarchy_level_sizes_agree(oracle_mod):
    O = oracle_mod
    A = W.powerlaw_symmetric(2000, seed=4)
    hg = O.build_from_matrix("symmetric", A)
    sizes = O.hierarchy(hg, 9)
    assert [O.hierarchy_level(hg, j, seed=9)["k"] for j in range(len(sizes))] == sizes


@pytest.mark.parametrize("d", [2, 3, 4])
def test_prolongation_keeps_density_and_jitters(oracle_mod, d):
    """Prolonged points sit at f x_c(pi(v)) plus an offset of at most 0.05 per
    coordinate, f^d = k_f / k_c (the coarse layout scaled to the fine point
    count at the same density); the offsets are uniform on [-0.05, 0.05),
    independent between coordinates, keyed by the fine vertex (the same for
    any grouping), and different for the members of one group."""
    O = oracle_mod
    A = W.grid_laplacian_2d(40)
    hg = O.build_from_matrix("symmetric", A)
    lv = O.hierarchy_level(hg, 2, seed=3)
    kf, kc, pi = len(lv["pi"]), lv["k"], lv["pi"]
    rng = np.random.default_rng(1)
    xc = np.zeros((kc, 4))
    xc[:, :d] = rng.uniform(1000.0, 2000.0, (kc, d))
    xf = O.prolong(kf, kc, d, 3, 2, pi, xc)
    assert np.all(xf[:, d:] == 0.0)
    # f from points far from the origin: |offset| / x_c <= 0.05 / 1000
    fest = xf[:, :d] / xc[pi, :d]
    f = float(np.median(fest))
    assert np.all(np.abs(fest - f) <= 0.05 / 1000 * 1.01)
    assert abs(f ** d * kc / kf - 1.0) < 1e-4
    off = xf[:, :d] - (kf / kc) ** (1.0 / d) * xc[pi, :d]
    assert np.all(off >= -0.05 - 1e-9) and np.all(off < 0.05 + 1e-9)
    for m in range(d):
        assert stats.kstest((off[:, m] + 0.05) / 0.1, "uniform").pvalue > 1e-3
        assert abs(off[:, m].mean()) < 0.005
    if d >= 2:
        assert abs(np.corrcoef(off[:, 0], off[:, 1])[0, 1]) < 0.1
    # offsets belong to the fine vertex: another grouping moves no offset
    zero_c = np.zeros((kc, 4))
    o1 = O.prolong(kf, kc, d, 3, 2, pi, zero_c)
    o2 = O.prolong(kf, kc, d, 3, 2, rng.permutation(pi), zero_c)
    assert np.array_equal(o1, o2)
    assert np.allclose(o1[:, :d], off, atol=1e-9)
    # members of a group start apart
    for g in np.flatnonzero(np.bincount(pi) >= 2)[:200]:
        mem = np.flatnonzero(pi == g)
        assert len(np.unique(xf[mem, :d], axis=0)) == len(mem)
    # another level or seed draws other offsets
    assert not np.allclose(O.prolong(kf, kc, d, 3, 1, pi, zero_c), o1)
    assert not np.allclose(O.prolong(kf, kc, d, 4, 2, pi, zero_c), o1)


def test_prolongation_draws_keyed_splitmix(oracle_mod):
    """The reading of the jitter draw: u = (rand(seed ^ JITTER, v, 4 (j-1) + m)
    >> 40) 2^-24 with the SplitMix64-keyed generator pinned elsewhere against
    its published sequence; JITTER is the ASCII tag 'jitter'."""
    O = oracle_mod
    tag = int.from_bytes(b"jitter\0\0", "big")
    kf, kc, d, seed, j = 50, 20, 3, 77, 3
    pi = np.arange(kf) % kc
    off = O.prolong(kf, kc, d, seed, j, pi, np.zeros((kc, 4)))
    for v in range(kf):
        for m in range(d):
            u = (O.rand64(seed ^ tag, v, 4 * (j - 1) + m) >> 40) * 2.0 ** -24
            assert off[v, m] == 0.1 * (u - 0.5)


@pytest.mark.parametrize("d", [2, 3, 4])
def test_weighted_costed_gradient_matches_finite_differences(oracle_mod, d):
    """The gradient on a coarse level (vertex weights w, net costs c, the form
    every level above the finest takes) is the derivative of the energy of eq.
    graphenergysimple with those weights and costs."""
    O = oracle_mod
    A = W.powerlaw_symmetric(400, seed=2)
    hg = O.build_from_matrix("symmetric", A)
    lv = O.hierarchy_level(hg, 1, seed=2, w=np.random.default_rng(3).uniform(0.5, 2.0, hg.k))
    g, c = O.graph_nets(lv["k"], lv["adj_ptr"], lv["adj"], lv["acost"])
    assert c.max() > 1.0 and lv["w"].max() > 2.0  # merged edges and groups present
    x = O.init_coords(g.k, d, 5).astype(np.float64)
    y, _, L, _, _ = O.gradient(g, d, x, occ=10 ** 6, w=lv["w"], c=c)
    assert L == 1
    h = 1e-4  # fourth-order central difference: the energy is a sum of ~k^2 terms

    def e_at(n, m, t):
        xt = x.copy()
        xt[n, m] += t
        return O.energy(g, d, xt, w=lv["w"], c=c)

    for n in range(0, g.k, 7):
        for m in range(d):
            fd = (8 * (e_at(n, m, h) - e_at(n, m, -h)) - (e_at(n, m, 2 * h) - e_at(n, m, -2 * h))) / (12 * h)
            assert abs(fd - y[n, m]) <= 1e-6 * (1 + abs(y[n, m])), (n, m, fd, y[n, m])


def test_graph_nets_round_trip(oracle_mod):
    """graph_nets gives the symmetric model's own nets for a level-0 graph."""
    O = oracle_mod
    A = W.powerlaw_symmetric(800, seed=6)
    hg = O.build_from_matrix("symmetric", A)
    g, c = O.graph_nets(hg.k, hg.adj_ptr, hg.adj, np.ones(len(hg.adj)))
    for f in ("net_ptr", "pins", "vtx_ptr", "vnets"):
        assert np.array_equal(getattr(g, f), getattr(hg, f)), f
    assert np.all(c == 1.0)
