"""Parity at the full sizes of the measured workloads, in the configuration
the benchmark times (multilevel layout, d and depth of each workload).

For every full-size matrix: one layout step from the same random layout
within the layout tolerance of the oracle (gradient and displacement, keys
bit-exact), and the ordering of the GPU's own multilevel layout bit-exact
against the oracle's ordering of the same coordinates (permutation and
tree).  The rectangular SBD workload also checks its cut metrics, and the
batched workload (4,096 matrices) checks a seeded sample of its matrices
against their one-at-a-time orderings."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

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


def _step(V, O, hg, ref, d, seed):
    x0 = O.init_coords(ref.k, d, seed)
    p = V.Params(d=d)
    xg, yg, kg, L = hg.layout_step(torch.as_tensor(x0).cuda(), 0.37, p)
    xo, yo, ko, Lo = O.layout_step(ref, d, x0.astype(np.float64), 0.37)
    assert L == Lo
    assert np.array_equal(_np(kg).view(np.uint32), ko)
    yg, xg = _np(yg).astype(np.float64), _np(xg).astype(np.float64)
    ey = np.linalg.norm(yg[:, :d] - yo[:, :d]) / np.linalg.norm(yo[:, :d])
    dx = xo[:, :d] - x0[:, :d]
    ex = np.linalg.norm((xg[:, :d] - x0[:, :d]) - dx) / np.linalg.norm(dx)
    assert ey <= Y_TOL and ex <= Y_TOL, (ey, ex)


def _order(V, O, hg, ref, d, sbd, min_part, max_depth, seed):
    p = V.Params(d=d, min_part=min_part, max_depth=max_depth, seed=seed)
    x = hg.layout(p)
    perm, tree = hg.order_vertices(p, x, sbd=sbd)
    perm_o, tree_o = O.order(ref, d, _np(x), seed=seed, min_part=min_part, max_depth=max_depth, sbd=sbd)
    assert np.array_equal(_np(perm), perm_o)
    for f in ("offset", "n1", "n2", "nsep", "depth", "comp"):
        assert np.array_equal(_np(tree[f]), tree_o[f]), f
    return perm_o, tree_o


@pytest.mark.parametrize("name", ["powerlaw_500k", "stencil27_100"])
def test_full_size_symmetric(V, O, name):
    """500k power-law (the medium workload's second matrix; d = 3, depth 10)
    and the 27-point stencil on 100^3 (the served stream's large request;
    1,000,000 rows, 26,463,592 nnz; d = 3, parts of <= 64 rows)."""
    if name == "powerlaw_500k":
        A, d, depth = W.powerlaw_symmetric(500_000, seed=1), 3, 10
    else:
        A, d, depth = W.stencil27(100), 3, 62
    hg = V.Hypergraph.from_matrix(A)
    ref = O.build_from_matrix("symmetric", A)
    _step(V, O, hg, ref, d, seed=7)
    _order(V, O, hg, ref, d, False, 64, depth, seed=1)


def test_full_size_rectangular_sbd(V, O):
    """400,000 x 300,000 power-law pattern, bipartite model, d = 2, SBD to
    depth 6 (64 parts): step, ordering, and the cut metrics of the final
    parts over the row nets and the column nets."""
    A = W.powerlaw_rectangular(400_000, 300_000, seed=1)
    hg = V.Hypergraph.from_matrix(A, "bipartite")
    ref = O.build_from_matrix("bipartite", A)
    _step(V, O, hg, ref, 2, seed=7)
    perm_o, tree_o = _order(V, O, hg, ref, 2, True, 1, 6, seed=1)
    part = O.parts_from_tree(ref.k, perm_o, tree_o, sbd=True)
    rows, cols = part[:A.m].copy(), part[A.m:].copy()
    nparts = int(part.max()) + 1
    for model, p in (("rownet", cols), ("colnet", rows)):
        g = V.Hypergraph.from_matrix(A, model)
        r = O.build_from_matrix(model, A)
        assert g.cut_size(torch.as_tensor(p), nparts) == O.cut_size(r.net_ptr, r.pins, p), model


def test_full_size_batch_4096_sampled(V):
    """The 4,096-matrix batch (n log-uniform in [200, 20000], half grids, half
    random): a seeded sample of its permutations equals the one-at-a-time
    orderings of those matrices."""
    mats = W.batch_mix(4096, seed=1)
    dev = [(torch.as_tensor(A.rowptr).cuda(), torch.as_tensor(A.colidx).cuda(), A.m) for A in mats]
    p = V.Params(d=3, seed=1)
    perm, offs = V.batch_order(dev, p)
    perm = _np(perm)
    rng = np.random.default_rng(4096)
    for i in sorted(rng.choice(len(mats), 12, replace=False)):
        rp, ci, m = dev[i]
        one = V.Hypergraph(rp, ci, m, m).order_vertices(p)[0]
        assert np.array_equal(perm[offs[i]:offs[i + 1]], _np(one)), i
