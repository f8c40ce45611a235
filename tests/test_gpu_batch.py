"""Batched ordering (many independent matrices in one launch sequence) gives
every matrix exactly the permutation it gets alone, and that permutation is
the oracle's on the same coordinates."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1105_4490_gb300 as P
    return P


def _mix():
    mats = W.batch_mix(16, seed=3, nmin=20, nmax=3000)
    mats += [W.grid_laplacian_2d(1), W.random_symmetric(500, 1.6, 5),      # 1x1 and many components
             W.csr_from_coo(7, 7, np.array([], int), np.array([], int), "empty"),
             W.powerlaw_symmetric(2500, seed=4), W.grid_laplacian_3d(9)]
    return mats


@pytest.mark.parametrize("sbd", [False, True])
@pytest.mark.parametrize("d", [2, 3])
def test_batch_equals_plain(V, d, sbd):
    mats = _mix()
    p = V.Params(d=d, seed=9, min_part=16, iters=40)
    perm, offs = V.batch_order(mats, p, sbd=sbd)
    perm = perm.cpu().numpy()
    for i, A in enumerate(mats):
        hg = V.Hypergraph.from_matrix(A)
        alone, _ = hg.order_vertices(p, sbd=sbd)
        got = perm[offs[i]:offs[i + 1]]
        assert np.array_equal(got, alone.cpu().numpy()), (i, A.name)
        assert sorted(got.tolist()) == list(range(A.m))


def test_batch_layout_matches_oracle_ordering(V):
    """The batched permutation of a matrix is the oracle's ordering of the GPU
    layout of that matrix (the ordering stage is bit-exact)."""
    import oracle
    A = W.powerlaw_symmetric(3000, seed=6)
    mats = [W.grid_laplacian_2d(20), A, W.random_symmetric(800, 5, 2)]
    p = V.Params(d=3, seed=2)
    perm, offs = V.batch_order(mats, p)
    hg = V.Hypergraph.from_matrix(A)
    x = hg.layout(p)
    ref = oracle.build_from_matrix("symmetric", A)
    perm_o, _ = oracle.order(ref, 3, x.cpu().numpy(), seed=2)
    assert np.array_equal(perm[offs[1]:offs[2]].cpu().numpy(), perm_o)


def test_batch_rejects_bad_input(V):
    bad = W.csr_from_coo(4, 5, np.array([0, 1]), np.array([1, 2]), "rect")
    with pytest.raises(V.VmoError):
        V.batch_order([W.grid_laplacian_2d(4), bad])
