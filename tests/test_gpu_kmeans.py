"""m-way k-means++ (Algorithm 5 with m centres) on the GPU against the oracle:
labels and centres bit-exact (integer decisions taken in fp32 without FMA on
both sides, exact fixed-point means), for m from 1 to 256, d = 2, 3, 4, ragged
sizes up to a million points; m = 2 equals vmo_bisect."""
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
    assert torch.cuda.is_available()
    return P


@pytest.fixture(scope="module")
def O():
    import oracle
    oracle.build()
    return oracle


def _np(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("d", [2, 3, 4])
def test_kmeans_bit_exact(V, O, d):
    rng = np.random.default_rng(d)
    k = 30000
    x = O.init_coords(k, d, 40 + d)
    xt = torch.as_tensor(x).cuda()
    for m, n, km in ((1, 1000, 20), (3, 2999, 20), (17, 20011, 20), (64, 29999, 12), (256, 30000, 5),
                     (5, 7, 20), (8, 8, 3), (8, 3, 20)):
        verts = rng.choice(k, n, replace=False).astype(np.int32)
        key = int(rng.integers(1, 1 << 40))
        lab, z, ne = V.kmeans(xt, torch.as_tensor(verts), m, seed=77, key=key, km_iters=km, d=d)
        lab_o, z_o, ne_o = O.kmeans(d, x, verts, m, seed=77, key=key, km_iters=km)
        assert ne == ne_o
        assert np.array_equal(_np(lab), lab_o), (m, n)
        assert np.array_equal(_np(z).view(np.uint32), z_o.view(np.uint32)), (m, n)


def test_kmeans_m2_equals_bisect(V, O):
    A = W.grid_laplacian_2d(8)
    hg = V.Hypergraph.from_matrix(A)
    k = 50000
    x = O.init_coords(k, 3, 5)
    xt = torch.as_tensor(x).cuda()
    verts = torch.as_tensor(np.random.default_rng(1).choice(k, 40000, replace=False).astype(np.int32))
    ok, lab2, z1, z2 = hg.bisect(xt, verts, seed=3, key=11, km_iters=20, d=3)
    lab, z, ne = V.kmeans(xt, verts, 2, seed=3, key=11, km_iters=20, d=3)
    assert ok and ne == 2
    assert torch.equal(lab, lab2.to(torch.int32) - 1)
    assert torch.equal(z[0].view(torch.int32), z1.view(torch.int32))
    assert torch.equal(z[1].view(torch.int32), z2.view(torch.int32))


def test_kmeans_full_size_and_degenerate(V, O):
    """A million points with 64 centres (bit-exact), coincident points (one
    non-empty cluster), an empty set, and rejected arguments."""
    k = 1_000_000
    x = O.init_coords(k, 3, 9)
    xt = torch.as_tensor(x).cuda()
    verts = np.arange(k, dtype=np.int32)
    lab, z, ne = V.kmeans(xt, torch.as_tensor(verts), 64, seed=1, key=1, km_iters=20, d=3)
    lab_o, z_o, ne_o = O.kmeans(3, x, verts, 64, seed=1, key=1, km_iters=20)
    assert ne == ne_o == 64
    assert np.array_equal(_np(lab), lab_o)
    assert np.array_equal(_np(z).view(np.uint32), z_o.view(np.uint32))
    same = torch.zeros((100, 4), device="cuda")
    same[:, :2] = 2.5
    lab, z, ne = V.kmeans(same, torch.arange(100), 8, seed=1, d=2)
    assert ne == 1 and int(lab.max()) == 0
    lab, z, ne = V.kmeans(same, torch.arange(0), 8, seed=1, d=2)
    assert ne == 0 and lab.numel() == 0
    for bad_m in (0, 257):
        with pytest.raises(V.VmoError):
            V.kmeans(same, torch.arange(10), bad_m, seed=1, d=2)
