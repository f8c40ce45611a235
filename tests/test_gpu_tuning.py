"""Launch-shape tuning (vmo_set_tuning / vmo_autotune): no setting changes a
result.  The layout (every level, both step-kernel variants), the ordering
and a batch are bit-identical under settings at the ends of every range, and
the autotuner leaves a valid setting no slower than where it started."""
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
    t0 = P.get_tuning()
    yield P
    P.set_tuning(**t0)


def _np(t):
    return t.detach().cpu().numpy()


SETTINGS = [(19456, 10, 8, 2048), (0, 8, 1, 0), (10 ** 9, 9, 4, 2048), (4864, 10, 2, 512)]


def test_settings_do_not_change_results(V):
    A = W.powerlaw_symmetric(60000, seed=41)
    G = W.grid_laplacian_3d(40)
    mats = W.batch_mix(20, 43, nmin=200, nmax=6000)
    ref = None
    for st in SETTINGS:
        V.set_tuning(*st)
        out = []
        for M in (A, G):
            hg = V.Hypergraph.from_matrix(M)
            p = V.Params(d=3, seed=2, max_depth=10)
            x = hg.layout(p)
            perm, tree = hg.order_vertices(p, x)
            out += [_np(x), _np(perm), _np(tree["nsep"])]
        bp, _ = V.batch_order(mats, V.Params(d=3, seed=3))
        out.append(_np(bp))
        if ref is None:
            ref = out
        else:
            for a, b in zip(ref, out):
                assert np.array_equal(a, b), st


def test_autotune(V):
    mats = W.batch_mix(12, 45, nmin=500, nmax=8000)
    V.set_tuning(19456, 10, 8, 2048)
    best, best_ms, default_ms = V.autotune(mats, V.Params(d=3, seed=1), reps=1)
    assert V.get_tuning() == best
    assert best["radix_max_bits"] in (8, 9, 10) and best["assign_items"] in (1, 2, 4, 8)
    assert best["small_bin_points"] in (0, 512, 2048)
    assert 0 < best_ms <= default_ms
    with pytest.raises(V.VmoError):
        V.autotune(mats, V.Params(), reps=0)
    assert V.get_tuning() == best


def test_small_bin_equals_device_wide(V):
    """The one-block binning of small levels (small_bin_points) gives the
    layouts of the device-wide sequence bit for bit: d = 2, 3, 4, a
    hypergraph model (nets of more than two pins), vertex weights, levels of
    up to one sort tile (2,048 points) and, at occupancy 1, of exactly 4,096
    finest cells (d = 2 and 4), one step with its keys and gradient, and a
    batch whose levels mix small and large problems."""
    t0 = V.get_tuning()
    cases = [(2, W.grid_laplacian_2d(64), "symmetric", False), (3, W.powerlaw_symmetric(1500, seed=5), "symmetric", True),
             (4, W.powerlaw_symmetric(3000, seed=6), "symmetric", False),
             (2, W.powerlaw_rectangular(1500, 1000, seed=7), "rownet", False),
             (3, W.grid_laplacian_2d(45), "symmetric", False),
             (2, W.grid_laplacian_2d(64), "symmetric", False, 1), (4, W.powerlaw_symmetric(2048, seed=8), "symmetric",
                                                                   False, 1)]
    mats = W.batch_mix(16, 47, nmin=200, nmax=5000)
    runs = []
    try:
        for sb in (2048, 0):
            V.set_tuning(t0["small_step_threads"], t0["radix_max_bits"], t0["assign_items"], sb)
            out = []
            for d, A, model, weighted, *occ in cases:
                hg = V.Hypergraph.from_matrix(A, model)
                if weighted:
                    w = torch.as_tensor(1.0 + W.rand_uniform(9, 1, hg.k).astype(np.float32))
                    hg = V.Hypergraph.from_matrix(A, model, w)
                p = V.Params(d=d, seed=4, occupancy=occ[0] if occ else 8)
                out.append(_np(hg.layout(p)))
                x0 = torch.as_tensor(W.rand_uniform(9, 2, hg.k * 4).astype(np.float32).reshape(hg.k, 4)).cuda()
                x1, y, keys, L = hg.layout_step(x0, 0.01, p)
                out += [_np(x1), _np(y), _np(keys), np.array([L])]
            bp, _ = V.batch_order(mats, V.Params(d=3, seed=3))
            out.append(_np(bp))
            runs.append(out)
    finally:
        V.set_tuning(**t0)
    for a, b in zip(*runs):
        assert np.array_equal(a, b)
