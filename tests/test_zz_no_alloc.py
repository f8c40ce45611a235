"""vmo_bisect_noalloc against vmo_bisect.

The allocation-free entry point serves callers that may not allocate device
memory (another allocator or a fixed budget owns it all, or the call sits in
a loop where an allocation could block).  It must give exactly what
vmo_bisect gives: the 2-means labels, the two centroids and the split flag,
bit for bit, which is the bar every bisection test here uses.  Its scratch is
one array shared by all calls, so each case makes two calls in a row, the
second on a smaller point set than the first, to show that nothing left by
the first call leaks into the second.  This file is collected last and also
runs alone in a fresh process: the fixture builds and loads the library
itself."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

MAX_POINTS = 131072


@pytest.fixture(scope="module")
def V():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1105_4490_gb300 as P
    assert torch.cuda.is_available()
    return P


def _same(a, b):
    ok_a, lab_a, z1_a, z2_a = a
    ok_b, lab_b, z1_b, z2_b = b
    assert ok_a == ok_b
    assert torch.equal(lab_a, lab_b)
    assert torch.equal(z1_a.view(torch.int32), z1_b.view(torch.int32))
    assert torch.equal(z2_a.view(torch.int32), z2_b.view(torch.int32))


@pytest.mark.parametrize("d", [2, 3, 4])
def test_noalloc_matches_bisect_two_calls(V, d):
    A = W.grid_laplacian_2d(400)  # 160,000 vertices: room for the maximum size
    hg = V.Hypergraph.from_matrix(A)
    x = V.init_coords(hg.k, d, seed=31)
    rng = np.random.default_rng(100 + d)
    sizes = [MAX_POINTS, int(rng.integers(2, 5000))]
    for nv in sizes:  # two calls in a row, largest first
        verts = torch.as_tensor(rng.choice(hg.k, nv, replace=False).astype(np.int32)).cuda()
        key = int(rng.integers(1, 1 << 40))
        for km in (0, 20):
            want = hg.bisect(x, verts, seed=5, key=key, km_iters=km, d=d)
            got = V.vmo.bisect_noalloc(x, verts, seed=5, key=key, km_iters=km, d=d)
            torch.cuda.synchronize()
            _same(got, want)


def test_noalloc_repeated_call_same_result(V):
    A = W.powerlaw_symmetric(6000, seed=3)
    hg = V.Hypergraph.from_matrix(A)
    x = V.init_coords(hg.k, 3, seed=7)
    verts = torch.arange(hg.k, dtype=torch.int32, device="cuda")
    want = hg.bisect(x, verts, seed=9, key=1, km_iters=20, d=3)
    first = V.vmo.bisect_noalloc(x, verts, seed=9, key=1, km_iters=20, d=3)
    second = V.vmo.bisect_noalloc(x, verts, seed=9, key=1, km_iters=20, d=3)
    _same(first, want)
    _same(second, want)


def test_noalloc_small_and_degenerate(V):
    A = W.grid_laplacian_2d(4)
    hg = V.Hypergraph.from_matrix(A)
    x = torch.zeros((16, 4), dtype=torch.float32, device="cuda")
    x[:, :2] = 3.0  # all points coincide: no split
    for nv in (16, 1, 0):
        verts = torch.arange(nv, dtype=torch.int32, device="cuda")
        want = hg.bisect(x, verts, seed=1, d=2)
        got = V.vmo.bisect_noalloc(x, verts, seed=1, d=2)
        _same(got, want)
        assert got[0] is False


def test_noalloc_rejects_oversize(V):
    x = torch.zeros((MAX_POINTS + 1, 4), dtype=torch.float32, device="cuda")
    verts = torch.arange(MAX_POINTS + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(V.VmoError, match="131072"):
        V.vmo.bisect_noalloc(x, verts, seed=1, d=3)


def test_noalloc_makes_no_device_allocation(V):
    """The defining property: around a warmed-up call through the C-ABI, with
    every output allocated beforehand by the caller, the library's own
    allocation counter and torch's allocator are unchanged (vmo_bisect, for
    contrast, does allocate, so the counter is live)."""
    import ctypes as C
    lib = V.load()
    A = W.powerlaw_symmetric(20000, seed=4)
    hg = V.Hypergraph.from_matrix(A)
    x = V.init_coords(hg.k, 3, seed=2)
    verts = torch.arange(hg.k, dtype=torch.int32, device="cuda")
    labels = torch.zeros(hg.k, dtype=torch.uint8, device="cuda")
    z = torch.zeros(8, dtype=torch.float32, device="cuda")
    split = C.c_int32()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call():
        st = lib.vmo_bisect_noalloc(3, C.c_void_p(x.data_ptr()), C.c_void_p(verts.data_ptr()), hg.k, 11, 1, 20,
                                    C.c_void_p(labels.data_ptr()), C.c_void_p(z.data_ptr()), C.byref(split), stream)
        assert st == 0

    call()  # warm-up: loads the library's device code on this device
    torch.cuda.synchronize()
    before_lib = V.stats()["device_allocations"]
    before_torch = torch.cuda.memory_allocated()
    for _ in range(2):
        call()
    torch.cuda.synchronize()
    assert V.stats()["device_allocations"] == before_lib
    assert torch.cuda.memory_allocated() == before_torch
    hg.bisect(x, verts, seed=11, key=1, km_iters=20, d=3)
    assert V.stats()["device_allocations"] > before_lib
