"""The host preprocessing that supplies a strengthened diagonal
(vmo_perfect_matching_host: heavy-edge start, Hopcroft-Karp augmentation),
checked against scipy's maximum bipartite matching on square patterns with
and without a perfect matching, the heavy-edge rule, and refused inputs.  It
runs on the host: no GPU needed."""
import numpy as np
import pytest

import workloads as W

sp = pytest.importorskip("scipy.sparse")
csgraph = pytest.importorskip("scipy.sparse.csgraph")


@pytest.fixture(scope="module")
def V():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1105_4490_gb300 as P
    return P


def _dense_entries(A):
    rows = np.repeat(np.arange(A.m), np.diff(A.rowptr))
    return set(zip(rows.tolist(), A.colidx.tolist()))


def _check_valid(A, match):
    ent = _dense_entries(A)
    used = match[match >= 0]
    assert len(set(used.tolist())) == len(used)
    assert all((i, int(c)) in ent for i, c in enumerate(match) if c >= 0)


def _scipy_size(A):
    M = sp.csr_matrix((np.ones(A.nnz), A.colidx, A.rowptr), shape=(A.m, A.m))
    return int((csgraph.maximum_bipartite_matching(M, perm_type="column") >= 0).sum())


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_planted_perfect_matching_found(V, seed):
    A = W.with_strengthened_diagonal(W.powerlaw_symmetric(3000, seed=seed), 0.5, seed)
    match, size = V.perfect_matching(A)
    assert size == A.m and sorted(match.tolist()) == list(range(A.m))
    _check_valid(A, match)


@pytest.mark.parametrize("seed,nnz", [(1, 400), (2, 900), (3, 2500), (4, 6000), (5, 20000)])
def test_maximum_size_equals_scipy(V, seed, nnz):
    """Random patterns from structurally singular to nonsingular: the size of
    the matching equals the maximum (scipy); a perfect one is returned, and
    otherwise the call refuses with the maximum matching in `match`."""
    A = W.random_pattern(1200, 1200, nnz, seed)
    want = _scipy_size(A)
    if want == A.m:
        match, size = V.perfect_matching(A)
        assert size == A.m
        _check_valid(A, match)
    else:
        with pytest.raises(V.VmoError) as e:
            V.perfect_matching(A)
        assert e.value.status == 6  # VMO_ERR_UNSUPPORTED
        import ctypes as C
        from paper_1105_4490_gb300 import vmo
        match = np.empty(A.m, dtype=np.int32)
        got = C.c_int32(0)
        st = vmo.load().vmo_perfect_matching_host(A.m, A.rowptr.ctypes.data, A.colidx.ctypes.data, None,
                                                 match.ctypes.data, C.byref(got))
        assert st == 6 and got.value == want == int((match >= 0).sum())
        _check_valid(A, match)


def test_heavy_entries_first(V):
    """With the diagonal heavier than everything else the heavy-edge start is
    the whole diagonal; with a heavier shifted diagonal (a cyclic shift that
    is also a perfect matching of the pattern) it is that shift."""
    n = 500
    rows = np.concatenate([np.arange(n), np.arange(n), np.arange(n)])
    cols = np.concatenate([np.arange(n), (np.arange(n) + 1) % n, (np.arange(n) + 7) % n])
    A = W.csr_from_coo(n, n, rows, cols, "three_diagonals")
    r = np.repeat(np.arange(n), np.diff(A.rowptr))
    vals = np.where(A.colidx == r, 10.0, 1.0).astype(np.float32)
    match, _ = V.perfect_matching(A, vals)
    assert np.array_equal(match, np.arange(n))
    vals = np.where(A.colidx == (r + 7) % n, -20.0, 1.0).astype(np.float32)  # |value| counts
    match, _ = V.perfect_matching(A, vals)
    assert np.array_equal(match, (np.arange(n) + 7) % n)


def test_refused_inputs(V):
    A = W.with_strengthened_diagonal(W.grid_laplacian_2d(8), 0.5, 1)
    bad_vals = np.ones(A.nnz, dtype=np.float32)
    bad_vals[3] = np.nan
    with pytest.raises(V.VmoError):
        V.perfect_matching(A, bad_vals)
    B = W.Matrix("bad", A.m, A.m, A.rowptr.copy(), A.colidx.copy(), {})
    B.colidx[5] = A.m
    with pytest.raises(V.VmoError):
        V.perfect_matching(B)
    C2 = W.Matrix("bad", A.m, A.m, A.rowptr.copy(), A.colidx.copy(), {})
    C2.rowptr[3], C2.rowptr[4] = C2.rowptr[4], C2.rowptr[3] + 0
    C2.rowptr[4] = C2.rowptr[3] - 1
    with pytest.raises(V.VmoError):
        V.perfect_matching(C2)
    E = W.csr_from_coo(0, 0, np.array([], int), np.array([], int), "empty")
    match, size = V.perfect_matching(E)
    assert size == 0 and match.size == 0
