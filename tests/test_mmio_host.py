"""Matrix Market input and output (host, no GPU): every field and symmetry
read as scipy.io reads it (symmetric storage expanded, duplicates summed,
complex entries as their modulus), round trips through our writer and
scipy's reader, and malformed files refused."""
import numpy as np
import pytest

import workloads as W

sp = pytest.importorskip("scipy.sparse")
sio = pytest.importorskip("scipy.io")
pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


@pytest.fixture(scope="module")
def V():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1105_4490_gb300 as P
    return P


def _same(B, M, values=True):
    M = sp.csr_matrix(M)
    M.sum_duplicates()
    M.sort_indices()
    assert (B.m, B.n) == M.shape
    assert np.array_equal(B.rowptr, M.indptr) and np.array_equal(B.colidx, M.indices)
    if values:
        assert np.allclose(B.values, M.data.astype(np.float64), rtol=1e-6, atol=0)


def _random(m, n, nnz, seed, symmetric=None):
    A = W.random_pattern(m, n, nnz, seed)
    rows = np.repeat(np.arange(m), np.diff(A.rowptr))
    vals = np.random.default_rng(seed).uniform(-3, 3, size=A.nnz)
    M = sp.coo_matrix((vals, (rows, A.colidx)), shape=(m, n)).tocsr()
    if symmetric == "symmetric":
        M = sp.tril(M) + sp.tril(M, -1).T
    elif symmetric == "skew":
        M = sp.tril(M, -1) - sp.tril(M, -1).T
    return sp.csr_matrix(M)


@pytest.mark.parametrize("kind", ["general", "symmetric", "skew-symmetric", "pattern", "integer", "hermitian"])
def test_read_like_scipy(V, tmp_path, kind):
    p = tmp_path / f"{kind}.mtx"
    if kind == "general":
        M = _random(300, 200, 1500, 1)
        sio.mmwrite(str(p), M)
    elif kind == "symmetric":
        M = _random(250, 250, 1200, 2, "symmetric")
        sio.mmwrite(str(p), M, symmetry="symmetric")
    elif kind == "skew-symmetric":
        M = _random(250, 250, 1200, 3, "skew")
        sio.mmwrite(str(p), M, symmetry="skew-symmetric")
    elif kind == "pattern":
        M = _random(120, 180, 700, 4)
        M.data[:] = 1.0
        sio.mmwrite(str(p), M, field="pattern")
    elif kind == "integer":
        M = _random(150, 150, 900, 5)
        M.data = np.round(M.data * 10)
        M.eliminate_zeros()
        sio.mmwrite(str(p), M.astype(np.int64), field="integer")
    else:
        R = _random(100, 100, 600, 6, "symmetric")
        Im = _random(100, 100, 600, 7, "skew")
        M = (R + 1j * Im).tocsr()
        M.eliminate_zeros()
        sio.mmwrite(str(p), M, symmetry="hermitian")
    B = V.read_matrix_market(str(p))
    want = sio.mmread(str(p))
    if kind == "hermitian":
        want = abs(sp.csr_matrix(want))
    _same(B, want)


def test_stored_triangle_only(V, tmp_path):
    M = _random(200, 200, 900, 8, "symmetric")
    p = tmp_path / "s.mtx"
    sio.mmwrite(str(p), M, symmetry="symmetric")
    B = V.read_matrix_market(str(p), expand_symmetric=False)
    _same(B, sp.tril(sio.mmread(str(p))))


def test_duplicates_summed_and_round_trips(V, tmp_path):
    p = tmp_path / "dup.mtx"
    p.write_text("%%MatrixMarket matrix coordinate real general\n% a comment\n3 4 5\n"
                 "1 2 1.5\n3 4 -2\n1 2 0.5\n2 1 7\n% inside\n3 1 1e-3\n")
    B = V.read_matrix_market(str(p))
    assert B.m == 3 and B.n == 4 and B.nnz == 4
    assert B.rowptr.tolist() == [0, 1, 2, 4] and B.colidx.tolist() == [1, 0, 0, 3]
    assert np.allclose(B.values, [2.0, 7.0, 1e-3, -2.0])
    q = tmp_path / "out.mtx"
    V.write_matrix_market(str(q), B)
    _same(V.read_matrix_market(str(q)), sio.mmread(str(q)))
    _same(V.read_matrix_market(str(q)), sp.csr_matrix((B.values, B.colidx, B.rowptr), shape=(3, 4)))
    A = W.powerlaw_symmetric(2000, seed=3)
    V.write_matrix_market(str(q), A, values=np.ones(A.nnz))
    C2 = V.read_matrix_market(str(q))
    assert np.array_equal(C2.rowptr, A.rowptr) and np.array_equal(C2.colidx, A.colidx)
    r = tmp_path / "pat.mtx"
    V.write_matrix_market(str(r), V.HostMatrix("p", A.m, A.n, A.rowptr, A.colidx, None))
    assert r.read_text().startswith("%%MatrixMarket matrix coordinate pattern general")
    P = V.read_matrix_market(str(r))
    assert np.array_equal(P.colidx, A.colidx) and (P.values == 1).all()


@pytest.mark.parametrize("text", [
    "",
    "not a banner\n1 1 1\n1 1 1\n",
    "%%MatrixMarket matrix array real general\n2 2\n1\n2\n3\n4\n",
    "%%MatrixMarket matrix coordinate real general\n2 2 1\n3 1 1.0\n",
    "%%MatrixMarket matrix coordinate real general\n2 2 2\n1 1 1.0\n",
    "%%MatrixMarket matrix coordinate real symmetric\n2 3 1\n1 1 1.0\n",
    "%%MatrixMarket matrix coordinate widget general\n2 2 1\n1 1 1.0\n",
])
def test_malformed_refused(V, tmp_path, text):
    p = tmp_path / "bad.mtx"
    p.write_text(text)
    with pytest.raises(V.VmoError):
        V.read_matrix_market(str(p))
    with pytest.raises(V.VmoError):
        V.read_matrix_market(str(tmp_path / "missing.mtx"))
