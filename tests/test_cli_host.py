"""The command line's host parts (no GPU): argument checks and the permuted
matrix it writes."""
import os
import subprocess
import sys

import numpy as np
import pytest

import workloads as W


def test_help_and_argument_errors():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-m", "paper_1105_4490_gb300", "--help"], capture_output=True, text=True,
                       cwd=root)
    assert r.returncode == 0 and "Matrix Market" in r.stdout
    from paper_1105_4490_gb300.__main__ import parse
    a = parse(["m.mtx", "out", "--sbd", "--cut-order", "2"])
    assert a.sbd and a.cut_order == 2 and a.model is None
    for bad in (["m.mtx"], ["m.mtx", "o", "--cut-order", "9"], ["m.mtx", "o", "--matched", "--model", "symmetric"],
                ["m.mtx", "o", "--d", "5"]):
        with pytest.raises(SystemExit):
            parse(bad)


def test_permuted_matrix():
    """Entry (i, j) of the input lands at (inverse row perm of i, inverse column
    perm of j) with its value; the result is a valid sorted CSR."""
    from paper_1105_4490_gb300.__main__ import permuted
    A = W.random_pattern(60, 45, 300, 5)
    rng = np.random.default_rng(5)
    rp, cp = rng.permutation(60), rng.permutation(45)
    vals = rng.uniform(size=A.nnz)

    class M:
        m, n, rowptr, colidx, values = A.m, A.n, A.rowptr, A.colidx, vals

    B = permuted(M, rp, cp)
    dense = np.zeros((60, 45))
    dense[np.repeat(np.arange(60), np.diff(A.rowptr)), A.colidx] = vals
    got = np.zeros((60, 45))
    got[np.repeat(np.arange(60), np.diff(B.rowptr)), B.colidx] = B.values
    assert np.array_equal(got, dense[np.ix_(rp, cp)])
    for i in range(60):
        row = B.colidx[B.rowptr[i]:B.rowptr[i + 1]]
        assert (np.diff(row) > 0).all()
