"""Command line: order a Matrix Market file.

    python -m paper_1105_4490_gb300 matrix.mtx out [--sbd] [--model bipartite] [--matched]
        [--d 3] [--max-depth 62] [--min-part 64] [--sep-recursion] [--cut-order B] [--seed 1]
        [--permuted]

Reads the file (vmo_read_matrix_market), builds the hypergraph model on the
GPU, lays it out and orders it (recursive BBD, or SBD with --sbd), and writes
`out.rowperm` and `out.colperm` (the old row / column index at every new
position, 0-based, one per line) and, with --permuted, the permuted matrix as
`out.mtx`.  --matched (square matrices, bipartite model) keeps a strengthened
diagonal computed by vmo_perfect_matching_host from the file's values.
"""
from __future__ import annotations

import argparse
import sys
import time


def parse(argv):
    ap = argparse.ArgumentParser(prog="python -m paper_1105_4490_gb300", description=__doc__.split("\n\n")[0])
    ap.add_argument("matrix", help="Matrix Market coordinate file")
    ap.add_argument("out", help="output prefix (writes OUT.rowperm, OUT.colperm, OUT.mtx)")
    ap.add_argument("--sbd", action="store_true", help="separated block diagonal (separator between the parts)")
    ap.add_argument("--model", choices=["symmetric", "bipartite"], default=None,
                    help="hypergraph model (default: symmetric for square matrices, else bipartite)")
    ap.add_argument("--matched", action="store_true",
                    help="keep a strengthened diagonal (square matrix, bipartite model)")
    ap.add_argument("--d", type=int, default=3, choices=[2, 3, 4], help="layout dimension")
    ap.add_argument("--max-depth", type=int, default=62)
    ap.add_argument("--min-part", type=int, default=64)
    ap.add_argument("--sep-recursion", action="store_true", help="order every separator recursively as well")
    ap.add_argument("--cut-order", type=int, default=0, metavar="B", help="two-bit cut-row ordering to B levels")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--permuted", action="store_true", help="also write the permuted matrix")
    a = ap.parse_args(argv)
    if a.matched and a.model == "symmetric":
        ap.error("--matched needs the bipartite model")
    if not 0 <= a.cut_order <= 8:
        ap.error("--cut-order must be in [0, 8]")
    return a


def permuted(A, row_perm, col_perm):
    """The matrix with row row_perm[t] and column col_perm[t] moved to position
    t (a HostMatrix, columns sorted within rows)."""
    import numpy as np

    from .vmo import HostMatrix
    inv_r = np.empty(A.m, dtype=np.int64)
    inv_r[np.asarray(row_perm)] = np.arange(A.m)
    inv_c = np.empty(A.n, dtype=np.int64)
    inv_c[np.asarray(col_perm)] = np.arange(A.n)
    rows = np.repeat(np.arange(A.m), np.diff(A.rowptr))
    nr, nc = inv_r[rows], inv_c[np.asarray(A.colidx)]
    order = np.lexsort((nc, nr))
    rowptr = np.zeros(A.m + 1, dtype=np.int32)
    np.cumsum(np.bincount(nr, minlength=A.m), out=rowptr[1:])
    values = getattr(A, "values", None)
    values = values() if callable(values) else values
    vals = None if values is None else np.asarray(values)[order]
    return HostMatrix("permuted", A.m, A.n, rowptr, nc[order].astype(np.int32), vals)


def main(argv=None) -> int:
    a = parse(sys.argv[1:] if argv is None else argv)
    import numpy as np
    import torch

    from . import vmo as V
    A = V.read_matrix_market(a.matrix)
    model = a.model or ("symmetric" if A.m == A.n and not a.matched else "bipartite")
    if a.matched and A.m != A.n:
        print("--matched needs a square matrix", file=sys.stderr)
        return 2
    p = V.Params(d=a.d, max_depth=a.max_depth, min_part=a.min_part, sep_recursion=int(a.sep_recursion),
                 cut_order=a.cut_order, seed=a.seed)
    t0 = time.perf_counter()
    hg = V.Hypergraph.from_matrix(A, model)
    if a.matched:
        match, _ = V.perfect_matching(A, A.values)
        rp, cp, _, _ = hg.order_matched(torch.as_tensor(match), p, sbd=a.sbd)
    else:
        rp, cp, _ = hg.order(p, sbd=a.sbd, with_tree=False)
    rp, cp = rp.cpu().numpy(), cp.cpu().numpy()
    dt = time.perf_counter() - t0
    np.savetxt(a.out + ".rowperm", rp, fmt="%d")
    np.savetxt(a.out + ".colperm", cp, fmt="%d")
    if a.permuted:
        V.write_matrix_market(a.out + ".mtx", permuted(A, rp, cp))
    print(f"{a.matrix}: {A.m} x {A.n}, {A.nnz} nnz, {model} model, {'SBD' if a.sbd else 'BBD'}"
          f"{' matched' if a.matched else ''}: ordered in {dt:.3f} s ({A.nnz / dt / 1e6:.2f} M nnz/s incl. copies)")
    return 0


if __name__ == "__main__":
    sys.exit(main())
