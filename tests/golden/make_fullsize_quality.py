"""Writes fullsize_quality.json: the oracle's own full runs (multilevel
layout of Algorithm 3 with Algorithm 4 on every level, then the recursive
ordering of Algorithm 7) on the full-size benchmark workloads, three seeds
each, and the quality metrics the GPU's full runs are held to (within 5%):

* 64^3 7-point grid (symmetric model, d = 3, BBD, depth 10): fill
  (nz(L) + nz(U) - n) / nz(A) of LU without pivoting of the ordered matrix
  (Table 2's measure), and the separator totals;
* 500,000-row power-law pattern (symmetric, d = 3, BBD, depth 10): the
  separator total sum |V3| and the largest separator max |V3| (Table 3's
  measure);
* 400,000 x 300,000 power-law pattern (bipartite model, d = 2, SBD to depth
  6, 64 parts): lambda - 1 and the cut nets of the final parts over the row
  nets and the column nets, and the separator totals.

Calls only the oracle (test infrastructure).  Run from the repository root:
python tests/golden/make_fullsize_quality.py"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402

SEEDS = (1, 2, 3)
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fullsize_quality.json")


def sep_stats(tree):
    ns = tree["nsep"].astype(np.int64)
    return {"sum_sep": int(ns.sum()), "max_sep": int(ns.max())}


def run():
    O.build()
    res = {"generator": "tests/golden/make_fullsize_quality.py (oracle only)", "seeds": list(SEEDS),
           "oracle_threads": O.threads(), "cases": {}}
    cases = [
        ("grid3d_64", lambda: W.grid_laplacian_3d(64), "symmetric", 3, False, 10, 64),
        ("powerlaw_500k", lambda: W.powerlaw_symmetric(500_000, seed=1), "symmetric", 3, False, 10, 64),
        ("rect_400k_300k_sbd", lambda: W.powerlaw_rectangular(400_000, 300_000, seed=1), "bipartite", 2, True, 6, 1),
    ]
    for name, make, model, d, sbd, depth, min_part in cases:
        A = make()
        hg = O.build_from_matrix(model, A)
        runs = []
        for seed in SEEDS:
            t0 = time.time()
            x = O.layout_multilevel(hg, d, seed)
            perm, tree = O.order(hg, d, x.astype(np.float32), seed=seed, min_part=min_part, max_depth=depth, sbd=sbd)
            r = {"seed": seed, **sep_stats(tree)}
            if name == "grid3d_64":
                r["fill"] = O.fill_in(A, perm)
            if model == "bipartite":
                part = O.parts_from_tree(hg.k, perm, tree, sbd=sbd)
                rows, cols = part[:A.m], part[A.m:]
                rn = O.build_from_matrix("rownet", A)
                cn = O.build_from_matrix("colnet", A)
                c1, l1 = O.cut_size(rn.net_ptr, rn.pins, cols)
                c2, l2 = O.cut_size(cn.net_ptr, cn.pins, rows)
                r.update(cut_nets=c1 + c2, lambda_minus_1=l1 + l2)
            r["seconds"] = round(time.time() - t0, 1)
            runs.append(r)
            print(name, r, flush=True)
        res["cases"][name] = {"model": model, "d": d, "sbd": sbd, "max_depth": depth, "min_part": min_part,
                              "m": A.m, "n": A.n, "nnz": int(A.nnz), "runs": runs}
    with open(OUT, "w") as f:
        json.dump(res, f, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    run()
