"""Writes work_counts.json: the work of the method on the measured workloads,
counted by the CPU oracle's counters (flops and bytes per kind of dense
operation; see the counter definitions in oracle/h2oracle.py).

Run from the repository root:  python tests/golden/make_work_counts.py
It calls only the oracle and the input generators; the benchmark reads the
JSON it writes as the algorithmic work of one product (the numerator of its
roofline fractions).
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import h2oracle as O  # noqa: E402
from paper_2403_01566_gb300 import inputs as I  # noqa: E402

CASES = [(128, 1e-6), (128, 1e-4), (128, 1e-8), (64, 1e-6)]


def main():
    out = {"what": "work of one product C = A*B counted by the oracle (numpy FP64, paper's algorithm)",
           "generator": "tests/golden/make_work_counts.py", "cases": {}}
    for grid, eps in CASES:
        w = I.grid_2d(grid, eps)
        X = O.build_h2(w.points, w.kernel_a.kind, w.kernel_a.kparam(), w.eta, w.leaf_size, w.order)
        Y = O.build_h2(w.points, w.kernel_b.kind, w.kernel_b.kparam(), w.eta, w.leaf_size, w.order, tree=X.rows)
        t0 = time.perf_counter()
        res = O.multiply(X, Y, eps)
        dt = time.perf_counter() - t0
        wk = res.stats["work"]
        key = f"{w.name}_eps{eps:g}"
        out["cases"][key] = {
            "n": w.n, "k": w.k, "eps": eps, "flops": wk["flops"], "bytes": wk["bytes"], "calls": wk["calls"],
            "total_flops": sum(wk["flops"].values()), "total_bytes": sum(wk["bytes"].values()),
            "agglomerated": res.agglomerated, "rank_max": max(max(res.ranks_row.values()), max(res.ranks_col.values())),
        }
        print(f"{key}: {sum(wk['flops'].values()) / 1e9:.3f} GFLOP, {sum(wk['bytes'].values()) / 1e9:.3f} GB, "
              f"{dt:.1f} s", flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "work_counts.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
