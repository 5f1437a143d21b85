"""Writes tests/golden/grid64_oracle.json by calling the oracle only.

Workload: the 64 x 64 unit-weight grid (4,096 nodes, 8,064 edges), K = 8
test vectors from seed 0, 5 weighted-Jacobi sweeps (omega = 0.7), one level
of two-pass aggregation to a target of 1,024 nodes, Galerkin coarsening.
Run from the repository root:  python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import workloads as W  # noqa: E402


def main():
    g = W.grid2d(64, 64)
    X = oracle.smooth(g.n, g.u, g.v, g.w, 8, 5, 0.7, 0, 0)
    d = oracle.affinity(g.n, g.u, g.v, X)
    agg, nc = oracle.aggregate(g.n, g.u, g.v, d, 1024, 2)
    uc, vc, wc = oracle.coarsen(g.n, g.u, g.v, g.w, agg, nc)
    ev = oracle.smallest_nontrivial_eigs(nc, uc, vc, wc, 10)
    out = {
        "workload": "grid2d 64x64, K=8, seed 0, 5 sweeps, omega 0.7, target 1024, 2 passes",
        "X_sha256": hashlib.sha256(X.tobytes()).hexdigest(),
        "d_sha256": hashlib.sha256(d.tobytes()).hexdigest(),
        "agg_sha256": hashlib.sha256(agg.tobytes()).hexdigest(),
        "nc": int(nc),
        "mc": int(len(uc)),
        "wc_sum": float(wc.sum()),
        "eig10": [float(x) for x in ev],
    }
    with open(os.path.join(HERE, "grid64_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
