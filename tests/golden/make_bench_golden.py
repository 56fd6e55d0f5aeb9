"""Write tests/golden/bench_oracle.json: the FP64 oracle's own run of the benchmark workloads.

Calls only the oracle and the seeded generators.  The benchmark's CPU-baseline legs time
a bounded sample of oracle iterations and scale it by the iteration count recorded here
(the oracle's own count to the same gap, with its own step constant).

    python tests/golden/make_bench_golden.py [workload ...]
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402

WORKLOADS = {
    "nnls_gaussian_2000x10000": lambda: W.nnls_gaussian(2000, 10000, 0.05, 0.01, 0),
}


def main(names):
    path = os.path.join(HERE, "bench_oracle.json")
    out = json.load(open(path)) if os.path.exists(path) else {}
    for name in names:
        p = WORKLOADS[name]()
        A = p.A.astype(np.float64)
        y = p.y.astype(np.float64)
        L = O.lipschitz(A)
        rec = {"L": L, "tol": 1e-6, "screen_every": 10}
        t0 = time.perf_counter()
        r = O.solve(A, y, p.l, p.u, tol=1e-6, screen_every=10, L=L, max_iter=200000)
        rec.update(iters=r.iters, gap=r.gap, primal=r.primal, converged=bool(r.converged),
                   dual_mode=r.dual_mode, n_screened=int((r.screened > 0).sum()),
                   seconds=time.perf_counter() - t0)
        out[name] = rec
        print(name, rec, flush=True)
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(WORKLOADS))
