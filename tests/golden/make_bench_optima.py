"""Write tests/golden/bench_optima.json: FP64 optima of the benchmark's workloads.

Calls only the oracle and the seeded generators.  For each workload (and, for batches, a
fixed sample of instances) the oracle solves to a tight gap, its polish step re-solves the
free set, and the result is kept when it satisfies the optimality conditions of Section 3.2
(KKT residual below 1e-9 relative) with a free set smaller than m and independent free
columns, i.e. when it is the unique optimum.  The benchmark reads these optima to report the
error of each GPU result against the FP64 oracle.  Where the optimum is not unique (P* = 0,
the Gaussian workloads with n >= 2m) only the oracle's objective is recorded.

    python tests/golden/make_bench_optima.py [name ...]
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

BATCH_SAMPLE = [0, 1, 2, 3, 1024, 2047, 3071, 4095]
RAGGED_SAMPLE = [0, 1, 2, 3, 62, 63]


def single(make, tol):
    def run():
        p = make()
        return [(None, p.A, p.y.reshape(-1), p.l, p.u, tol)]
    return run


def batch_sample():
    p = W.bvls_dirichlet_shared(224, 512, 4096, 8, 0.005, 0)
    return [(b, p.A, p.y[b], p.l, p.u, 1e-10) for b in BATCH_SAMPLE]


def ragged_sample():
    probs = W.mixed_uneven(64, 0, abs_matrix=True, noise=1.0)
    return [(k, probs[k].A, probs[k].y, probs[k].l, probs[k].u, 1e-9) for k in RAGGED_SAMPLE]


WORKLOADS = {
    "nnls_abs_gaussian_2000x10000": single(lambda: W.nnls_abs_gaussian(2000, 10000, 0.05, 1.0, 0), 1e-8),
    "bvls_table2_1000x2000": single(lambda: W.bvls_table2(1000, 2000, 0), 1e-10),
    "bvls_dirichlet_224x512_B4096": batch_sample,
    "mixed_uneven_abs_B64": ragged_sample,
}


def optimum(A, y, l, u, tol):
    A = A.astype(np.float64)
    y = y.astype(np.float64)
    t0 = time.perf_counter()
    r = O.solve(A, y, l, u, tol=tol, screen_every=10, max_iter=400000)
    # the free set of the polish step is read off the solve's iterate with a margin tau; the
    # first margin whose polished point passes the optimality conditions is kept
    bound = 1e-9 * (1 + float(np.abs(A.T @ y).max()))
    for tau in (1e-7, 1e-9, 1e-6, 1e-5):
        xs = O.polish(A, y, r.x, l, u, tau=tau)
        kkt = O.kkt_residual(A, y, xs, l, u)
        if kkt < bound:
            break
    F = O.free_set(xs, l, u, 1e-7)
    inside = bool(np.all(xs >= l - 1e-12) and np.all(xs <= u + 1e-12))
    unique = inside and F.size < A.shape[0] and np.linalg.matrix_rank(A[:, F]) == F.size
    ok = unique and kkt < bound
    rec = {"m": int(A.shape[0]), "n": int(A.shape[1]), "oracle_iters": int(r.iters), "oracle_gap": float(r.gap),
           "oracle_P": float(r.primal), "seconds": time.perf_counter() - t0}
    if ok:
        nz = np.flatnonzero(xs)
        rec.update(unique=True, P_star=O.primal_objective(A, y, xs), kkt=float(kkt), free_set=int(F.size),
                   x_star_idx=[int(i) for i in nz], x_star_val=[float(v) for v in xs[nz]])
    else:
        rec.update(unique=False)
    return rec


def main(names):
    path = os.path.join(HERE, "bench_optima.json")
    out = json.load(open(path)) if os.path.exists(path) else {}
    for name in names:
        recs = {}
        for key, A, y, l, u, tol in WORKLOADS[name]():
            rec = optimum(A, y, l, u, tol)
            recs["single" if key is None else str(key)] = rec
            print(name, key, {k: v for k, v in rec.items() if not k.startswith("x_star")}, flush=True)
        out[name] = recs
        with open(path, "w") as f:
            json.dump(out, f, indent=0, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(WORKLOADS))
