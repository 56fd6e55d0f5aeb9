"""The setup's step constant against the exact largest eigenvalue of A^T A.

bvls_setup takes L = 1.05 x the largest eigenvalue of the tridiagonal matrix of 32 Lanczos
steps on A^T A, a Rayleigh quotient of A^T A: it never exceeds 1.05 ||A||_2^2 (up to float32
rounding of the products) and, with 32 steps, comes within a small fraction of it.  The
reference ||A||_2^2 is numpy's float64 singular value.  A solve without an explicit step
constant reports the setup's L in its info.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2202_07258_gb300 as pkg
    return pkg


CASES = [
    # no spectral gap at the top of a Gaussian matrix's spectrum: 20 Lanczos steps land within
    # about 1e-3 of ||A||^2 (float64 replay), far inside the factor 1.05
    ("gaussian_2000x10000", lambda: W.nnls_gaussian(2000, 10000, 0.05, 0.01, 0), 5e-3),
    ("abs_1000x2000", lambda: W.nnls_abs_gaussian(1000, 2000, 0.05, 1.0, 0), 1e-5),
    ("bvls_224x512", lambda: W.bvls_dirichlet_shared(224, 512, 1, 8, 0.005, 0), 1e-5),
    ("abs_30x50", lambda: W.nnls_abs_gaussian(30, 50, 0.2, 1.0, 3), 1e-5),
    ("gaussian_40x8", lambda: W.nnls_gaussian(40, 8, 0.5, 0.01, 1), 1e-5),   # n below the step count
    # two and four float4 row chunks per thread in the Lanczos kernel (lda > 2048, > 4096)
    ("abs_3000x900", lambda: W.nnls_abs_gaussian(3000, 900, 0.05, 1.0, 2), 1e-5),
    ("abs_5000x700", lambda: W.nnls_abs_gaussian(5000, 700, 0.05, 1.0, 4), 1e-5),
]


@pytest.mark.parametrize("name,make,low", CASES, ids=[c[0] for c in CASES])
def test_step_constant_brackets_the_spectral_norm(P, name, make, low):
    p = make()
    A64 = np.asarray(p.A, dtype=np.float64)
    lam = float(np.linalg.norm(A64, 2) ** 2)
    dev = torch.device("cuda:0")
    s = P.Solver(torch.from_numpy(np.ascontiguousarray(p.A)).to(dev), p.l, p.u)
    y = torch.from_numpy(np.ascontiguousarray(np.asarray(p.y, np.float32).reshape(-1)[: p.A.shape[0]])).to(dev)
    x, scr, info, st = s.solve(y, tol=1e-3, max_iter=20)
    torch.cuda.synchronize()
    s.close()
    ratio = info["L"] / (1.05 * lam)
    assert ratio <= 1.0 + 1e-5, (name, ratio)        # a Rayleigh quotient: never above
    assert ratio >= 1.0 - low, (name, ratio)         # and close after 20 steps
