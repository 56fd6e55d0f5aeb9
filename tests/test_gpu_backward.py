"""GPU parity of the backward pass (bvls_backward) against the FP64 oracle's dense
free-set solve (itself pinned by central differences in test_oracle_backward.py), plus an
end-to-end central-difference check through the GPU forward and the autograd wrapper."""
import numpy as np
import pytest

import oracle as O
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


def certified(A, y, x, l, u):
    xs = O.polish(A, y, x, l, u, tau=1e-7)
    assert O.kkt_residual(A, y, xs, l, u) < 1e-9 * (1 + np.abs(A.T @ y).max())
    F = O.free_set(xs, l, u)
    g = A.T @ (y - A @ xs)
    B = np.setdiff1d(np.arange(A.shape[1]), F)
    assert np.linalg.matrix_rank(A[:, F]) == F.size and np.abs(g[B]).min() > 1e-7   # non-degenerate
    return xs


def test_backward_matches_oracle_at_the_same_point(P):
    """Differentiable-NNLS shape with a unique optimum: A 256 x 1024 |N(0,1)|, noise N(0,1)."""
    p = W.nnls_shared(256, 1024, 6, 0.08, 1.0, 11, abs_matrix=True, x_low=0.1)
    A = p.A.astype(np.float64)
    dev = torch.device("cuda:0")
    s = P.Solver(torch.from_numpy(p.A).to(dev), p.l, p.u)
    Xg, S, gaps, its, sts, info, st = s.solve_batched(torch.from_numpy(p.y).to(dev), tol=1e-8, precision="fp32x2")
    assert st == P.BVLS_OK
    Xg = Xg.cpu().numpy()
    rng = np.random.default_rng(0)
    XS = np.stack([certified(A, p.y[b].astype(np.float64), Xg[b], p.l, p.u) for b in range(6)])
    V = rng.standard_normal(XS.shape)
    dY, dA, bst, binfo = s.backward(XS, p.y, V)
    assert np.all(bst == 0) and binfo["n_converged"] == 6
    dA_ref = np.zeros_like(A)
    for b in range(6):
        dy, da, F, w = O.backward(A, p.y[b].astype(np.float64), XS[b], V[b], p.l, p.u)
        assert np.allclose(dY[b], dy, rtol=1e-7, atol=1e-9 * np.abs(dy).max()), b
        dA_ref += da
    assert np.allclose(dA, dA_ref, rtol=1e-7, atol=1e-9 * np.abs(dA_ref).max())
    # the work counters: every instance's CG ran on its free set (oracle's |F|), within the maxima
    nF = [O.backward(A, p.y[b].astype(np.float64), XS[b], V[b], p.l, p.u)[2].size for b in range(6)]
    assert binfo["max_free"] == max(nF)
    assert 0 < binfo["cg_work"] <= 6 * binfo["max_cg_iters"] * binfo["max_free"]
    assert binfo["cg_work"] >= binfo["max_cg_iters"] * min(nF)
    assert binfo["kernel_ms"] > 0
    s.close()


def test_backward_end_to_end_central_differences(P):
    """GPU forward (gap 1e-10), the FP64 polish of its free set, then GPU backward, against
    central differences of the loss at exact solutions of the perturbed problems (scipy's
    active-set BVLS, test harness only).  A rigorous NNLS gap cannot go much below 1e-11
    here: the rounding margin of the correlations enters the translation step."""
    from scipy.optimize import lsq_linear
    p = W.nnls_abs_gaussian(30, 50, 0.2, 1.0, 3)
    A = p.A.astype(np.float64)
    y = p.y.astype(np.float64)

    def exact(Ap, yp):
        r = lsq_linear(Ap, yp, bounds=(p.l, p.u), method="bvls", tol=1e-15)
        return O.polish(Ap, yp, r.x, p.l, p.u, tau=1e-9)

    xt = np.random.default_rng(2).uniform(0, 1, 50)
    loss = lambda x: 0.5 * float((x - xt) @ (x - xt))
    dev = torch.device("cuda:0")
    s = P.Solver(torch.from_numpy(p.A).to(dev), p.l, p.u)
    X, S, gaps, its, sts, info, st = s.solve_batched(torch.from_numpy(p.y[None]).to(dev), tol=1e-10,
                                                     precision="fp32x2", max_iter=200000)
    assert st == P.BVLS_OK and gaps[0].item() < 1e-10
    x = O.polish(A, y, X[0].cpu().numpy(), p.l, p.u, tau=1e-7)
    assert np.abs(x - X[0].cpu().numpy()).max() < 1e-4 and O.kkt_residual(A, y, x, p.l, p.u) < 1e-12
    X = torch.from_numpy(x[None]).to(dev)
    dY, dA, bst, binfo = s.backward(X, torch.from_numpy(p.y[None]).to(dev), X - torch.from_numpy(xt[None]).to(dev))
    dY, dA = dY[0].cpu().numpy(), dA.cpu().numpy()
    assert int(bst[0]) == 0
    h = 1e-4
    for i in range(0, 30, 3):
        e = np.zeros(30)
        e[i] = h
        fd = (loss(exact(A, y + e)) - loss(exact(A, y - e))) / (2 * h)
        assert abs(fd - dY[i]) <= 2e-5 * (1 + abs(fd)), (i, fd, dY[i])
    F = O.free_set(x, p.l, p.u)
    for j in list(F[:3]) + [int(np.setdiff1d(np.arange(50), F)[0])]:
        for i in (0, 17):
            Ap, Am = A.copy(), A.copy()
            Ap[i, j] += h
            Am[i, j] -= h
            fd = (loss(exact(Ap, y)) - loss(exact(Am, y))) / (2 * h)
            assert abs(fd - dA[i, j]) <= 2e-5 * (1 + abs(fd)), (i, j, fd, dA[i, j])
    s.close()


def test_autograd_wrapper_matches_direct_call(P):
    p = W.nnls_shared(64, 160, 5, 0.1, 1.0, 4, abs_matrix=True, x_low=0.1)
    dev = torch.device("cuda:0")
    A = torch.from_numpy(p.A).to(dev).requires_grad_(True)
    Y = torch.from_numpy(p.y).to(dev).requires_grad_(True)
    Xt = torch.rand(5, 160, dtype=torch.float64, device=dev)
    X, S = P.solve_batched_autograd(A, Y, p.l, p.u, tol=1e-10, precision="fp32x2")
    loss = 0.5 * ((X - Xt) ** 2).sum()
    loss.backward()
    s = P.Solver(A.detach(), p.l, p.u)
    dY, dA, bst, _ = s.backward(X.detach(), Y.detach(), (X - Xt).detach())
    assert torch.allclose(Y.grad.double(), dY.to(Y.grad.device), rtol=1e-5, atol=1e-6)
    assert torch.allclose(A.grad.double(), dA, rtol=1e-5, atol=1e-6)
    s.close()


def test_free_set_over_the_limit_gives_status_2(P):
    rng = np.random.default_rng(5)
    m = n = 1100
    A = rng.standard_normal((m, n)).astype(np.float32)
    dev = torch.device("cuda:0")
    s = P.Solver(torch.from_numpy(A).to(dev), -np.ones(n), np.ones(n))
    X = torch.from_numpy(rng.uniform(-0.5, 0.5, (2, n))).to(dev)          # every coordinate free
    Y = torch.from_numpy(rng.standard_normal((2, m)).astype(np.float32)).to(dev)
    dY, dA, bst, info = s.backward(X, Y, torch.ones(2, n, dtype=torch.float64, device=dev))
    assert torch.all(bst == 2) and info["n_too_large"] == 2 and info["max_free"] == n
    assert torch.all(dY == 0)
    s.close()


def test_free_set_larger_than_m_is_declined(P):
    """Gaussian A with n = 4m (the degenerate differentiable-NNLS shape): an optimum with more
    than m positive coordinates cannot have A_F of full column rank, so it is not unique and
    has no derivative.  Those instances get status 3, zero gradients and no CG iterations; the
    others are solved as usual."""
    p = W.nnls_shared(40, 160, 8, 0.08, 0.01, 21, abs_matrix=False, x_low=0.1)
    dev = torch.device("cuda:0")
    s = P.Solver(torch.from_numpy(p.A).to(dev), p.l, p.u)
    X, S, gaps, its, sts, info, st = s.solve_batched(torch.from_numpy(p.y).to(dev), tol=1e-8, precision="fp32x2")
    assert st == P.BVLS_OK
    X = X.cpu().numpy()
    V = np.random.default_rng(2).standard_normal(X.shape)
    dY, dA, bst, binfo = s.backward(X, p.y, V)
    s.close()
    nfree = (X > 1e-9).sum(axis=1)        # l = 0, u = +inf: free means x_j > free_tol (1 + |l_j|)
    assert np.array_equal(bst == 3, nfree > p.m), (bst, nfree)
    assert np.any(bst == 3)
    assert binfo["n_not_unique"] == int((bst == 3).sum())
    assert np.all(dY[bst == 3] == 0.0)
    assert binfo["cg_work"] <= binfo["max_cg_iters"] * int(nfree[bst != 3].sum())
