"""GPU parity of the ragged batch (independent problems of uneven sizes, mixed NNLS / BVLS)
against the FP64 oracle, instance by instance: certified gap, zero false screens, and the
solution against an optimum certified by the optimality conditions of Section 3.2."""
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


def run(P, probs, device=True, **kw):
    dev = torch.device("cuda:0")
    items = []
    for p in probs:
        A = torch.from_numpy(p.A).to(dev) if device else p.A
        y = torch.from_numpy(p.y).to(dev) if device else p.y
        items.append((A, y, p.l, p.u))
    return P.solve_ragged(items, **kw)


def check(p, x, scr, gap, status, tol, xtol=None):
    A, y = p.A.astype(np.float64), p.y.astype(np.float64)
    assert status == 0 and gap < tol, (p.name, status, gap)
    ref = O.solve(A, y, p.l, p.u, tol=min(tol, 1e-9) * 1e-1)
    Ps = O.primal_objective(A, y, ref.x)
    Pg = O.primal_objective(A, y, x)
    assert np.all(x >= p.l) and np.all(x <= p.u)
    assert Pg <= Ps + gap * (1 + 1e-9) + ref.gap + 1e-12, (p.name, Pg - Ps, gap)
    if xtol is not None:
        xs = O.polish(A, y, ref.x, p.l, p.u, tau=1e-7)
        assert O.kkt_residual(A, y, xs, p.l, p.u) < 1e-9 * (1 + np.abs(A.T @ y).max())
        err = float(np.abs(x - xs).max())
        assert err <= xtol * max(1.0, float(np.abs(xs).max())), (p.name, err)
    if scr.any():
        xs = O.polish(A, y, ref.x, p.l, p.u, tau=1e-7)
        assert O.kkt_residual(A, y, xs, p.l, p.u) < 1e-8 * (1 + np.abs(A.T @ y).max())
        g = A.T @ (y - A @ xs)
        low, upp = scr == 1, scr == 2
        assert np.all(xs[low] == p.l[low]) and np.all(g[low] < 0), p.name
        assert np.all(xs[upp] == p.u[upp]) and np.all(g[upp] > 0), p.name
        assert np.all(x[low] == p.l[low]) and np.all(x[upp] == p.u[upp])


def unique_optimum(p):
    """Whether the FP64 optimum is unique: its free set has fewer than m coordinates and
    independent columns (else theta* = y - A x* is unique but x* is not)."""
    A, y = p.A.astype(np.float64), p.y.astype(np.float64)
    ref = O.solve(A, y, p.l, p.u, tol=1e-10)
    F = O.free_set(ref.x, p.l, p.u, 1e-7)
    return F.size < p.m and np.linalg.matrix_rank(A[:, F]) == F.size


def test_mixed_uneven_nondegenerate_matches_oracle(P):
    """|N| matrices with unit noise (screenable): NNLS on even k (dual translation with
    t = -1, unique optima), BVLS on [-1, 1] on odd k (dual scaling; several of these have
    P* = 0 and a free set larger than m, so x* is not unique).  The refinement returns the
    optimum to 1e-7 where it is unique and declines elsewhere."""
    probs = W.mixed_uneven(10, 1, m_lo=40, m_hi=160, abs_matrix=True, noise=1.0)
    xs, ss, gaps, its, sts, info, st = run(P, probs, tol=1e-7, refine=True)
    assert st == P.BVLS_OK and info["n_converged"] == 10
    assert info["n_translation"] == 5 and info["n_zero"] == 0
    uniq = [unique_optimum(p) for p in probs]
    assert all(uniq[0::2]) and not all(uniq)
    assert info["n_refined"] == sum(uniq), (info["n_refined"], info["refine_out_of_rounds"], info["refine_not_unique"])
    assert info["refine_not_unique"] == 10 - sum(uniq)
    assert len(set(its.tolist())) > 1
    for k, p in enumerate(probs):
        check(p, xs[k], ss[k], gaps[k], sts[k], 1e-7, xtol=1e-7 if uniq[k] else None)
    assert sum(int((s > 0).sum()) for s in ss) > 0


def test_mixed_uneven_gaussian_shape(P):
    """The Gaussian shape of the uneven workload (degenerate NNLS half: theta = 0)."""
    probs = W.mixed_uneven(8, 2, m_lo=40, m_hi=120, abs_matrix=False, noise=0.01)
    xs, ss, gaps, its, sts, info, st = run(P, probs, tol=1e-6, device=False)
    assert st == P.BVLS_OK
    assert info["n_zero"] >= 1
    for k, p in enumerate(probs):
        check(p, xs[k], ss[k], gaps[k], sts[k], 1e-6)


def test_ragged_agrees_with_single_instance_solver_and_edge_sizes(P):
    probs = W.mixed_uneven(4, 3, m_lo=30, m_hi=90, abs_matrix=True, noise=1.0)
    rng = np.random.default_rng(0)
    a = rng.standard_normal((5, 1)).astype(np.float32)          # one column, five rows
    yv = rng.standard_normal(5).astype(np.float32)
    probs.append(W.Problem("one_col", a, yv, np.array([-0.2]), np.array([0.3]), None, {}))
    xs, ss, gaps, its, sts, info, st = run(P, probs, tol=1e-9)
    assert st == P.BVLS_OK
    A1 = a.astype(np.float64)[:, 0]
    exact = np.clip(A1 @ yv.astype(np.float64) / (A1 @ A1), -0.2, 0.3)
    assert abs(xs[4][0] - exact) <= 1e-7
    dev = torch.device("cuda:0")
    for k in range(2):
        p = probs[k]
        s = P.Solver(torch.from_numpy(p.A).to(dev), p.l, p.u)
        x1, s1, i1, st1 = s.solve(torch.from_numpy(p.y).to(dev), tol=1e-9)
        s.close()
        A, y = p.A.astype(np.float64), p.y.astype(np.float64)
        assert np.linalg.norm(A @ (xs[k] - x1.cpu().numpy())) <= 2 * np.sqrt(2e-9) + 1e-9


def test_ragged_nonfinite_and_max_iter(P):
    probs = W.mixed_uneven(3, 4, m_lo=30, m_hi=60, abs_matrix=True, noise=1.0)
    xs, ss, gaps, its, sts, info, st = run(P, probs, tol=1e-14, max_iter=20)
    assert st == P.BVLS_EMAXITER and np.all(sts == P.BVLS_EMAXITER) and np.all(its == 20)
    bad = W.Problem("bad", probs[0].A, probs[0].y.copy(), probs[0].l, probs[0].u, None, {})
    bad.y[3] = np.nan
    with pytest.raises(P.BVLSError) as e:
        run(P, [probs[1], bad], tol=1e-6)
    assert e.value.status == P.BVLS_ENONFINITE


def test_autotuner_picks_tile_and_period_and_keeps_them(P):
    """screen_every = 0: the autotuner times the tile widths (8, 16, 32 columns) and the
    screening periods (5, 10, 20) and keeps its choice for batches of the same shape; the
    tuned solve reaches the same certified results as a fixed-period solve."""
    probs = W.mixed_uneven(12, 4, m_lo=40, m_hi=200, abs_matrix=True, noise=1.0)
    a = run(P, probs, tol=1e-7, screen_every=0)
    info = a[5]
    assert a[6] == P.BVLS_OK and info["n_converged"] == 12
    assert info["tile_cols"] in (8, 16, 32) and info["screen_every"] in (5, 10, 20)
    assert info["tuned"] == 1 and info["tune_ms"] > 0
    again = run(P, probs, tol=1e-7, screen_every=0)
    assert again[5]["tuned"] == 0 and again[5]["tile_cols"] == info["tile_cols"]
    assert again[5]["screen_every"] == info["screen_every"]
    fixed = run(P, probs, tol=1e-7, screen_every=10)
    assert fixed[5]["screen_every"] == 10 and fixed[5]["tile_cols"] in (8, 16, 32)
    for k, p in enumerate(probs):
        check(p, a[0][k], a[1][k], a[2][k], a[4][k], 1e-7)
        A, y = p.A.astype(np.float64), p.y.astype(np.float64)
        Pa, Pf = O.primal_objective(A, y, a[0][k]), O.primal_objective(A, y, fixed[0][k])
        assert abs(Pa - Pf) <= a[2][k] + fixed[2][k] + 1e-12


def test_full_range_uneven_batch_sampled(P):
    """The full size range of the uneven workload (m_k up to 1024, n_k up to 8 m_k) on the
    screenable |N| family: every instance certified, then the refined solutions of sampled
    NNLS instances (the largest and two others) element by element against FP64 optima certified
    by the optimality conditions.  The oracle's own solve at these sizes is too slow for a
    test, so its polish step (an FP64 least-squares solve on the free set) takes the free set
    of the GPU's result; the CPU check of the optimality conditions then certifies that the
    polished point is the optimum whatever its free set came from."""
    probs = W.mixed_uneven(24, 5, m_lo=64, m_hi=1024, abs_matrix=True, noise=1.0)
    a = run(P, probs, tol=1e-6)
    b = run(P, probs, tol=1e-6, refine=True)
    assert a[6] == P.BVLS_OK and b[6] == P.BVLS_OK
    assert max(p.m for p in probs) > 900
    # the NNLS half has unique optima; the BVLS half on [-1, 1] is mostly degenerate (P* = 0)
    assert b[5]["n_refined"] >= 12, (b[5]["n_refined"], b[5]["refine_out_of_rounds"], b[5]["refine_not_unique"])
    assert b[5]["n_refined"] + b[5]["refine_not_unique"] == 24
    big = int(np.argmax([p.m * p.n if k % 2 == 0 else 0 for k, p in enumerate(probs)]))
    for k in sorted({big, 0, 2}):
        p = probs[k]
        A, y = p.A.astype(np.float64), p.y.astype(np.float64)
        xs = O.polish(A, y, b[0][k], p.l, p.u, tau=1e-7)
        assert O.kkt_residual(A, y, xs, p.l, p.u) < 1e-9 * (1 + np.abs(A.T @ y).max()), p.name
        assert np.all(xs >= p.l - 1e-12) and np.all(xs <= p.u + 1e-12)
        err = float(np.abs(b[0][k] - xs).max())
        assert err <= 1e-7 * max(1.0, float(np.abs(xs).max())), (p.name, err)
        g = A.T @ (y - A @ xs)
        low, upp = b[1][k] == 1, b[1][k] == 2
        assert np.all(g[low] < 0) and np.all(g[upp] > 0)
