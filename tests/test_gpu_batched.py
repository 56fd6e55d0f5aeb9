"""GPU parity of the batched solver (one shared A, many right-hand sides) against the FP64 oracle.

Each instance of a batch is compared with the oracle's own solve of that instance:
  * the GPU's gap bound holds: P(x_gpu) - P(x*) <= gap_gpu < tol, with x* an FP64 optimum
    certified by the optimality conditions of Section 3.2;
  * zero false screens: every coordinate the GPU fixed sits at that bound in x*, and
    a_j^T theta* has the sign Eq. (screen_cond) requires;
  * the solution agrees with x* to 1e-4 relative (the bar of the reduced-precision forms:
    the non-evaluation steps use bf16 tensor-core products), and after the free-set
    refinement (opts.refine) to 1e-7 relative.
"""
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


def batched(P, p, Y=None, X0=None, **kw):
    dev = torch.device("cuda:0")
    s = P.Solver(torch.from_numpy(np.ascontiguousarray(p.A)).to(dev), p.l, p.u)
    Yt = torch.from_numpy(np.ascontiguousarray(p.y if Y is None else Y)).to(dev)
    X0t = None if X0 is None else torch.from_numpy(np.asarray(X0, np.float64)).to(dev)
    X, S, gaps, its, sts, info, st = s.solve_batched(Yt, X0t, **kw)
    torch.cuda.synchronize()
    out = (X.cpu().numpy(), S.cpu().numpy(), gaps.cpu().numpy(), its.cpu().numpy(), sts.cpu().numpy(), info, st)
    s.close()
    return out


def certified_optimum(A, y, l, u, tol):
    ref = O.solve(A, y, l, u, tol=tol, screen_every=10)
    xs = O.polish(A, y, ref.x, l, u, tau=1e-7)
    assert np.all(xs >= l - 1e-12) and np.all(xs <= u + 1e-12)
    assert O.kkt_residual(A, y, xs, l, u) < 1e-9 * (1 + np.abs(A.T @ y).max())
    return xs


def check_instance(A, y, l, u, x, scr, gap, status, xs, tol, name, xtol=1e-4):
    assert status == 0 and gap < tol, (name, status, gap)
    assert np.all(x >= l) and np.all(x <= u), name
    Pg, Ps = O.primal_objective(A, y, x), O.primal_objective(A, y, xs)
    assert Ps - 1e-12 <= Pg <= Ps + gap * (1 + 1e-9) + 1e-12, (name, Pg - Ps, gap)
    g = A.T @ (y - A @ xs)
    low, upp = scr == 1, scr == 2
    assert np.all(np.abs(xs[low] - l[low]) <= 1e-12) and np.all(g[low] < 0), name
    assert np.all(np.abs(xs[upp] - u[upp]) <= 1e-12) and np.all(g[upp] > 0), name
    assert np.all(x[low] == l[low]) and np.all(x[upp] == u[upp]), name
    err = float(np.abs(x - xs).max())
    assert err <= xtol * max(1.0, float(np.abs(xs).max())), (name, err)


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-6), ("fp32x2", 1e-8)])
def test_dirichlet_shared_matches_oracle(P, precision, tol):
    """The shape of the batched BVLS workload: A 224 x 512 U[0,1] unit columns, box [0,1]."""
    p = W.bvls_dirichlet_shared(224, 512, 12, 8, 0.005, 1)
    A = p.A.astype(np.float64)
    X, S, gaps, its, sts, info, st = batched(P, p, tol=tol, precision=precision)
    assert st == P.BVLS_OK and info["n_converged"] == 12
    assert info["dual"] == "scaling"
    XR, SR, gR, iR, sR, infoR, stR = batched(P, p, tol=tol, precision=precision, refine=True)
    assert infoR["n_refined"] == 12 and np.array_equal(iR, its) and np.array_equal(SR, S)
    for b in range(12):
        y = p.y[b].astype(np.float64)
        xs = certified_optimum(A, y, p.l, p.u, 1e-10)
        check_instance(A, y, p.l, p.u, X[b], S[b], gaps[b], sts[b], xs, tol, f"inst{b}")
        check_instance(A, y, p.l, p.u, XR[b], SR[b], gR[b], sR[b], xs, tol, f"inst{b}", xtol=1e-7)
    assert (S > 0).sum() > 0.5 * S.size   # most coordinates are fixed at 0 by the end


def test_nnls_translation_ragged_tiles(P):
    """NNLS (dual translation, Eq. (BVLR_dual_up2)) with n = 300 (three coordinate tiles,
    the last ragged) and B = 150 instances (two instance tiles, the last ragged)."""
    p = W.nnls_shared(96, 300, 150, 0.06, 1.0, 2)
    A = p.A.astype(np.float64)
    X, S, gaps, its, sts, info, st = batched(P, p, tol=1e-7, precision="fp32x2", refine=True)
    assert st == P.BVLS_OK and info["dual"] == "translation"
    assert len(set(its.tolist())) > 1          # uneven convergence: instances retire apart
    assert info["n_refined"] == 150, info
    for b in list(range(0, 150, 13)) + [149]:
        y = p.y[b].astype(np.float64)
        xs = certified_optimum(A, y, p.l, p.u, 1e-9)
        check_instance(A, y, p.l, p.u, X[b], S[b], gaps[b], sts[b], xs, 1e-7, f"inst{b}", xtol=1e-7)


def test_gaussian_box_both_bounds(P):
    """BVLS with both bounds active (N(0,1) data, box [-0.05, 0.05]): fixes at l and at u."""
    p = W.bvls_box_shared(80, 150, 40, 0.05, 3)
    A = p.A.astype(np.float64)
    X, S, gaps, its, sts, info, st = batched(P, p, tol=1e-8, precision="fp32x2", refine=True)
    assert st == P.BVLS_OK
    assert (S == 1).sum() > 0 and (S == 2).sum() > 0
    assert info["n_refined"] == 40, info
    for b in range(0, 40, 5):
        y = p.y[b].astype(np.float64)
        xs = certified_optimum(A, y, p.l, p.u, 1e-11)
        check_instance(A, y, p.l, p.u, X[b], S[b], gaps[b], sts[b], xs, 1e-8, f"inst{b}", xtol=1e-7)


def test_screening_off_reaches_the_same_optimum(P):
    p = W.bvls_dirichlet_shared(128, 256, 20, 6, 0.005, 4)
    a = batched(P, p, tol=1e-7, precision="fp32x2")
    b = batched(P, p, tol=1e-7, precision="fp32x2", screening=False)
    assert a[6] == P.BVLS_OK and b[6] == P.BVLS_OK
    assert (a[1] > 0).sum() > 0 and (b[1] > 0).sum() == 0
    assert a[5]["sum_preserved"] < b[5]["sum_preserved"]
    A = p.A.astype(np.float64)
    for i in range(20):
        y = p.y[i].astype(np.float64)
        Pa, Pb = O.primal_objective(A, y, a[0][i]), O.primal_objective(A, y, b[0][i])
        assert abs(Pa - Pb) <= a[2][i] + b[2][i]


def test_batched_agrees_with_single_instance_solver(P):
    p = W.bvls_dirichlet_shared(224, 512, 4, 8, 0.005, 5)
    X, S, gaps, its, sts, info, st = batched(P, p, tol=1e-8, precision="fp32x2")
    dev = torch.device("cuda:0")
    s = P.Solver(torch.from_numpy(np.ascontiguousarray(p.A)).to(dev), p.l, p.u)
    A = p.A.astype(np.float64)
    for b in range(4):
        x1, s1, i1, st1 = s.solve(torch.from_numpy(p.y[b]).to(dev), tol=1e-8)
        x1 = x1.cpu().numpy()
        y = p.y[b].astype(np.float64)
        # both certify gap < 1e-8, so both residuals lie within sqrt(2 * 1e-8) of theta*
        r_b, r_1 = y - A @ X[b], y - A @ x1
        assert np.linalg.norm(r_b - r_1) <= 2 * np.sqrt(2e-8) + 1e-9
    s.close()


def test_max_iter_warm_start_zero_rhs_and_single_instance(P):
    p = W.bvls_dirichlet_shared(64, 160, 6, 5, 0.005, 6)
    A = p.A.astype(np.float64)
    # max_iter: every instance stops at the evaluation k = max_iter with a valid bound
    X, S, gaps, its, sts, info, st = batched(P, p, tol=1e-12, max_iter=20)
    assert st == P.BVLS_EMAXITER and np.all(sts == P.BVLS_EMAXITER) and np.all(its == 20)
    for b in range(6):
        y = p.y[b].astype(np.float64)
        xs = certified_optimum(A, y, p.l, p.u, 1e-11)
        assert O.primal_objective(A, y, X[b]) - O.primal_objective(A, y, xs) <= gaps[b] * (1 + 1e-9) + 1e-12
    # warm start at the optimum: the first evaluation already certifies it
    XS = np.stack([certified_optimum(A, p.y[b].astype(np.float64), p.l, p.u, 1e-11) for b in range(6)])
    X, S, gaps, its, sts, info, st = batched(P, p, X0=XS, tol=1e-6)
    assert st == P.BVLS_OK and np.all(its <= 10)
    # y = 0: x = 0 is optimal with gap 0 at k = 0
    Y = p.y.copy()
    Y[2] = 0.0
    X, S, gaps, its, sts, info, st = batched(P, p, Y=Y, tol=1e-9)
    assert its[2] == 0 and np.all(X[2] == 0.0) and gaps[2] < 1e-12
    # B = 1
    X, S, gaps, its, sts, info, st = batched(P, p, Y=p.y[:1], tol=1e-8, precision="fp32x2")
    xs = certified_optimum(A, p.y[0].astype(np.float64), p.l, p.u, 1e-11)
    check_instance(A, p.y[0].astype(np.float64), p.l, p.u, X[0], S[0], gaps[0], sts[0], xs, 1e-8, "B1")


def test_repeat_calls_are_identical_and_nonfinite_is_rejected(P):
    p = W.bvls_dirichlet_shared(64, 160, 9, 5, 0.005, 7)
    dev = torch.device("cuda:0")
    s = P.Solver(torch.from_numpy(np.ascontiguousarray(p.A)).to(dev), p.l, p.u)
    Y = torch.from_numpy(p.y).to(dev)
    a = s.solve_batched(Y, tol=1e-8)
    b = s.solve_batched(Y, tol=1e-8)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]) and torch.equal(a[3], b[3])
    Yb = Y.clone()
    Yb[3, 7] = float("nan")
    with pytest.raises(P.BVLSError) as e:
        s.solve_batched(Yb, tol=1e-8)
    assert e.value.status == P.BVLS_ENONFINITE
    c = s.solve_batched(Y, tol=1e-8)   # the handle stays usable
    assert torch.equal(a[0], c[0])
    s.close()


def test_full_size_batch_refined_against_certified_optima(P):
    """The full 4096-instance batch of the 224 x 512 BVLS workload with refinement: sampled
    instances element by element against FP64 optima certified by the optimality conditions."""
    p = W.bvls_dirichlet_shared(224, 512, 4096, 8, 0.005, 0)
    A = p.A.astype(np.float64)
    X, S, gaps, its, sts, info, st = batched(P, p, tol=1e-6, precision="fp32x2", refine=True)
    assert st == P.BVLS_OK and info["n_converged"] == 4096
    assert info["n_refined"] >= 4090, info
    for b in [0, 1, 777, 2048, 4095]:
        y = p.y[b].astype(np.float64)
        xs = certified_optimum(A, y, p.l, p.u, 1e-10)
        check_instance(A, y, p.l, p.u, X[b], S[b], gaps[b], sts[b], xs, 1e-6, f"inst{b}", xtol=1e-7)


@pytest.mark.parametrize("make,K", [
    (lambda: W.bvls_dirichlet_shared(224, 512, 300, 8, 0.005, 2), 10),   # 4 coordinate tiles, ragged last instance tile
    (lambda: W.bvls_dirichlet_shared(224, 512, 4096, 8, 0.005, 0), 10),  # the benchmark's batch
    (lambda: W.bvls_box_shared(96, 384, 130, 0.5, 3), 3),                # 3 tiles, runs of 2 steps
    (lambda: W.nnls_shared(120, 200, 129, 0.05, 1.0, 4), 10),            # 2 tiles, translation dual point
    (lambda: W.bvls_box_shared(60, 100, 40, 1.0, 5), 2),                 # 1 tile, runs of 1 step
])
def test_persistent_steps_match_per_step_launches(P, make, K):
    """single_pass 1 runs the K - 1 tensor-core steps between two evaluations as one launch of
    clusters that keep x, g and d on chip; single_pass 0 launches every step.  Both take the
    same operations in the same order, so every output agrees bit for bit."""
    p = make()
    runs = [batched(P, p, tol=1e-7, screen_every=K, max_iter=20000, single_pass=sp) for sp in (1, 0)]
    (X1, S1, g1, i1, s1, info1, st1), (X0, S0, g0, i0, s0, info0, st0) = runs
    assert info1["steps_persistent"] == 1 and info0["steps_persistent"] == 0
    assert st1 == st0 and st1 in (P.BVLS_OK, P.BVLS_EMAXITER)
    assert info1["n_converged"] == info0["n_converged"] > 0
    assert np.array_equal(i1, i0) and np.array_equal(s1, s0)
    assert np.array_equal(S1, S0)
    assert np.array_equal(g1, g0)
    assert np.array_equal(X1, X0)
    assert info1["sum_step"] == info0["sum_step"]
    # one launch per run of K - 1 steps instead of K - 1 launches
    assert info1["kernel_launches"] < info0["kernel_launches"] or K == 2


def test_wide_batch_takes_per_step_launches(P):
    """npad = 640 needs five coordinate tiles, more than the persistent step's clusters hold:
    the solve falls back to one step launch per iteration and still matches the oracle."""
    p = W.bvls_dirichlet_shared(150, 600, 6, 8, 0.005, 7)
    A = p.A.astype(np.float64)
    X, S, gaps, its, sts, info, st = batched(P, p, tol=1e-7, precision="fp32x2")
    assert st == P.BVLS_OK and info["n_converged"] == 6
    assert info["steps_persistent"] == 0
    for b in range(6):
        y = p.y[b].astype(np.float64)
        xs = certified_optimum(A, y, p.l, p.u, 1e-10)
        check_instance(A, y, p.l, p.u, X[b], S[b], gaps[b], sts[b], xs, 1e-7, f"inst{b}")


@pytest.mark.parametrize("kw", [dict(profile=True), dict(screening=False), dict(restart=False), dict(refine=True),
                                dict(warm=True), dict(precision="fp32")])
def test_persistent_steps_match_under_options(P, kw):
    """The persistent and per-step forms agree bit for bit under the other options too: the
    event-timed chunk graph (profile), no screening, no restart, the refinement that follows
    the solve, a warm start and float32 evaluations."""
    kw = dict(kw)
    p = W.bvls_box_shared(120, 320, 140, 0.5, 9)
    X0 = None
    if kw.pop("warm", False):
        X0 = np.random.default_rng(9).uniform(-0.5, 0.5, (140, 320))
    runs = [batched(P, p, X0=X0, tol=1e-7, screen_every=10, max_iter=20000, single_pass=sp, **kw) for sp in (1, 0)]
    (X1, S1, g1, i1, s1, info1, st1), (X0r, S0, g0, i0, s0, info0, st0) = runs
    assert info1["steps_persistent"] == 1 and info0["steps_persistent"] == 0
    assert st1 == st0 and info1["n_converged"] == info0["n_converged"] > 0
    assert np.array_equal(i1, i0) and np.array_equal(s1, s0) and np.array_equal(S1, S0)
    assert np.array_equal(g1, g0) and np.array_equal(X1, X0r)
    if kw.get("profile"):
        # every step is timed (a persistent launch as a whole, its later steps as empty intervals)
        assert info1["step_launches"] == info0["step_launches"] > 0
        assert info1["step_ms"] > 0 and info0["step_ms"] > 0


@pytest.mark.parametrize("single_pass", [1, 0])
def test_tensor_core_iterates_follow_the_bf16_gram_oracle(P, single_pass):
    """Iterate-level parity of the tensor-core path.  Between two evaluations the GPU forms the
    correlations by the Gram recurrence g_k = g_{k-1} - bf16(A^T A) bf16(x_k - x_{k-1})
    (float32 accumulation); oracle.gram_fista_batch runs the same iteration in float64 with
    the same two bf16 roundings.  Exact agreement is out of reach: a change of a few float32
    units in x_k - x_{k-1} moves some entries across a bf16 rounding boundary (2^-8 relative),
    so float32 arithmetic alone puts a float64 copy of the iteration about 1.5e-5 away from
    the oracle after 30 iterations, against about 1e-4 between the bf16 iteration and the
    exact-gradient FISTA.  After 30 iterations (evaluations at 0, 10, 20, 30; no screening,
    no restart, the same L) the GPU must sit within 1e-4 of the bf16 oracle and at most half
    as far from it as from the exact-gradient FISTA: the deviation the bf16 operands cause is
    the oracle's, what is left is float32 arithmetic."""
    p = W.bvls_dirichlet_shared(224, 512, 16, 8, 0.005, 3)
    A, Y = p.A.astype(np.float64), p.y.astype(np.float64)
    L = 1.05 * float(np.linalg.norm(A, 2) ** 2)
    N = 30
    X, S, gaps, its, sts, info, st = batched(P, p, tol=0.0, screen_every=10, max_iter=N, screening=False,
                                             restart=False, lipschitz=L, precision="fp32",
                                             single_pass=single_pass, check=False)
    assert np.all(its == N) and not np.any(S)
    Xb = O.gram_fista_batch(A, Y, p.l, p.u, L, screen_every=10, max_iter=N, bf16=True)
    Xe = O.gram_fista_batch(A, Y, p.l, p.u, L, screen_every=10, max_iter=N, bf16=False)
    scale = max(1.0, float(np.abs(Xb).max()))
    err_b = float(np.abs(X - Xb).max())
    err_e = float(np.abs(X - Xe).max())
    assert err_b <= 1e-4 * scale, (err_b, err_e)
    assert err_b <= 0.5 * err_e, (err_b, err_e)
