"""GPU parity of the single-instance solver against the FP64 oracle (through the C ABI).

Two kinds of comparison:
  * trajectory parity -- both sides run exactly N iterations (tol = 0) from the same point
    with the same step constant; the iterates must agree element by element;
  * result parity -- both converge to the gap tolerance; the GPU's certified gap, its
    objective, its solution and its screened set are checked against the oracle and
    against an FP64 optimum certified by the optimality conditions of Section 3.2.
"""
import json
import os

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


def _f64(p):
    return p.A.astype(np.float64), p.y.astype(np.float64).reshape(-1)


def _L(A64):
    return 1.05 * float(np.linalg.norm(A64, 2) ** 2)


def gpu_solve(P, p, t=None, x0=None, **kw):
    dev = torch.device("cuda:0")
    s = P.Solver(torch.from_numpy(np.ascontiguousarray(p.A)).to(dev), p.l, p.u, t=t)
    y = torch.from_numpy(np.ascontiguousarray(p.y.reshape(-1))).to(dev)
    x0t = None if x0 is None else torch.from_numpy(np.asarray(x0, np.float64)).to(dev)
    x, scr, info, st = s.solve(y, x0t, **kw)
    torch.cuda.synchronize()
    s.close()
    return x.cpu().numpy(), scr.cpu().numpy(), info, st


def certified_optimum(A, y, l, u, x_guess):
    """Polish x_guess in FP64 and verify the optimality conditions (Eq. (optimality2))."""
    xs = O.polish(A, y, x_guess, l, u, tau=1e-7)
    assert np.all(xs >= l - 1e-12) and np.all(xs <= u + 1e-12)
    assert O.kkt_residual(A, y, xs, l, u) < 1e-9 * (1 + np.abs(A.T @ y).max())
    return xs


def mixed_problem(seed=3, m=180, n=140):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n))
    x = rng.uniform(-1.5, 1.5, n)
    y = A @ x + 0.5 * rng.standard_normal(m)
    h = n // 2
    l = np.concatenate([np.zeros(h), np.full(n - h, -1.0)])
    u = np.concatenate([np.full(h, np.inf), np.full(n - h, 1.0)])
    return W.Problem("mixed", A.astype(np.float32), y.astype(np.float32), l, u, x, {})


def mixed_direction(p):
    """A_inf^T t = -1 by least squares (Proposition 2, case 1), computed here in numpy."""
    A64 = p.A.astype(np.float64)
    cols = ~np.isfinite(p.u)
    return np.linalg.lstsq(A64[:, cols].T, -np.ones(cols.sum()), rcond=None)[0]


CASES = {
    "nnls_abs_300x700": lambda: (W.nnls_abs_gaussian(300, 700, 0.05, 1.0, 1), None),
    "bvls_t2_200x500": lambda: (W.bvls_table2(200, 500, 2), None),
    "mixed_180x140": lambda: (lambda p: (p, mixed_direction(p)))(mixed_problem()),
    "nnls_gauss_100x200": lambda: (W.nnls_gaussian(100, 200, 0.1, 0.01, 0), None),
    "bvls_dir_224x512": lambda: (W.bvls_dirichlet_shared(224, 512, 1, 8, 0.005, 0), None),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_trajectory_matches_oracle(P, name):
    p, t = CASES[name]()
    A, y = _f64(p)
    L = _L(A)
    N = 300
    ref = O.solve(A, y, p.l, p.u, tol=0.0, screen_every=10, max_iter=N, L=L, t=t)
    x, scr, info, st = gpu_solve(P, p, t=t, tol=0.0, screen_every=10, max_iter=N, lipschitz=L)
    assert st == P.BVLS_EMAXITER and info["iters"] == N == ref.iters
    assert info["dual"] == ref.dual_mode
    scale = max(1.0, float(np.abs(ref.x).max()))
    err = float(np.abs(x - ref.x).max())
    assert err <= 1e-9 * scale, (name, err)
    # The GPU test carries wider rounding margins, so it may fix slightly fewer coordinates.
    gpu_fixed, ref_fixed = scr > 0, ref.screened > 0
    assert np.all(ref_fixed[gpu_fixed] | (np.abs(x[gpu_fixed] - ref.x[gpu_fixed]) == 0))
    assert gpu_fixed.sum() >= 0.97 * ref_fixed.sum() - 2, (gpu_fixed.sum(), ref_fixed.sum())


@pytest.mark.parametrize("make", [lambda: W.nnls_abs_gaussian(1500, 400, 0.05, 1.0, 4),   # 2 row chunks per q lane
                                  lambda: W.bvls_table2(3000, 500, 5),                    # 4
                                  lambda: W.nnls_abs_gaussian(6000, 300, 0.05, 1.0, 6)])  # 8
def test_trajectory_row_templates(P, make):
    """The persistent pass picks its q-warp template by m (1, 2, 4 or 8 float4 row chunks per
    lane, for m up to 1024, 2048, 4096 and 8192); the trajectory cases above all take the first.
    200 iterations from the same point and step constant agree with the FP64 oracle to 1e-9."""
    p = make()
    A, y = _f64(p)
    L = _L(A)
    N = 200
    ref = O.solve(A, y, p.l, p.u, tol=0.0, screen_every=10, max_iter=N, L=L)
    x, scr, info, st = gpu_solve(P, p, tol=0.0, screen_every=10, max_iter=N, lipschitz=L)
    assert st == P.BVLS_EMAXITER and info["iters"] == N == ref.iters
    assert info["single_pass"] == 2          # the persistent form ran
    scale = max(1.0, float(np.abs(ref.x).max()))
    err = float(np.abs(x - ref.x).max())
    assert err <= 1e-9 * scale, (p.m, err)


def test_mixed_trajectory_headline_template(P):
    """Mode MIXED on the headline's template (2 row chunks per q lane, half of r in the dot
    warps' registers) against the FP64 trajectory, at the reduced-precision bar of the mode
    (1e-4 relative, as test_mixed_precision_parity_nondegenerate): its forward product is
    good to about (cps + 1) u = 9 x 2^-24 relative to sum_j |a_ij x_j| per iteration, its
    correlations to float32 accuracy."""
    p = W.nnls_abs_gaussian(1800, 500, 0.05, 1.0, 8)
    A, y = _f64(p)
    L = _L(A)
    N = 200
    ref = O.solve(A, y, p.l, p.u, tol=0.0, screen_every=10, max_iter=N, L=L)
    x, scr, info, st = gpu_solve(P, p, tol=0.0, screen_every=10, max_iter=N, lipschitz=L, precision="mixed")
    assert info["iters"] == N and info["single_pass"] == 2
    scale = max(1.0, float(np.abs(ref.x).max()))
    assert float(np.abs(x - ref.x).max()) <= 1e-4 * scale


@pytest.mark.parametrize("name", ["nnls_abs_300x700", "bvls_t2_200x500", "mixed_180x140", "bvls_dir_224x512"])
def test_result_matches_oracle_and_screens_safely(P, name):
    p, t = CASES[name]()
    A, y = _f64(p)
    L = _L(A)
    # the FP64 oracle's own rounding margin floors its gap near 1e-7 on the unnormalised mixed case
    tol = 1e-6 if name.startswith("mixed") else 1e-8
    ref = O.solve(A, y, p.l, p.u, tol=tol, screen_every=10, L=L, t=t)
    assert ref.converged
    x, scr, info, st = gpu_solve(P, p, t=t, tol=tol, screen_every=10, lipschitz=L, refine=True)
    assert st == P.BVLS_OK and info["converged"] and info["gap"] < tol
    assert abs(info["iters"] - ref.iters) <= 20, (info["iters"], ref.iters)
    assert info["refined"] == 1, info
    xs = certified_optimum(A, y, p.l, p.u, ref.x)
    th = y - A @ xs
    g = A.T @ th
    low, upp = scr == 1, scr == 2
    # zero false screens: fixed coordinates sit at their bound in the certified optimum and
    # a_j^T theta* has the fixed sign (Eq. (screen_cond)).
    assert np.all(np.abs(xs[low] - p.l[low]) <= 1e-12) and np.all(g[low] < 0), name
    assert np.all(np.abs(xs[upp] - p.u[upp]) <= 1e-12) and np.all(g[upp] > 0), name
    assert np.all(x[low] == p.l[low]) and np.all(x[upp] == p.u[upp])
    Pg = O.primal_objective(A, y, x)
    Ps = O.primal_objective(A, y, xs)
    assert Ps - 1e-12 <= Pg <= Ps + tol * 1.0001 + 1e-12
    # the refined solution against the certified optimum: the FP64-checked bar
    assert float(np.abs(x - xs).max()) <= 1e-7 * max(1.0, float(np.abs(xs).max())), float(np.abs(x - xs).max())
    assert info["kkt"] <= 1e-9 * (1 + np.abs(A.T @ y).max())


@pytest.mark.parametrize("name", ["nnls_abs_300x700", "bvls_t2_200x500", "mixed_180x140", "bvls_dir_224x512"])
def test_refinement_from_a_coarse_gap(P, name):
    """Refinement started from a coarse iterate (gap 1e-3): the active-set rounds must still
    land on the certified optimum, or decline and return the solver's iterate unchanged."""
    p, t = CASES[name]()
    A, y = _f64(p)
    L = _L(A)
    ref = O.solve(A, y, p.l, p.u, tol=1e-9 if not name.startswith("mixed") else 1e-6, screen_every=10, L=L, t=t)
    xs = certified_optimum(A, y, p.l, p.u, ref.x)
    x0, s0, i0, st0 = gpu_solve(P, p, t=t, tol=1e-3, lipschitz=L)
    x1, s1, i1, st1 = gpu_solve(P, p, t=t, tol=1e-3, lipschitz=L, refine=True)
    assert i1["iters"] == i0["iters"] and np.array_equal(s0, s1)
    if i1["refined"]:
        assert float(np.abs(x1 - xs).max()) <= 1e-7 * max(1.0, float(np.abs(xs).max()))
    else:
        assert np.array_equal(x0, x1)
    assert i1["refine_rounds"] >= 1 and i1["refine_ms"] > 0


@pytest.mark.parametrize("name", ["nnls_abs_300x700", "bvls_t2_200x500", "mixed_180x140"])
def test_single_pass_matches_two_pass(P, name):
    """One streaming read per iteration gives the same iterates as the two-pass form."""
    p, t = CASES[name]()
    A, y = _f64(p)
    L = _L(A)
    a = gpu_solve(P, p, t=t, tol=0.0, max_iter=300, lipschitz=L, single_pass=True)
    b = gpu_solve(P, p, t=t, tol=0.0, max_iter=300, lipschitz=L, single_pass=False)
    assert a[2]["iters"] == b[2]["iters"] == 300
    assert float(np.abs(a[0] - b[0]).max()) <= 1e-10 * max(1.0, float(np.abs(b[0]).max()))
    assert np.array_equal(a[1] > 0, b[1] > 0) or abs(int((a[1] > 0).sum()) - int((b[1] > 0).sum())) <= 2


@pytest.mark.parametrize("name,K", [("nnls_abs_300x700", 10), ("bvls_t2_200x500", 3), ("mixed_180x140", 1)])
def test_persistent_launch_matches_per_iteration_launches(P, name, K):
    """The persistent form (K iterations per cooperative launch, grid barriers in place of
    kernel boundaries) follows the iterates of the form with two launches per iteration,
    for even, odd and unit screening periods (the slot parity crosses launches)."""
    p, t = CASES[name]()
    A, y = _f64(p)
    L = _L(A)
    a = gpu_solve(P, p, t=t, tol=0.0, max_iter=120, screen_every=K, lipschitz=L, single_pass=1)
    b = gpu_solve(P, p, t=t, tol=0.0, max_iter=120, screen_every=K, lipschitz=L, single_pass=2)
    assert a[2]["single_pass"] == 2 and b[2]["single_pass"] == 1
    assert a[2]["iters"] == b[2]["iters"] == 120
    assert float(np.abs(a[0] - b[0]).max()) <= 1e-10 * max(1.0, float(np.abs(b[0]).max()))
    assert abs(int((a[1] > 0).sum()) - int((b[1] > 0).sum())) <= 2
    c = gpu_solve(P, p, t=t, tol=0.0, max_iter=120, screen_every=K, lipschitz=L, profile=True)
    assert c[2]["tr_launches"] == 120 // K and c[2]["tr_ms"] > 0 and c[2]["fwd_launches"] == 0
    assert float(np.abs(c[0] - a[0]).max()) <= 1e-10 * max(1.0, float(np.abs(b[0]).max()))
    # every kernel launched directly from the host (no graph): the same iterates bit for bit
    d = gpu_solve(P, p, t=t, tol=0.0, max_iter=120, screen_every=K, lipschitz=L, profile=2)
    assert d[2]["iters"] == 120 and np.array_equal(d[0], a[0]) and np.array_equal(d[1], a[1])


def test_screened_and_unscreened_follow_the_same_iterates(P):
    p = W.nnls_abs_gaussian(400, 1500, 0.05, 1.0, 4)
    A, y = _f64(p)
    L = _L(A)
    a = gpu_solve(P, p, tol=1e-8, lipschitz=L)
    b = gpu_solve(P, p, tol=1e-8, lipschitz=L, screening=False)
    assert a[2]["converged"] and b[2]["converged"]
    assert abs(a[2]["iters"] - b[2]["iters"]) <= 10
    assert (a[1] > 0).sum() > 0.5 * p.n and (b[1] > 0).sum() == 0
    assert a[2]["sum_preserved"] < 0.8 * b[2]["sum_preserved"]
    assert float(np.abs(a[0] - b[0]).max()) < 1e-6


def test_fp32_precision_mode(P):
    p = W.bvls_table2(200, 500, 5)
    A, y = _f64(p)
    L = _L(A)
    ref = O.solve(A, y, p.l, p.u, tol=1e-9, screen_every=10, L=L)
    xs = certified_optimum(A, y, p.l, p.u, ref.x)
    # float32 accumulation: the rigorous rounding margin puts the reachable gap near 1e-3 here
    x, scr, info, st = gpu_solve(P, p, tol=3e-3, lipschitz=L, precision="fp32")
    assert info["converged"]
    g = A.T @ (y - A @ xs)
    assert np.all(g[scr == 1] < 0) and np.all(g[scr == 2] > 0)
    assert O.primal_objective(A, y, x) <= O.primal_objective(A, y, xs) + 3e-3


def test_mixed_precision_mode(P):
    """Float32 correlations with the double-float forward product.  With the zero dual point
    (no interior direction) the certificate 1/2 (||r|| + E_r)^2 needs only the residual, so
    the gap reaches the fp32x2 tolerance; with a scaled dual point the screens stay safe
    under the float32 margins of the correlations."""
    p = W.nnls_gaussian(400, 1200, 0.05, 0.01, 1)
    A, y = _f64(p)
    assert O.choose_translation(A, p.u) is None
    for single_pass in (True, False):
        x, scr, info, st = gpu_solve(P, p, tol=1e-7, precision="mixed", single_pass=single_pass)
        assert st == P.BVLS_OK and info["dual"] == "zero" and info["gap"] < 1e-7
        assert np.all(x >= 0) and O.primal_objective(A, y, x) <= info["gap"] * (1 + 1e-9)
    q = W.bvls_table2(200, 500, 5)
    A, y = _f64(q)
    L = _L(A)
    ref = O.solve(A, y, q.l, q.u, tol=1e-9, screen_every=10, L=L)
    xs = certified_optimum(A, y, q.l, q.u, ref.x)
    x, scr, info, st = gpu_solve(P, q, tol=3e-3, lipschitz=L, precision="mixed")
    assert info["converged"] and info["gap"] < 3e-3
    g = A.T @ (y - A @ xs)
    assert np.all(g[scr == 1] < 0) and np.all(g[scr == 2] > 0)
    assert np.all(np.abs(xs[scr == 1] - q.l[scr == 1]) <= 1e-12)
    assert np.all(np.abs(xs[scr == 2] - q.u[scr == 2]) <= 1e-12)
    Pg, Ps = O.primal_objective(A, y, x), O.primal_objective(A, y, xs)
    assert Ps - 1e-12 <= Pg <= Ps + info["gap"] * (1 + 1e-9) + 1e-12


@pytest.mark.parametrize("name", ["nnls_abs_300x700", "bvls_t2_200x500"])
def test_mixed_precision_parity_nondegenerate(P, name):
    """The reduced-precision bar of the mixed mode: with a unique optimum the iterates agree
    with the certified FP64 optimum to 1e-4 relative, nothing is screened off its bound, and
    the reported gap bounds P(x) - P*.  (With theta != 0 the float32 correlations enter the
    certificate through the margin eta, so the mode certifies only coarse gaps here; its
    tight certificate is the theta = 0 one.)"""
    p, t = CASES[name]()
    A, y = _f64(p)
    L = _L(A)
    ref = O.solve(A, y, p.l, p.u, tol=1e-10, screen_every=10, L=L, t=t)
    xs = certified_optimum(A, y, p.l, p.u, ref.x)
    x, scr, info, st = gpu_solve(P, p, t=t, tol=0.0, screen_every=10, max_iter=4000, lipschitz=L,
                                 precision="mixed")
    assert info["iters"] == 4000
    assert float(np.abs(x - xs).max()) <= 1e-4 * max(1.0, float(np.abs(xs).max()))
    g = A.T @ (y - A @ xs)
    assert np.all(np.abs(xs[scr == 1] - p.l[scr == 1]) <= 1e-12) and np.all(g[scr == 1] < 0)
    assert np.all(np.abs(xs[scr == 2] - p.u[scr == 2]) <= 1e-12) and np.all(g[scr == 2] > 0)
    Pg, Ps = O.primal_objective(A, y, x), O.primal_objective(A, y, xs)
    assert Ps - 1e-12 <= Pg <= Ps + info["gap"] * (1 + 1e-9) + 1e-12


def test_single_column_closed_form(P):
    rng = np.random.default_rng(0)
    for lo, hi in [(0.0, np.inf), (-0.3, 0.4), (0.0, 1.0)]:
        a = rng.standard_normal((37, 1))
        yv = rng.standard_normal(37) * 2
        p = W.Problem("one", a.astype(np.float32), yv.astype(np.float32), np.array([lo]), np.array([hi]), None)
        A, y = _f64(p)
        exact = np.clip(A[:, 0] @ y / (A[:, 0] @ A[:, 0]), lo, hi)
        x, scr, info, st = gpu_solve(P, p, tol=1e-12, screen_every=1, max_iter=2000)
        assert abs(x[0] - exact) <= 1e-7 * max(1.0, abs(exact)), (x, exact)


def test_single_row_and_odd_screen_period(P):
    p = W.bvls_gaussian_box(1, 9, 0.5, 0)
    A, y = _f64(p)
    xb, Pb = O.brute_force(A, y, p.l, p.u)
    x, scr, info, st = gpu_solve(P, p, tol=1e-12, screen_every=3, max_iter=30000)
    assert info["converged"] and abs(O.primal_objective(A, y, x) - Pb) < 1e-9


def test_zero_column_is_never_screened(P):
    p = W.nnls_abs_gaussian(64, 90, 0.1, 1.0, 6)
    A = p.A.copy()
    A[:, 5] = 0.0
    p = W.Problem("zc", A, p.y, p.l, p.u, None)
    x, scr, info, st = gpu_solve(P, p, tol=1e-8)
    assert info["converged"] and scr[5] == 0 and x[5] == 0.0


def test_warm_start_and_status_codes(P):
    p = W.bvls_table2(120, 260, 8)
    A, y = _f64(p)
    ref = O.solve(A, y, p.l, p.u, tol=1e-10, screen_every=10)
    x, scr, info, st = gpu_solve(P, p, x0=ref.x, tol=1e-8)
    assert st == P.BVLS_OK and info["iters"] <= 20
    x, scr, info, st = gpu_solve(P, p, tol=1e-30, max_iter=25)
    assert st == P.BVLS_EMAXITER and info["iters"] == 30 and not info["converged"]
    bad = W.Problem("nan", p.A, p.y.copy(), p.l, p.u, None)
    bad.y[3] = np.nan
    x, scr, info, st = gpu_solve(P, bad, check=False)
    assert st == P.BVLS_ENONFINITE
    with pytest.raises(P.BVLSError):
        P.Solver(torch.zeros(4, 3, device="cuda"), l=[0, 0, 1], u=[1, 1, 0])


def test_degenerate_single_instance_full_size(P):
    """The 2000 x 10000 Gaussian NNLS workload: no interior dual direction, nothing screens."""
    p = W.nnls_gaussian(2000, 10000, 0.05, 0.01, 0)
    A, y = _f64(p)
    assert O.choose_translation(A, p.u) is None
    x, scr, info, st = gpu_solve(P, p, tol=1e-6)
    assert st == P.BVLS_OK and info["dual"] == "zero" and (scr > 0).sum() == 0
    assert np.all(x >= 0)
    Pval = O.primal_objective(A, y, x)
    assert Pval <= info["gap"] * (1 + 1e-9) and info["gap"] < 1e-6      # Gap(x, 0) = P(x)
    b = gpu_solve(P, p, tol=1e-6, screening=False)
    assert b[2]["iters"] == info["iters"]


def test_degenerate_refinement_never_worsens(P):
    """Where the optimum is not unique (Gaussian n >> m, theta* = 0) the free set may exceed
    m: the refinement either declines and returns the solver's iterate, or returns a point
    that satisfies the optimality conditions."""
    p = W.nnls_gaussian(100, 200, 0.1, 0.01, 0)
    A, y = _f64(p)
    a = gpu_solve(P, p, tol=1e-9)
    b = gpu_solve(P, p, tol=1e-9, refine=True)
    if b[2]["refined"]:
        assert np.all(b[0] >= 0)
        assert O.kkt_residual(A, y, b[0], p.l, p.u) <= 1e-8 * (1 + np.abs(A.T @ y).max())
        assert O.primal_objective(A, y, b[0]) <= O.primal_objective(A, y, a[0]) + 1e-12
    else:
        assert np.array_equal(a[0], b[0])


def test_screenable_single_instance_full_size(P):
    """2000 x 10000 |N(0,1)| NNLS (Table 1 family): certified gap and safe screens at full size,
    and the refined solution element by element against an FP64 optimum certified by the
    optimality conditions.  The FP64 oracle's own solve at this size takes tens of minutes, so
    its polish step (an FP64 least-squares solve on the free set) takes the free set of the
    GPU's result; the CPU check of the optimality conditions then certifies that the polished
    point is the optimum whatever its free set came from."""
    p = W.nnls_abs_gaussian(2000, 10000, 0.05, 1.0, 0)
    A, y = _f64(p)
    x0, scr0, info0, st0 = gpu_solve(P, p, tol=1e-6)
    x, scr, info, st = gpu_solve(P, p, tol=1e-6, refine=True)
    assert info["refined"] == 1 and info["iters"] == info0["iters"]
    xs = O.polish(A, y, x, p.l, p.u, tau=1e-7)
    assert np.all(xs >= 0)
    assert O.kkt_residual(A, y, xs, p.l, p.u) < 1e-9 * (1 + np.abs(A.T @ y).max())
    assert float(np.abs(x - xs).max()) <= 1e-7 * max(1.0, float(np.abs(xs).max()))
    g_s = A.T @ (y - A @ xs)
    assert np.all(g_s[scr == 1] < 0) and np.all(xs[scr == 1] == 0)
    # the FP64 optimum of the oracle's own run (tests/golden/make_bench_optima.py: oracle solve,
    # polish, optimality conditions), independent of the GPU's free set
    rec = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "bench_optima.json")))
    rec = rec["nnls_abs_gaussian_2000x10000"]["single"]
    assert rec["unique"]
    x_star = np.zeros(p.n)
    x_star[np.asarray(rec["x_star_idx"], dtype=int)] = rec["x_star_val"]
    scale = max(1.0, float(np.abs(x_star).max()))
    assert float(np.abs(x - x_star).max()) <= 1e-7 * scale
    assert float(np.abs(x0 - x_star).max()) <= 1e-6 * scale
    assert O.primal_objective(A, y, x0) <= rec["P_star"] + info0["gap"] * (1 + 1e-9) + 1e-9
    assert st == P.BVLS_OK and info["dual"] == "translation"
    assert np.all(x >= 0) and np.all(x[scr == 1] == 0)
    t = -np.ones(p.m)
    cols = ~np.isfinite(p.u)
    r = y - A @ x
    th, eps = O.translate(A, r, t, cols)
    gap = O.duality_gap(A, y, x, th, p.l, p.u)
    assert gap <= 1e-6 * 1.01 + 1e-9, gap
    g = A.T @ th
    rad = O.safe_radius(gap)
    # at the final dual point every fixed column is still strictly on its side of 0
    assert np.all(g[scr == 1] < 0)
    assert (scr > 0).sum() > 0.5 * p.n
    assert np.sum(g[scr == 1] >= -rad * np.linalg.norm(A[:, scr == 1], axis=0)) < 0.05 * (scr > 0).sum()


@pytest.mark.parametrize("name", ["nnls_abs_300x700", "bvls_t2_200x500"])
def test_fixed_dual_point_matches_oracle(P, name):
    """The oracle-dual-point option: the same iterates as the oracle run with the same fixed
    dual point, safe screening, and earlier fixing than with Theta(x_k)."""
    p, t = CASES[name]()
    A, y = _f64(p)
    L = _L(A)
    ref = O.solve(A, y, p.l, p.u, tol=1e-10, L=L)
    xs = certified_optimum(A, y, p.l, p.u, ref.x)
    th = y - A @ xs
    N = 300
    o = O.solve(A, y, p.l, p.u, tol=0.0, max_iter=N, L=L, dual_point=th)
    x, scr, info, st = gpu_solve(P, p, tol=0.0, max_iter=N, lipschitz=L, dual_point=th)
    scale = max(1.0, float(np.abs(o.x).max()))
    assert float(np.abs(x - o.x).max()) <= 1e-9 * scale
    g = A.T @ th
    assert np.all(g[scr == 1] < 0) and np.all(xs[scr == 1] == p.l[scr == 1])
    assert np.all(g[scr == 2] > 0) and np.all(xs[scr == 2] == p.u[scr == 2])
    x2, scr2, info2, st2 = gpu_solve(P, p, tol=1e-8, lipschitz=L, dual_point=th)
    x3, scr3, info3, st3 = gpu_solve(P, p, tol=1e-8, lipschitz=L)
    assert info2["converged"] and info2["iters"] <= info3["iters"]
    assert info2["sum_preserved"] <= info3["sum_preserved"]
    assert O.primal_objective(A, y, x2) - O.primal_objective(A, y, xs) <= info2["gap"] * (1 + 1e-9) + 1e-12


@pytest.mark.parametrize("name", ["bvls_t2_200x500", "bvls_dir_224x512"])
def test_chambolle_pock_matches_oracle(P, name):
    """Primal-dual solver: the same iterates as the oracle's Chambolle-Pock over 300
    iterations, then the certified optimum with safe screening on its own dual iterate."""
    p, t = CASES[name]()
    A, y = _f64(p)
    L = _L(A)
    N = 300
    o = O.solve_cp(A, y, p.l, p.u, tol=0.0, max_iter=N, L=L)
    x, scr, info, st = gpu_solve(P, p, tol=0.0, max_iter=N, lipschitz=L, algorithm="cp")
    assert info["iters"] == N == o.iters
    assert float(np.abs(x - o.x).max()) <= 1e-9 * max(1.0, float(np.abs(o.x).max()))
    ref = O.solve_cp(A, y, p.l, p.u, tol=1e-8, L=L)
    x, scr, info, st = gpu_solve(P, p, tol=1e-8, lipschitz=L, algorithm="cp")
    assert st == P.BVLS_OK and info["gap"] < 1e-8 and abs(info["iters"] - ref.iters) <= 20
    xs = certified_optimum(A, y, p.l, p.u, ref.x)
    g = A.T @ (y - A @ xs)
    assert np.all(xs[scr == 1] == p.l[scr == 1]) and np.all(g[scr == 1] < 0)
    assert np.all(xs[scr == 2] == p.u[scr == 2]) and np.all(g[scr == 2] > 0)
    assert (scr > 0).sum() > 0
    Pg, Ps = O.primal_objective(A, y, x), O.primal_objective(A, y, xs)
    assert Ps - 1e-12 <= Pg <= Ps + info["gap"] * (1 + 1e-9) + 1e-12
    # Without screening the iterates are the same, but the gap keeps the terms of the
    # coordinates the screened run has fixed; with theta = -z those can stay positive, so the
    # screened run (which certifies the reduced problem, same optimum) may stop earlier.
    u = gpu_solve(P, p, tol=1e-8, lipschitz=L, algorithm="cp", screening=False)
    assert u[2]["iters"] >= info["iters"] and u[2]["gap"] < 1e-8
    assert abs(O.primal_objective(A, y, u[0]) - Pg) <= info["gap"] + u[2]["gap"]


def test_chambolle_pock_rejects_nnls(P):
    p = W.nnls_abs_gaussian(50, 80, 0.1, 1.0, 1)
    x, scr, info, st = gpu_solve(P, p, tol=1e-6, algorithm="cp", check=False)
    assert st == P.BVLS_ENOTSUP
