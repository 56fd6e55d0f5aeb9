"""Pins of the FP64 oracle against mathematics that does not come from the oracle itself.

Each check is chosen so that a plausible slip in the oracle (a dropped term, a sign, a
transposed operand, a wrong radius) fails at least one of them; ``test_mutations`` plants
such slips in the oracle and confirms that the pins catch them.
"""
import json
import os

import numpy as np
import pytest
import scipy.optimize as so

import oracle as O
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _f64(p):
    return p.A.astype(np.float64), p.y.astype(np.float64).reshape(-1)


def _sigma(g, l, u):
    """sup_{x in [l,u]} x g, written out per coordinate (Appendix B)."""
    out = np.empty_like(g)
    for j in range(g.size):
        if g[j] >= 0:
            out[j] = 0.0 if g[j] == 0 else (u[j] * g[j] if np.isfinite(u[j]) else np.inf)
        else:
            out[j] = l[j] * g[j]
    return out


# ----------------------------------------------------------------------------- pin helpers
def check_closed_form_1col(solve_kw):
    rng = np.random.default_rng(11)
    for _ in range(6):
        m = int(rng.integers(2, 9))
        a = rng.standard_normal((m, 1))
        y = rng.standard_normal(m) * 3
        lo = float(rng.uniform(-1, 0))
        hi = float(rng.uniform(0, 1)) if rng.random() < 0.7 else np.inf
        exact = np.clip((a[:, 0] @ y) / (a[:, 0] @ a[:, 0]), lo, hi)
        r = O.solve(a, y, [lo], [hi], tol=1e-12, screen_every=1, max_iter=5000, **solve_kw)
        assert abs(r.x[0] - exact) < 1e-9 * (1 + abs(exact)), (r.x, exact)


def check_golden():
    with open(os.path.join(GOLDEN, "hand_derived.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        A = np.array(c["A"], float)
        y = np.array(c["y"], float)
        l = np.array(c["l"], float)
        u = np.array([np.inf if v == "inf" else v for v in c["u"]], float)
        xs = np.array(c["x_star"], float)
        th = np.array(c["theta_star"], float)
        xb, Pb = O.brute_force(A, y, l, u)
        assert np.allclose(xb, xs, atol=1e-12), (c["name"], xb)
        assert abs(Pb - c["P_star"]) < 1e-12
        assert abs(O.primal_objective(A, y, xs) - c["P_star"]) < 1e-12
        assert abs(O.dual_objective(A, y, th, l, u) - c["P_star"]) < 1e-12, c["name"]
        assert np.allclose(O.theta_scaling(A, y, xs), th, atol=1e-12)
        assert O.dual_feasible(A, th, u, tol=1e-12)
        r = O.solve(A, y, l, u, tol=1e-12, screen_every=1, max_iter=20000)
        assert np.allclose(r.x, xs, atol=1e-7), (c["name"], r.x)
        S_l, S_u = O.safe_rule(A, th, 0.0, u)
        sign = np.array(c["screen_sign"])
        assert np.array_equal(S_l, sign == -1) and np.array_equal(S_u, sign == 1), c["name"]


def check_strong_duality(kinds=("bvls", "mixed", "nnls_abs")):
    for kind in kinds:
        for seed in range(3):
            p = W.random_tiny(7, 5, kind, seed)
            A, y = _f64(p)
            xb, Pb = O.brute_force(A, y, p.l, p.u)
            th = O.theta_scaling(A, y, xb)       # theta* = -f'(A x*) (Eq. (optimality1))
            assert O.dual_feasible(A, th, p.u, tol=1e-9)
            D = O.dual_objective(A, y, th, p.l, p.u)
            assert abs(Pb - D) < 1e-9 * (1 + abs(Pb)), (kind, seed, Pb, D)


def check_weak_duality_and_identity():
    rng = np.random.default_rng(5)
    for kind in ("bvls", "mixed", "nnls_abs", "nnls_gauss"):
        for seed in range(4):
            p = W.random_tiny(9, 6, kind, seed)
            A, y = _f64(p)
            l, u = p.l, p.u
            ub = np.where(np.isfinite(u), u, l + 3.0)
            t = O.choose_translation(A, u) if not np.all(np.isfinite(u)) else None
            for _ in range(10):
                x = rng.uniform(l, ub)
                r = y - A @ x
                if t is None and not np.all(np.isfinite(u)):
                    th = np.zeros_like(y)
                elif t is None:
                    th = r + 0.3 * rng.standard_normal(y.size)
                else:
                    th, _ = O.translate(A, r + 0.3 * rng.standard_normal(y.size), t,
                                        O.translation_columns(A, u))
                assert O.dual_feasible(A, th, u, tol=1e-10)
                P = O.primal_objective(A, y, x)
                D = O.dual_objective(A, y, th, l, u)
                assert D <= P + 1e-10 * (1 + abs(P)), (kind, seed)
                # Identity derived from |y|^2 = |Ax|^2 + 2<Ax, r> + |r|^2:
                # P(x) - D(theta) = sum_j [sigma_j(a_j^T theta) - x_j a_j^T theta] + |theta - r|^2 / 2.
                g = A.T @ th
                inf_cols = ~np.isfinite(u)
                assert np.all(g[inf_cols] <= 1e-10 * (1 + np.abs(g).max()))
                g = np.where(inf_cols, np.minimum(g, 0.0), g)   # F_D up to rounding
                rhs = float(np.sum(_sigma(g, l, u) - x * g) + 0.5 * (th - r) @ (th - r))
                gap = O.duality_gap(A, y, x, th, l, u)
                assert abs(gap - rhs) < 1e-9 * (1 + abs(P)), (kind, seed, gap, rhs)


def check_sphere_contains_theta_star():
    """Gap safe sphere (Eq. (GAP_Safe_sph), alpha = 1): ||theta - theta*|| <= sqrt(2 Gap)."""
    rng = np.random.default_rng(9)
    for kind in ("bvls", "nnls_abs", "mixed"):
        for seed in range(3):
            p = W.random_tiny(8, 6, kind, seed)
            A, y = _f64(p)
            xb, _ = O.brute_force(A, y, p.l, p.u)
            th_star = y - A @ xb
            ub = np.where(np.isfinite(p.u), p.u, p.l + 3.0)
            t = O.choose_translation(A, p.u) if not np.all(np.isfinite(p.u)) else None
            for _ in range(20):
                x = rng.uniform(p.l, ub)
                r = y - A @ x
                if t is None:
                    th = r
                else:
                    th, _ = O.translate(A, r, t, O.translation_columns(A, p.u))
                rad = O.safe_radius(O.duality_gap(A, y, x, th, p.l, p.u))
                assert np.linalg.norm(th - th_star) <= rad * (1 + 1e-9) + 1e-9, (kind, seed)


def check_solver_vs_brute_force(**kw):
    for kind in ("nnls_abs", "nnls_gauss", "bvls", "mixed"):
        for seed in range(3):
            p = W.random_tiny(9, 6, kind, seed)
            A, y = _f64(p)
            xb, Pb = O.brute_force(A, y, p.l, p.u)
            r = O.solve(A, y, p.l, p.u, tol=1e-11, screen_every=5, max_iter=200000, **kw)
            assert r.converged, (kind, seed, r.gap, r.dual_mode)
            assert abs(r.primal - Pb) < 1e-10 * (1 + Pb), (kind, seed)
            assert np.max(np.abs(r.x - xb)) < 1e-5, (kind, seed, r.x, xb)
            th_star = y - A @ xb
            g = A.T @ th_star
            # Every screened coordinate sits at its bound in the optimum (Eq. (screen_cond)).
            low, upp = r.screened == 1, r.screened == 2
            assert np.all(np.abs(xb[low] - p.l[low]) < 1e-9), (kind, seed)
            assert np.all(np.abs(xb[upp] - p.u[upp]) < 1e-9), (kind, seed)
            assert np.all(g[low] < 1e-9) and np.all(g[upp] > -1e-9)


def check_translation_validity():
    rng = np.random.default_rng(3)
    for seed in range(5):
        p = W.random_tiny(10, 8, "nnls_abs", seed)
        A, y = _f64(p)
        t = O.choose_translation(A, p.u)
        assert t is not None and np.all(A.T @ t < 0)
        cols = O.translation_columns(A, p.u)
        for _ in range(20):
            z = rng.standard_normal(y.size) * 3
            th, eps = O.translate(A, z, t, cols)
            g = A.T @ th
            assert np.all(g <= 1e-12 * (1 + np.abs(A.T @ z)))       # Proposition 1: in F_D
            if np.any(A.T @ z > 0):
                assert np.max(g) > -1e-9                               # eps is the smallest such step
            else:
                assert eps == 0.0 and np.array_equal(th, z)


# ----------------------------------------------------------------------------- tests
def test_golden_hand_derived():
    check_golden()


def test_closed_form_single_column():
    check_closed_form_1col({})
    check_closed_form_1col({"screening": False})


def test_identity_and_orthonormal_closed_forms():
    rng = np.random.default_rng(1)
    for trial in range(4):
        m, n = 12, 7
        Q, _ = np.linalg.qr(rng.standard_normal((m, n)))
        y = 2 * rng.standard_normal(m)
        for l, u in [(np.zeros(n), np.full(n, np.inf)), (-0.5 * np.ones(n), 0.7 * np.ones(n))]:
            exact = np.clip(Q.T @ y, l, u)            # separable after the change of basis
            r = O.solve(Q, y, l, u, tol=1e-12, screen_every=1, max_iter=5000)
            assert np.max(np.abs(r.x - exact)) < 1e-8
            if trial == 0:
                r = O.solve(np.eye(m), y, np.zeros(m), None, tol=1e-12, screen_every=1)
                assert np.allclose(r.x, np.maximum(y, 0), atol=1e-12)
                th = O.theta_scaling(np.eye(m), y, r.x)
                assert np.allclose(th, np.minimum(y, 0), atol=1e-12)


def test_brute_force_matches_scipy():
    for seed in range(4):
        p = W.random_tiny(10, 7, "nnls_abs", seed)
        A, y = _f64(p)
        xb, Pb = O.brute_force(A, y, p.l, p.u)
        xs, rn = so.nnls(A, y)
        assert abs(Pb - 0.5 * rn ** 2) < 1e-10 * (1 + Pb)
        assert np.allclose(xb, xs, atol=1e-8)
        p = W.random_tiny(10, 7, "bvls", seed)
        A, y = _f64(p)
        xb, Pb = O.brute_force(A, y, p.l, p.u)
        res = so.lsq_linear(A, y, bounds=(p.l, p.u), method="bvls", tol=1e-14)
        assert abs(Pb - O.primal_objective(A, y, res.x)) < 1e-9 * (1 + Pb)


def test_strong_duality_at_optimum():
    check_strong_duality()


def test_weak_duality_and_gap_identity():
    check_weak_duality_and_identity()


def test_sphere_contains_dual_optimum():
    check_sphere_contains_theta_star()


def test_translation_validity():
    check_translation_validity()


@pytest.mark.parametrize("kw", [{}, {"screening": False}, {"eps_scope": "all"}, {"restart": False}])
def test_solver_matches_brute_force(kw):
    check_solver_vs_brute_force(**kw)


def test_solver_matches_scipy_midsize():
    p = W.nnls_abs_gaussian(60, 150, 0.1, 1.0, 2)
    A, y = _f64(p)
    xs, rn = so.nnls(A, y, maxiter=5000)
    r = O.solve(A, y, p.l, p.u, tol=1e-10, screen_every=10)
    assert r.converged and abs(r.primal - 0.5 * rn ** 2) < 1e-9 * (1 + r.primal)
    assert np.max(np.abs(O.polish(A, y, r.x, p.l, p.u) - xs)) < 1e-7
    assert O.kkt_residual(A, y, r.x, p.l, p.u) < 1e-5
    th_star = y - A @ xs
    g = A.T @ th_star
    assert np.all(xs[r.screened == 1] == 0.0) and np.all(g[r.screened == 1] < 0)
    p = W.bvls_table2(80, 50, 4)
    A, y = _f64(p)
    res = so.lsq_linear(A, y, bounds=(p.l, p.u), method="bvls", tol=1e-14)
    r = O.solve(A, y, p.l, p.u, tol=1e-11, screen_every=10)
    assert r.converged and abs(r.primal - O.primal_objective(A, y, res.x)) < 1e-9 * (1 + r.primal)
    assert np.max(np.abs(r.x - res.x)) < 1e-5


def test_screening_does_not_change_iterates_when_pins_sit_at_bounds():
    p = W.nnls_abs_gaussian(40, 120, 0.1, 1.0, 7)
    A, y = _f64(p)
    a = O.solve(A, y, tol=1e-10, screen_every=10, record=True)
    b = O.solve(A, y, tol=1e-10, screen_every=10, screening=False, record=True)
    assert a.iters == b.iters and (a.screened > 0).sum() > 0
    assert np.max(np.abs(a.x - b.x)) < 1e-10


def test_degenerate_gaussian_family_has_no_interior_direction():
    # n = 2m Gaussian columns: 0 is inside conv{a_j} with overwhelming probability (Wendel),
    # so Int(F_D) is empty (remark after Proposition 1) and the NNLS optimum interpolates y.
    p = W.nnls_gaussian(100, 200, 0.1, 0.01, 0)
    A, y = _f64(p)
    assert O.choose_translation(A, p.u) is None
    xs, rn = so.nnls(A, y, maxiter=20000)
    assert rn < 1e-6
    r = O.solve(A, y, tol=1e-9, screen_every=10)
    assert r.converged and r.dual_mode == "zero" and r.screened.sum() == 0
    assert abs(r.gap - r.primal) < 1e-15


def test_choose_translation_cases():
    rng = np.random.default_rng(0)
    A = np.abs(rng.standard_normal((6, 9)))           # Proposition 2, case 3
    assert np.array_equal(O.choose_translation(A, np.full(9, np.inf)), -np.ones(6))
    A = rng.standard_normal((12, 5))                  # case 1: rank n <= m
    t = O.choose_translation(A, np.full(5, np.inf))
    assert t is not None and np.all(A.T @ t < 0)
    assert O.choose_translation(A, np.ones(5)) is None   # no column in J_inf


def test_bad_bounds_rejected():
    with pytest.raises(ValueError):
        O.as_problem(np.eye(2), np.ones(2), [0, 1], [1, 0])
    with pytest.raises(ValueError):
        O.as_problem(np.eye(2), np.ones(2), [-np.inf, 0], None)


# ----------------------------------------------------------------------------- planted slips
MUTANTS = {
    "dual_drops_upper_term": ("dual_objective",
        lambda A, y, th, l, u: 0.5 * y @ y - 0.5 * (y - th) @ (y - th) - np.sum(l * np.minimum(A.T @ th, 0))),
    "dual_sign_flip": ("dual_objective",
        lambda A, y, th, l, u: 0.5 * y @ y - 0.5 * (y - th) @ (y - th) + np.sum(l * np.minimum(A.T @ th, 0))
        + np.sum(np.where(np.isfinite(u), u, 0) * np.maximum(A.T @ th, 0))),
    "theta_sign_slip": ("theta_scaling", lambda A, y, x: y + A @ x),
    "primal_half_missing": ("primal_objective", lambda A, y, x: float((y - A @ x) @ (y - A @ x))),
    "radius_without_two": ("safe_radius", lambda gap, alpha=1.0: float(np.sqrt(max(gap, 0.0) / alpha))),
    "translation_wrong_sign": ("translate",
        lambda A, z, t, cols, w=None, margin=None: (z - 0.5 * t, 0.5)),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutations_are_caught(name, monkeypatch):
    import oracle.bvls as B
    attr, fn = MUTANTS[name]
    monkeypatch.setattr(B, attr, fn)
    monkeypatch.setattr(O, attr, fn)
    caught = 0
    for check in (check_golden, check_strong_duality, check_weak_duality_and_identity,
                  check_sphere_contains_theta_star, check_translation_validity):
        try:
            check()
        except (AssertionError, ValueError, RuntimeError, IndexError):
            caught += 1
    assert caught > 0, name


def test_fixed_dual_point_screens_safely_and_earlier():
    """Oracle-dual-point experiment (Section 5): with theta* itself as the dual point the
    gap of every evaluation is P(x_k) - P* (up to the folding), so the sphere is as small as
    Gap-safe screening allows; the solution and the screened set stay correct."""
    p = W.nnls_abs_gaussian(120, 400, 0.05, 1.0, 2)
    A, y = p.A.astype(np.float64), p.y.astype(np.float64)
    ref = O.solve(A, y, p.l, p.u, tol=1e-10)
    xs = O.polish(A, y, ref.x, p.l, p.u, tau=1e-7)
    assert O.kkt_residual(A, y, xs, p.l, p.u) < 1e-10
    th = y - A @ xs
    a = O.solve(A, y, p.l, p.u, tol=1e-8, record=True)
    b = O.solve(A, y, p.l, p.u, tol=1e-8, record=True, dual_point=th)
    assert b.converged and b.iters <= a.iters
    g = A.T @ th
    low = b.screened == 1
    assert np.all(xs[low] == 0.0) and np.all(g[low] < 0)
    pa = [h[2] for h in a.history]
    pb = [h[2] for h in b.history]
    k = min(len(pa), len(pb))
    assert all(pb[i] <= pa[i] for i in range(k)) and pb[k // 2] < pa[k // 2]
    assert O.primal_objective(A, y, b.x) - O.primal_objective(A, y, xs) <= b.gap + 1e-12


def test_chambolle_pock_matches_brute_force_and_fista():
    """The primal-dual solver (Section 5's PD) reaches the brute-force optimum on tiny BVLS
    problems, the FISTA solver's optimum on a Table-2 instance, and its dual iterate -z
    converges to theta*; screening does not change its iterates."""
    for seed in range(6):
        p = W.random_tiny(9, 6, "bvls", seed)
        A, y = p.A.astype(np.float64), p.y.astype(np.float64)
        xb, Pb = O.brute_force(A, y, p.l, p.u)
        r = O.solve_cp(A, y, p.l, p.u, tol=1e-12, screen_every=5)
        assert r.converged and abs(O.primal_objective(A, y, r.x) - Pb) <= 1e-10 * max(1.0, Pb)
    p = W.bvls_table2(100, 250, 3)
    A, y = p.A.astype(np.float64), p.y.astype(np.float64)
    a = O.solve(A, y, p.l, p.u, tol=1e-10)
    b = O.solve_cp(A, y, p.l, p.u, tol=1e-10)
    c = O.solve_cp(A, y, p.l, p.u, tol=1e-10, screening=False)
    xs = O.polish(A, y, a.x, p.l, p.u, tau=1e-7)
    assert O.kkt_residual(A, y, xs, p.l, p.u) < 1e-10
    assert np.abs(b.x - xs).max() < 1e-6 and np.abs(b.x - c.x).max() < 1e-12 and b.iters == c.iters
    g = A.T @ (y - A @ xs)
    assert np.all(xs[b.screened == 1] == 0.0) and np.all(g[b.screened == 1] < 0)
    assert np.all(xs[b.screened == 2] == 1.0) and np.all(g[b.screened == 2] > 0)
    with pytest.raises(ValueError):
        O.solve_cp(A, y, p.l, np.full(A.shape[1], np.inf))


@pytest.mark.parametrize("make", [lambda: W.nnls_abs_gaussian(300, 700, 0.05, 1.0, 1),
                                  lambda: W.bvls_table2(200, 500, 2),
                                  lambda: W.bvls_dirichlet_shared(224, 512, 1, 8, 0.005, 0),
                                  lambda: W.nnls_abs_gaussian(120, 400, 0.1, 1.0, 5)])
def test_fixing_at_bound_defers_nothing_on_the_test_families(make):
    """Algorithm 1 sets a coordinate that passes the test to its bound at once; the default
    reading fixes it once x_k and x_{k+1} already sit there.  On the test families every
    coordinate that passes the test already sits at its bound, so the two readings run the
    same iterates bit for bit."""
    p = make()
    A, y = _f64(p)
    L = 1.05 * O.lipschitz(A)
    a = O.solve(A, y, p.l, p.u, tol=1e-9, L=L, record=True)
    b = O.solve(A, y, p.l, p.u, tol=1e-9, L=L, record=True, pin="immediate")
    assert sum(h[3] for h in a.history) == 0
    assert a.iters == b.iters and np.array_equal(a.x, b.x) and np.array_equal(a.screened, b.screened)
    assert (a.screened > 0).sum() > 0


def test_literal_and_at_bound_fixing_reach_the_same_optimum():
    """A case where the readings differ: start at the certified optimum with a few
    coordinates that belong at 0 lifted to 1e-3, screen every iteration with the optimal dual
    point theta*.  The first evaluation (k = 0) sees a tiny sphere while those coordinates
    are still off their bound: the literal reading pins them at once, the default defers
    them.  At that evaluation the literal pins are the default's pins plus the deferred ones;
    both readings fix only coordinates that sit at that bound in the optimum and both reach
    it."""
    p = W.nnls_abs_gaussian(120, 400, 0.05, 1.0, 2)
    A, y = _f64(p)
    ref = O.solve(A, y, p.l, p.u, tol=1e-11)
    xs = O.polish(A, y, ref.x, p.l, p.u, tau=1e-7)
    assert O.kkt_residual(A, y, xs, p.l, p.u) < 1e-10
    th = y - A @ xs
    g = A.T @ th
    lifted = np.argsort(g)[:5]                      # the most negative a_j^T theta*
    assert np.all(xs[lifted] == 0.0)
    x0 = xs.copy()
    x0[lifted] = 1e-3
    a = O.solve(A, y, p.l, p.u, tol=1e-9, screen_every=1, x0=x0, dual_point=th, record=True)
    b = O.solve(A, y, p.l, p.u, tol=1e-9, screen_every=1, x0=x0, dual_point=th, record=True, pin="immediate")
    assert a.converged and b.converged
    assert a.history[0][3] >= 5                     # the lifted coordinates were deferred
    fixed_a0 = a.history[0][2] - a.history[1][2]
    fixed_b0 = b.history[0][2] - b.history[1][2]
    assert fixed_b0 == fixed_a0 + a.history[0][3]
    for r in (a, b):
        low = r.screened == 1
        assert np.all(xs[low] == 0.0) and np.all(g[low] < 0)
        xp = O.polish(A, y, r.x, p.l, p.u, tau=1e-7)
        assert np.abs(xp - xs).max() <= 1e-9 * max(1.0, np.abs(xs).max())
    with pytest.raises(ValueError):
        O.solve(A, y, p.l, p.u, pin="later")


# ---------------------------------------------------------------- batched Gram recurrence
def test_round_bf16_matches_the_library_conversion():
    """round_bf16 against torch's float32 -> bfloat16 conversion (round to nearest even), on
    ties, subnormal-range, large and random values."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    v = np.concatenate([
        [0.0, -0.0, 1.0, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -9, 1 - 2.0 ** -9, -2.5, 1e-30, 3.0e38, 65504.0],
        rng.standard_normal(2000) * 10.0 ** rng.integers(-6, 6, 2000)])
    ref = torch.tensor(v, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(O.round_bf16(v), ref)


@pytest.mark.parametrize("restart", [False, True])
def test_gram_recurrence_with_exact_operands_is_fista(restart):
    """Without the bf16 roundings the Gram-form iteration (exact correlations every K steps,
    g_k = g_{k-1} - A^T A (x_k - x_{k-1}) in between) is the exact-gradient FISTA of solve()
    step for step: the recurrence is exact because A x is affine in x.  solve() returns the
    iterate its last evaluation certifies, x_N after N + 1 iterations."""
    p = W.bvls_dirichlet_shared(64, 128, 5, 8, 0.005, 2)
    A, Y = p.A.astype(np.float64), p.y.astype(np.float64)
    L = 1.05 * np.linalg.norm(A, 2) ** 2
    for N in (1, 9, 10, 11, 30):
        G = O.gram_fista_batch(A, Y, p.l, p.u, L, screen_every=10, max_iter=N, restart=restart, bf16=False)
        for b in range(Y.shape[0]):
            r = O.solve(A, Y[b], p.l, p.u, tol=0.0, screen_every=10, screening=False, max_iter=N + 1,
                        L=L, restart=restart)
            assert np.abs(G[b] - r.x).max() <= 1e-13 * max(1.0, np.abs(r.x).max()), (N, b)


def test_gram_recurrence_bf16_operands_perturb_the_iterates():
    """The bf16 operands change the iterates between evaluations (so a comparison against
    the bf16 form tests the rounding, not only FISTA), by far less than the iterate."""
    p = W.bvls_dirichlet_shared(64, 128, 5, 8, 0.005, 2)
    A, Y = p.A.astype(np.float64), p.y.astype(np.float64)
    L = 1.05 * np.linalg.norm(A, 2) ** 2
    Gb = O.gram_fista_batch(A, Y, p.l, p.u, L, screen_every=10, max_iter=30, bf16=True)
    Ge = O.gram_fista_batch(A, Y, p.l, p.u, L, screen_every=10, max_iter=30, bf16=False)
    d = np.abs(Gb - Ge).max()
    assert 1e-7 < d < 1e-2 * np.abs(Ge).max()
    assert np.all(Gb >= p.l) and np.all(Gb <= p.u)
