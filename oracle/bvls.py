"""FP64 oracle: box-constrained least squares with dynamic Gap safe screening.

TEST INFRASTRUCTURE (see the package docstring): only the tests, the smoke check and the
CPU-baseline leg of the benchmark use this module.

Problem (Section 2, Eq. (LR) with the least-squares loss of Section 5):

    x* in argmin_x  P(x) = 1/2 ||y - A x||^2   s.t.  l <= x <= u,

l finite, u in R U {+inf}.  J_inf = {j : u_j = +inf}.  NNLS is l = 0, u = +inf;
BVLS has every u_j finite.

Everything here is float64 NumPy written for readability, not speed.  A library primitive
(matrix-vector product, lstsq, SVD norm) may serve as a step; no blocking or fusion.

Readings of points the paper leaves open:
  * Primal solver: FISTA with step 1/L and the gradient-based adaptive restart of
    O'Donoghue and Candes; the paper's experiments use plain projected gradient.
  * The screening step of Algorithm 1 is evaluated every ``screen_every`` iterations at the
    iterate x_k whose gradient the step has just used (so the inner products of the safe
    rule are those of the step).  A coordinate that passes the test is fixed once x_k and
    x_{k+1} both sit at that bound (the assignment of Algorithm 1 is then exact); the
    momentum is kept and the extrapolation runs over the preserved set only.
  * The dual point and the gap are those of the reduced problem on the preserved set
    (data y folded as in the remark after Eq. (decmposition_fwd)); the translation maximum
    runs over the preserved columns of J_inf.  ``eps_scope="all"`` gives the literal
    reading (maximum over all of [n], gap of the original problem).
  * Zero columns are never screened and take no part in the translation maximum.
  * When no interior translation direction is found, theta = 0 (always dual feasible);
    the gap is then P(x) and nothing can be screened.
  * The sphere test runs with the FP64 rounding bounds of ``rounding_pads`` added to the
    radius and to the translation step, so rounding never fixes a free coordinate.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "as_problem",
    "primal_objective",
    "support_function",
    "dual_objective",
    "dual_feasible",
    "duality_gap",
    "theta_scaling",
    "translate",
    "translation_columns",
    "safe_radius",
    "safe_rule",
    "rounding_pads",
    "choose_translation",
    "lipschitz",
    "SolveResult",
    "solve",
    "brute_force",
    "kkt_residual",
    "polish",
    "free_set",
    "backward",
    "solve_cp",
    "round_bf16",
    "gram_fista_batch",
]


def as_problem(A, y, l=None, u=None):
    """Return (A, y, l, u) as float64 arrays with the bounds broadcast to length n.

    l defaults to 0 and u to +inf (the NNLS problem).  Raises ValueError when l is not
    finite or l > u (the box [l, u] of Section 2 must be nonempty with l in R^n).
    """
    A = np.asarray(A, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if A.ndim != 2 or y.shape != (A.shape[0],):
        raise ValueError("A must be (m, n) and y (m,)")
    n = A.shape[1]
    l = np.zeros(n) if l is None else np.array(np.broadcast_to(np.asarray(l, np.float64), (n,)))
    u = np.full(n, np.inf) if u is None else np.array(np.broadcast_to(np.asarray(u, np.float64), (n,)))
    if not np.all(np.isfinite(l)):
        raise ValueError("lower bounds must be finite")
    if np.any(np.isnan(u)) or np.any(u == -np.inf) or np.any(l > u):
        raise ValueError("need l <= u with u in R or +inf")
    return A, y, l, u


def primal_objective(A, y, x):
    """P(x) = sum_i f([Ax]_i; y_i) with f(z; y) = 1/2 (z - y)^2  (Eq. (LR), Section 5)."""
    r = y - A @ x
    return 0.5 * float(r @ r)


def support_function(g, l, u):
    """sigma_j(g_j) = sup_{x_j in [l_j, u_j]} x_j g_j = l_j [g_j]^- + u_j [g_j]^+  (Appendix B).

    For u_j = +inf the value is +inf when g_j > 0 (the indicator of Appendix B).
    """
    g = np.asarray(g, dtype=np.float64)
    neg = np.minimum(g, 0.0)
    pos = np.maximum(g, 0.0)
    out = l * neg
    fin = np.isfinite(u)
    out = out + np.where(fin, np.where(fin, u, 0.0) * pos, np.where(pos > 0, np.inf, 0.0))
    return out


def dual_objective(A, y, theta, l, u):
    """D(theta) of Eq. (Dual_obj) with the least-squares conjugate of Section 5.

    f*(theta; y) = 1/2 ((y + theta)^2 - y^2), so -sum_i f*(-theta_i; y_i)
    = 1/2 ||y||^2 - 1/2 ||y - theta||^2.  The box terms are
    - sum_j l_j [A^T theta]^-_j - sum_{j not in J_inf} u_j [A^T theta]^+_j.

    This is the finite part of the dual function; membership in F_D (Eq. (Dual_set)) is
    checked separately by ``dual_feasible``.
    """
    g = A.T @ theta
    fin = np.isfinite(u)
    lin = 0.5 * float(y @ y) - 0.5 * float((y - theta) @ (y - theta))
    low = float(np.sum(l * np.minimum(g, 0.0)))
    upp = float(np.sum(u[fin] * np.maximum(g[fin], 0.0)))
    return lin - low - upp


def dual_feasible(A, theta, u, tol=0.0):
    """theta in F_D  <=>  a_j^T theta <= 0 for every j in J_inf  (Eq. (Dual_set))."""
    inf_cols = ~np.isfinite(u)
    if not inf_cols.any():
        return True
    return bool(np.all(A[:, inf_cols].T @ theta <= tol))


def duality_gap(A, y, x, theta, l, u):
    """Gap(x, theta) = P(x) - D(theta)  (Eq. (Dual_Gap))."""
    return primal_objective(A, y, x) - dual_objective(A, y, theta, l, u)


def theta_scaling(A, y, x):
    """Theta(x) = -grad F(Ax; y) = y - Ax  (Eq. (BVLR_dual_up); for least squares grad F(z) = z - y)."""
    return y - A @ x


def translation_columns(A, u):
    """Columns over which the translation maximum of Section 4.2 runs: J_inf minus zero columns.

    A zero column satisfies a_j^T theta = 0 <= 0 for every theta, so it never constrains F_D.
    """
    return (~np.isfinite(u)) & np.any(A != 0.0, axis=0)


def translate(A, z, t, cols, w=None, margin=None):
    """Xi_t(z) = z + (max_{j in cols} (a_j^T z)^+ / |a_j^T t|) t   (Section 4.2, dual translation).

    ``cols`` is a boolean mask of the columns in the maximum (the paper's [n], restricted
    to J_inf for mixed bounds).  Requires a_j^T t < 0 on those columns (t in Int(F_D)).
    ``margin`` (per column, optional) is added to a_j^T z inside the maximum so that the
    result stays in F_D despite rounding.  Returns (theta, eps).
    """
    if w is None:
        w = A.T @ t
    if not cols.any():
        return z.copy(), 0.0
    wc = w[cols]
    if np.any(wc >= 0.0):
        raise ValueError("t is not an interior direction of F_D on the given columns")
    gc = A[:, cols].T @ z
    if margin is not None:
        gc = gc + margin[cols]
    eps = float(np.max(np.maximum(gc, 0.0) / np.abs(wc)))
    return z + eps * t, eps


def rounding_pads(A, y, x, theta):
    """(tau, pad): FP64 rounding bounds for the screening step of this module.

    With s = ||y|| + sum_j |x_j| ||a_j|| + ||theta|| and gamma = (m+4) 2^-53 / (1 - (m+4) 2^-53),
    every computed a_j^T theta is within tau ||a_j||, tau = 4 gamma s, of its exact value
    and the computed gap within pad = 4 gamma s^2 of the exact P - D.  The safe rule is
    applied with radius sqrt(2 (Gap + pad)) + tau so that rounding can never fix a free
    coordinate (the rule of Eq. (safe_rule) is stated in exact arithmetic).
    """
    m = A.shape[0]
    u = 2.0 ** -53
    gamma = (m + 4) * u / (1.0 - (m + 4) * u)
    nrm = np.linalg.norm(A, axis=0)
    s = float(np.linalg.norm(y) + np.sum(np.abs(x) * nrm) + np.linalg.norm(theta))
    return 4.0 * gamma * s, 4.0 * gamma * s * s


def safe_radius(gap, alpha=1.0):
    """r = sqrt(2 Gap / alpha)  (Eq. (GAP_Safe_sph)); alpha = 1 for the least-squares loss."""
    return float(np.sqrt(2.0 * max(gap, 0.0) / alpha))


def safe_rule(A, theta, radius, u):
    """The Gap safe sphere test of Eq. (safe_rule).

    Returns boolean masks (S_l, S_u): a_j^T theta < -r ||a_j||  =>  x*_j = l_j;
    for j not in J_inf, a_j^T theta > r ||a_j||  =>  x*_j = u_j.
    """
    g = A.T @ theta
    nrm = np.linalg.norm(A, axis=0)
    S_l = g < -radius * nrm
    S_u = np.isfinite(u) & (g > radius * nrm)
    return S_l, S_u


def choose_translation(A, u):
    """A direction t in Int(F_D) for the translation of Section 4.2, or None.

    Candidates, in order: t = -1 (Proposition 2, case 3, the choice of the NNLS
    experiments), t = -(1/n) sum_j a_j and t = -a_+ where a_+ is the column most correlated
    with all the others (the choices compared in Section 5; case 4 of Proposition 2 when
    A^T a_+ > 0), then, when n <= m, the least-squares solution of A^T t = -1 (case 1).
    A candidate is kept when a_j^T t < 0 on every translation column.
    """
    cols = translation_columns(A, u)
    if not cols.any():
        return None
    m, n = A.shape
    s = A.sum(axis=1)                      # sum_j a_j
    cands = [-np.ones(m), -s / n]
    corr = A.T @ s                         # a_j^T sum_k a_k
    cands.append(-A[:, int(np.argmax(corr))].copy())
    if n <= m:
        # Proposition 2, case 1: rank(A) = n <= m, so A^T t = -1 has a solution.
        cands.append(np.linalg.lstsq(A.T, -np.ones(n), rcond=None)[0])
    for t in cands:
        w = A[:, cols].T @ t
        if np.all(w < 0.0):
            return t
    return None


def lipschitz(A):
    """Lipschitz constant of grad P: ||A||_2^2 (largest singular value squared)."""
    return float(np.linalg.norm(A, 2) ** 2)


@dataclass
class SolveResult:
    x: np.ndarray
    gap: float
    primal: float
    iters: int
    screened: np.ndarray          # int8 per coordinate: 0 preserved, 1 fixed at l, 2 fixed at u
    converged: bool
    dual_mode: str                # "scaling", "translation" or "zero"
    L: float
    t: np.ndarray | None
    history: list = field(default_factory=list)   # (iteration, gap, |preserved|, deferred) per evaluation


def _dual_point(A, y, x, l, u, mode, t, w, cols):
    """Theta(x) for the given problem: scaling (BVLS), translation (J_inf nonempty) or zero."""
    if mode == "scaling":
        return theta_scaling(A, y, x)
    if mode == "translation":
        z = theta_scaling(A, y, x)
        tau, _ = rounding_pads(A, y, x, z)
        theta, _ = translate(A, z, t, cols, w, margin=tau * np.linalg.norm(A, axis=0))
        return theta
    return np.zeros(A.shape[0])


def _fixed_dual_point(A, y, x, theta0, mode, t, w, cols):
    """A caller-given dual point, translated into F_D (Eq. (BVLR_dual_up2)) when some
    a_j^T theta0 > 0 on J_inf; with no interior direction it is used only if feasible."""
    theta0 = np.asarray(theta0, dtype=np.float64)
    if mode == "translation":
        tau, _ = rounding_pads(A, y, x, theta0)
        theta, _ = translate(A, theta0, t, cols, w, margin=tau * np.linalg.norm(A, axis=0))
        return theta
    if mode == "zero" and cols.size and np.max(A[:, cols].T @ theta0) > 0.0:
        return np.zeros(A.shape[0])
    return theta0


def solve(A, y, l=None, u=None, *, tol=1e-6, screen_every=10, screening=True,
          max_iter=100_000, x0=None, L=None, t=None, eps_scope="preserved",
          restart=True, record=False, dual_point=None, pin="at_bound"):
    """Algorithm 1 (Algorithm 2 for NNLS) with a FISTA primal update.

    Each iteration k computes, on the preserved set A:
      v_k     = x_k + beta_k (x_k - x_{k-1}),   beta_k = (t_k - 1)/t_{k+1},
                t_{k+1} = (1 + sqrt(1 + 4 t_k^2))/2, t_0 = 1;
      x_{k+1} = clip(v_k + A^T (y' - A v_k) / L, l, u)                (PrimalUpdate);
      restart (t_{k+1} = 1) when (A^T (y' - A v_k))^T (x_{k+1} - x_k) < 0.
    Every ``screen_every`` iterations (and at the last one) the screening step runs at x_k:
      theta = Theta(x_k) (Eq. (BVLR_dual_up) or Eq. (BVLR_dual_up2)), Gap (Eq. (Dual_Gap)),
      r = sqrt(2 Gap) (Eq. (GAP_Safe_sph)), S_l, S_u by Eq. (safe_rule) among coordinates
      already at that bound in x_k and x_{k+1}, y' <- y' - A_S x_S, A <- A \\ S (momentum
      kept), and the loop stops when Gap < tol, returning x_k.
    ``screening=False`` runs the same iteration and gap evaluations with nothing fixed.
    ``dual_point`` (length m) replaces Theta(x_k) in every screening step by a fixed dual
    point (translated into F_D when needed) -- the oracle-dual-point experiment of Section 5,
    where theta* itself informs the test; any feasible point keeps the sphere safe.
    ``pin="immediate"`` is Algorithm 1 read literally: every coordinate that passes the
    test is set to its bound at once (x_S <- bounds), also when x_k or x_{k+1} is not there
    yet; ``pin="at_bound"`` (default) fixes it only once both sit at that bound and records,
    per evaluation, how many passing coordinates it deferred (the fourth history entry).
    """
    A, y, l, u = as_problem(A, y, l, u)
    m, n = A.shape
    K = int(screen_every)
    if K < 1 or max_iter < 1:
        raise ValueError("screen_every and max_iter must be >= 1")
    if pin not in ("at_bound", "immediate"):
        raise ValueError("pin must be 'at_bound' or 'immediate'")
    fin = np.isfinite(u)
    if fin.all():
        mode = "scaling"
        t_dir = None
    else:
        t_dir = choose_translation(A, u) if t is None else np.asarray(t, dtype=np.float64)
        mode = "zero" if t_dir is None else "translation"
    w_all = A.T @ t_dir if t_dir is not None else None
    cols_all = translation_columns(A, u)
    if L is None:
        L = lipschitz(A)
    L = float(L)

    x = np.zeros(n) if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    x = np.clip(x, l, u)
    active = np.ones(n, dtype=bool)
    screened = np.zeros(n, dtype=np.int8)
    y_red = y.copy()
    x_prev = x.copy()
    tk = 1.0
    history = []
    gap = np.inf

    for k in range(max_iter):
        P = np.flatnonzero(active)
        A_P = A[:, P]
        lP, uP = l[P], u[P]
        xP = x[P]
        # PrimalUpdate: one accelerated projected-gradient step on the preserved set.
        t_next = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * tk * tk))
        beta = (tk - 1.0) / t_next
        v = xP + beta * (xP - x_prev[P])
        g_v = A_P.T @ (y_red - A_P @ v)
        x_new = x.copy()
        x_new[P] = np.clip(v + g_v / L, lP, uP)
        if restart and float(g_v @ (x_new[P] - xP)) < 0.0:
            t_next = 1.0

        if (k + 1) % K == 0 or k == max_iter - 1:
            # Dynamic safe screening at x_k.
            if eps_scope == "all":
                theta = _dual_point(A, y, x, l, u, mode, t_dir, w_all, cols_all) if dual_point is None \
                    else _fixed_dual_point(A, y, x, dual_point, mode, t_dir, w_all, cols_all)
                gap = duality_gap(A, y, x, theta, l, u)
            else:
                cols_P = cols_all[P]
                w_P = w_all[P] if w_all is not None else None
                theta = _dual_point(A_P, y_red, xP, lP, uP, mode, t_dir, w_P, cols_P) if dual_point is None \
                    else _fixed_dual_point(A_P, y_red, xP, dual_point, mode, t_dir, w_P, cols_P)
                gap = duality_gap(A_P, y_red, xP, theta, lP, uP)
            deferred = 0
            if screening and mode != "zero":
                if eps_scope == "all":
                    tau, pad = rounding_pads(A, y, x, theta)
                else:
                    tau, pad = rounding_pads(A_P, y_red, xP, theta)
                radius = safe_radius(gap + pad)
                S_l, S_u = safe_rule(A_P, theta, radius + tau, uP)
                S_u &= ~S_l
                if pin == "at_bound":
                    # A coordinate is fixed once x_k and x_{k+1} both sit at the bound the rule
                    # names (the assignment x_S <- bounds of Algorithm 1 is then exact and the
                    # momentum stays consistent); until then it stays in the preserved set.
                    passing = int(S_l.sum() + S_u.sum())
                    S_l &= (xP == lP) & (x_new[P] == lP)
                    S_u &= (xP == uP) & (x_new[P] == uP)
                    deferred = passing - int(S_l.sum() + S_u.sum())
                low, upp = P[S_l], P[S_u]
                pinned = np.concatenate([low, upp])
                if pinned.size:
                    x[low] = l[low]
                    x[upp] = u[upp]
                    x_new[pinned] = x[pinned]
                    y_red = y_red - A[:, pinned] @ x[pinned]
                    active[pinned] = False
                    screened[low] = 1
                    screened[upp] = 2
            history.append((k, gap, int(P.size), deferred))
            if gap < tol or k == max_iter - 1:
                # x_k is the iterate the gap certifies (also when max_iter ends the loop)
                return SolveResult(x, gap, primal_objective(A, y, x), k + 1, screened,
                                   bool(gap < tol), mode, L, t_dir, history if record else [])
        x_prev, x, tk = x, x_new, t_next
    raise AssertionError("unreachable: the last iteration always evaluates the gap")


def brute_force(A, y, l=None, u=None, tol=1e-9):
    """Exact optimum by enumerating which coordinates sit at l, at u, or are free.

    For each pattern the free coordinates solve the unconstrained least-squares problem
    with the others fixed; a candidate is kept when it lies in the box and satisfies the
    optimality conditions of Section 3.2 (Eq. (optimality2)): a_j^T theta <= 0 at l,
    >= 0 at u, = 0 inside.  Any such point is a global minimiser (convex problem); the one
    with the smallest objective is returned as (x*, P*).  Patterns whose free columns are
    rank deficient are skipped (an optimum with independent free columns always exists).
    """
    A, y, l, u = as_problem(A, y, l, u)
    m, n = A.shape
    if n > 12:
        raise ValueError("brute force is for n <= 12")
    scale = max(1.0, float(np.max(np.abs(A.T @ y))), float(np.linalg.norm(A) ** 2))
    choices = [(0, 1, 2) if np.isfinite(u[j]) else (0, 1) for j in range(n)]
    best_x, best_P = None, np.inf
    for pat in itertools.product(*choices):
        pat = np.array(pat)
        x = np.where(pat == 2, np.where(np.isfinite(u), u, 0.0), l).astype(np.float64)
        F = np.flatnonzero(pat == 1)
        if F.size:
            A_F = A[:, F]
            if np.linalg.matrix_rank(A_F) < F.size:
                continue
            fixed = np.flatnonzero(pat != 1)
            rhs = y - A[:, fixed] @ x[fixed]
            z = np.linalg.lstsq(A_F, rhs, rcond=None)[0]
            if np.any(z < l[F] - tol * (1 + np.abs(l[F]))) or np.any(z > u[F] + tol * (1 + np.abs(u[F]))):
                continue
            x[F] = np.clip(z, l[F], u[F])
        g = A.T @ (y - A @ x)
        at_l, at_u = pat == 0, pat == 2
        if np.any(g[at_l] > tol * scale) or np.any(g[at_u] < -tol * scale):
            continue
        Pv = primal_objective(A, y, x)
        if Pv < best_P:
            best_x, best_P = x, Pv
    if best_x is None:
        raise RuntimeError("no pattern satisfied the optimality conditions")
    return best_x, best_P


def kkt_residual(A, y, x, l=None, u=None):
    """|| x - clip(x + A^T (y - A x), l, u) ||_inf: zero exactly at the optima of Section 3.2."""
    A, y, l, u = as_problem(A, y, l, u)
    g = A.T @ (y - A @ x)
    return float(np.max(np.abs(x - np.clip(x + g, l, u)))) if x.size else 0.0


def polish(A, y, x, l=None, u=None, tau=1e-9):
    """Snap coordinates within tau of a bound to it and re-solve the free ones exactly.

    The free set is {j : l_j + tau < x_j < u_j - tau}; the returned point solves the
    normal equations on it with the other coordinates fixed.  The caller checks feasibility
    and ``kkt_residual``.
    """
    A, y, l, u = as_problem(A, y, l, u)
    x = np.asarray(x, dtype=np.float64)
    at_l = x <= l + tau * (1 + np.abs(l))
    uu = np.where(np.isfinite(u), u, np.inf)
    at_u = np.isfinite(u) & (x >= uu - tau * (1 + np.abs(np.where(np.isfinite(u), u, 0.0))))
    at_u &= ~at_l
    xp = np.where(at_l, l, np.where(at_u, np.where(np.isfinite(u), u, 0.0), x))
    F = np.flatnonzero(~(at_l | at_u))
    if F.size:
        fixed = np.flatnonzero(at_l | at_u)
        rhs = y - A[:, fixed] @ xp[fixed]
        xp[F] = np.linalg.lstsq(A[:, F], rhs, rcond=None)[0]
    return xp


def free_set(x, l, u, tau=1e-9):
    """Indices of the coordinates strictly inside the box, with a relative margin tau:
    l_j + tau (1 + |l_j|) < x_j < u_j - tau (1 + |u_j|)."""
    x = np.asarray(x, dtype=np.float64)
    l = np.asarray(l, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    above = x > l + tau * (1 + np.abs(l))
    uu = np.where(np.isfinite(u), u, 0.0)
    below = ~np.isfinite(u) | (x < uu - tau * (1 + np.abs(uu)))
    return np.flatnonzero(above & below)


def backward(A, y, x, dLdx, l=None, u=None, tau=1e-9):
    """Gradients of a loss L(x*) through the solution map (y, A) -> x*(y, A).

    At a non-degenerate optimum (strict complementarity, A_F of full column rank on the free
    set F of ``free_set``) the optimality conditions of Section 3.2 pin the other
    coordinates at their bounds and make x_F the solution of the restricted normal
    equations  A_F^T A_F x_F = A_F^T (y - A_B x_B).  Differentiating them gives, with
    w = (A_F^T A_F)^{-1} (dL/dx)_F extended by zeros off F and r = y - A x:

        dL/dy = A_F w_F,        dL/dA = r w^T - (A_F w_F) x^T.

    Components of dL/dx on the fixed coordinates do not flow back (the solution does not
    move with y or A there).  Returns (dL/dy, dL/dA, F, w).
    """
    A, y, l, u = as_problem(A, y, l, u)
    x = np.asarray(x, dtype=np.float64)
    v = np.asarray(dLdx, dtype=np.float64)
    F = free_set(x, l, u, tau)
    w = np.zeros(A.shape[1])
    if F.size:
        AF = A[:, F]
        w[F] = np.linalg.solve(AF.T @ AF, v[F])
    q = A[:, F] @ w[F] if F.size else np.zeros(A.shape[0])
    r = y - A @ x
    return q, np.outer(r, w) - np.outer(q, x), F, w


def solve_cp(A, y, l, u, *, tol=1e-6, screen_every=10, screening=True, max_iter=100_000,
             x0=None, L=None, step=0.99, record=False):
    """Chambolle-Pock primal-dual iteration for BVLS (every u_j finite) with the screening
    of Algorithm 1, the paper's PD solver of Section 5 (Table 2).

    Saddle form  min_x max_z <A x, z> - f*(z) + i_[l,u](x)  with f(v) = 1/2 ||v - y'||^2,
    f*(z) = 1/2 ||z||^2 + <z, y'>; with sigma = tau = step / sqrt(L), L >= ||A||_2^2:
        z_{k+1}    = (z_k + sigma (A xbar_k - y')) / (1 + sigma)        (prox of sigma f*)
        x_{k+1}    = clip(x_k - tau A^T z_{k+1}, l, u)
        xbar_{k+1} = 2 x_{k+1} - x_k,        z_0 = A x_0 - y', xbar_0 = x_0.
    At the optimum z* = -theta*.  Every ``screen_every`` iterations the screening step runs
    on the pair (x_{k+1}, theta = -z_{k+1}) -- the solver's own dual iterate, feasible for
    BVLS -- with the gap of Eq. (Dual_Gap), the radius of Eq. (GAP_Safe_sph) and the rule
    of Eq. (safe_rule); a coordinate is fixed once x_k and x_{k+1} sit at the bound the rule
    names, its column is folded into y', and the loop stops when Gap < tol, returning x_{k+1}.
    """
    A, y, l, u = as_problem(A, y, l, u)
    if not np.all(np.isfinite(u)):
        raise ValueError("solve_cp covers BVLS (every u_j finite)")
    m, n = A.shape
    K = int(screen_every)
    if L is None:
        L = lipschitz(A)
    tau = sigma = float(step) / np.sqrt(float(L))
    x = np.clip(np.zeros(n) if x0 is None else np.asarray(x0, dtype=np.float64).copy(), l, u)
    active = np.ones(n, dtype=bool)
    screened = np.zeros(n, dtype=np.int8)
    y_red = y.copy()
    z = A @ x - y_red
    xbar = x.copy()
    history = []
    gap = np.inf
    for k in range(max_iter):
        P = np.flatnonzero(active)
        A_P = A[:, P]
        z = (z + sigma * (A_P @ xbar[P] - y_red)) / (1.0 + sigma)
        gz = A_P.T @ z
        x_new = x.copy()
        x_new[P] = np.clip(x[P] - tau * gz, l[P], u[P])
        xbar = 2.0 * x_new - x
        if (k + 1) % K == 0 or k == max_iter - 1:
            theta = -z
            xP = x_new[P]
            gap = duality_gap(A_P, y_red, xP, theta, l[P], u[P])
            history.append((k, gap, int(P.size)))
            if screening:
                tau_r, pad = rounding_pads(A_P, y_red, xP, theta)
                radius = safe_radius(gap + pad)
                S_l, S_u = safe_rule(A_P, theta, radius + tau_r, u[P])
                S_l &= (x[P] == l[P]) & (xP == l[P])
                S_u &= ~S_l & (x[P] == u[P]) & (xP == u[P])
                low, upp = P[S_l], P[S_u]
                pinned = np.concatenate([low, upp])
                if pinned.size:
                    y_red = y_red - A[:, pinned] @ x_new[pinned]
                    active[pinned] = False
                    screened[low] = 1
                    screened[upp] = 2
            if gap < tol or k == max_iter - 1:
                return SolveResult(x_new, gap, primal_objective(A, y, x_new), k + 1, screened,
                                   bool(gap < tol), "scaling", float(L), None,
                                   history if record else [])
        x = x_new
    raise AssertionError("unreachable: the last iteration always evaluates the gap")



def round_bf16(v):
    """Round float64 values to bfloat16 (8 significant bits, round to nearest, ties to even),
    returned as float64: the value is first rounded to float32 (the precision the operands
    have before conversion), then its float32 bit pattern is rounded at bit 16."""
    f = np.asarray(v, dtype=np.float64).astype(np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    rounded = ((bits + 0x7FFF + lsb) >> 16) << 16
    out = (rounded & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)
    finite = np.isfinite(f)
    return np.where(finite, out, f.astype(np.float64))


def gram_fista_batch(A, Y, l, u, L, *, screen_every=10, max_iter=30, restart=False, x0=None,
                     bf16=True):
    """The batched iteration for B right-hand sides sharing A, without screening: FISTA (as
    ``solve``) whose correlations g_k = A^T (y - A x_k) are formed exactly every
    ``screen_every`` iterations (k = 0, K, 2K, ...) and in between by the Gram recurrence

        g_k = g_{k-1} - H d_k,   d_k = x_k - x_{k-1},   H = A^T A,

    exact in exact arithmetic because A x is affine in x.  With ``bf16`` the recurrence uses
    H~ = bf16(A^T A) and d~_k = bf16(d_k) (the tensor-core operands), and the step's
    momentum term uses d~_k as well; the evaluation steps use the exact d_k.  Every step:

        t_k = 1 at k = 0 (or after a restart), else (1 + sqrt(1 + 4 t_{k-1}^2)) / 2,
        beta_k = (t_k - 1) / t_{k+1},   g_v = (1 + beta_k) g_k - beta_k g_{k-1},
        x_{k+1} = clip(x_k + beta_k d_k + g_v / L, l, u),

    and with ``restart`` t_k = 1 when g_v^T (x_k - x_{k-1}) < 0 at step k - 1.  Y is B x m;
    returns X (B x n) after ``max_iter`` steps.  With bf16=False this is the exact-gradient
    FISTA of ``solve(..., screening=False)``, step for step."""
    A = np.asarray(A, dtype=np.float64)
    Y = np.atleast_2d(np.asarray(Y, dtype=np.float64))
    m, n = A.shape
    l = np.zeros(n) if l is None else np.asarray(l, dtype=np.float64)
    u = np.full(n, np.inf) if u is None else np.asarray(u, dtype=np.float64)
    K = int(screen_every)
    H = A.T @ A
    if bf16:
        H = round_bf16(H)
    out = np.empty((Y.shape[0], n))
    for b in range(Y.shape[0]):
        y = Y[b]
        x = np.clip(np.zeros(n) if x0 is None else np.asarray(x0[b], dtype=np.float64), l, u)
        x_prev = x.copy()
        g_prev = np.zeros(n)
        d_op = np.zeros(n)          # the recurrence's operand for the next step
        t_prev, dsum_prev = 1.0, 0.0
        for k in range(max_iter):
            if k == 0 or (restart and dsum_prev < 0.0):
                t = 1.0
            else:
                t = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t_prev * t_prev))
            t_next = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
            beta = (t - 1.0) / t_next
            if k % K == 0:
                g = A.T @ (y - A @ x)
                d_mom = x - x_prev
            else:
                g = g_prev - H @ d_op
                d_mom = d_op
            gv = (1.0 + beta) * g - beta * g_prev
            x_next = np.clip(x + beta * d_mom + gv / L, l, u)
            d = x_next - x
            dsum_prev = float(gv @ d)
            d_op = round_bf16(d) if bf16 else d
            x_prev, x = x, x_next
            g_prev, t_prev = g, t
        out[b] = x
    return out
