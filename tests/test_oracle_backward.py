"""Pins of the oracle's backward pass (gradients through the solution map) on the CPU.

The oracle differentiates the restricted normal equations of the free set.  Here that is
checked against central finite differences (h = 1e-4, float64) of a loss evaluated at
solutions of the perturbed problems obtained independently of the oracle: scipy's
bounded-variable least squares (an exact active-set method, run in the test harness only),
polished on its free set and checked against the optimality conditions.  The instances are
non-degenerate (strict complementarity, full-column-rank free block), verified first.
Planted slips in the formula must fail the same comparison.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

H = 1e-4


def solution(A, y, l, u):
    from scipy.optimize import lsq_linear
    r = lsq_linear(A, y, bounds=(l, u), method="bvls", tol=1e-15)
    x = O.polish(A, y, r.x, l, u, tau=1e-9)
    assert O.kkt_residual(A, y, x, l, u) < 1e-11
    return x


def instances():
    out = []
    p = W.nnls_abs_gaussian(30, 50, 0.2, 1.0, 3)                    # NNLS, |N| matrix
    out.append(("nnls", p.A.astype(np.float64), p.y.astype(np.float64), p.l, p.u))
    p = W.bvls_box_shared(24, 40, 1, 0.08, 5)                         # BVLS, both bounds active
    out.append(("bvls", p.A.astype(np.float64), p.y[0].astype(np.float64), p.l, p.u))
    return out


def non_degenerate(A, y, x, l, u):
    F = O.free_set(x, l, u, 1e-9)
    g = A.T @ (y - A @ x)
    B = np.setdiff1d(np.arange(A.shape[1]), F)
    assert F.size > 0 and np.linalg.matrix_rank(A[:, F]) == F.size
    assert np.abs(g[B]).min() > 1e-6          # strict complementarity on the fixed coordinates
    return F


def fd_checks(backward_fn, name, A, y, l, u, n_entries=8, seed=0):
    rng = np.random.default_rng(seed)
    x = solution(A, y, l, u)
    F = non_degenerate(A, y, x, l, u)
    xt = rng.uniform(0.0, 1.0, A.shape[1])
    loss = lambda xx: 0.5 * float((xx - xt) @ (xx - xt))
    dy, dA, F2, w = backward_fn(A, y, x, x - xt, l, u)
    assert np.array_equal(F, F2)
    for i in range(A.shape[0]):
        e = np.zeros(A.shape[0])
        e[i] = H
        fd = (loss(solution(A, y + e, l, u)) - loss(solution(A, y - e, l, u))) / (2 * H)
        assert abs(fd - dy[i]) <= 1e-6 * (1 + abs(fd)), (name, "y", i, fd, dy[i])
    cols = np.concatenate([rng.choice(F, min(4, F.size), replace=False),
                           rng.choice(np.setdiff1d(np.arange(A.shape[1]), F), 2, replace=False)])
    for j in cols:
        for i in rng.choice(A.shape[0], max(1, n_entries // len(cols)), replace=False):
            Ap, Am = A.copy(), A.copy()
            Ap[i, j] += H
            Am[i, j] -= H
            fd = (loss(solution(Ap, y, l, u)) - loss(solution(Am, y, l, u))) / (2 * H)
            assert abs(fd - dA[i, j]) <= 1e-5 * (1 + abs(fd)), (name, "A", i, j, fd, dA[i, j])


@pytest.mark.parametrize("case", [0, 1])
def test_backward_matches_central_differences(case):
    name, A, y, l, u = instances()[case]
    fd_checks(O.backward, name, A, y, l, u)


def test_backward_closed_form_single_free_column():
    """One column, interior optimum x = a^T y / ||a||^2: dx/dy = a / ||a||^2 and
    dx/da = (y - 2 a x) / ||a||^2, so for L = x both gradients are known in closed form."""
    rng = np.random.default_rng(1)
    a = rng.standard_normal(7)
    y = 3.0 * a + 0.1 * rng.standard_normal(7)
    A = a[:, None]
    x = np.array([a @ y / (a @ a)])
    dy, dA, F, w = O.backward(A, y, x, np.ones(1), np.zeros(1), np.full(1, np.inf))
    assert np.allclose(dy, a / (a @ a), rtol=1e-12, atol=1e-14)
    assert np.allclose(dA[:, 0], (y - 2 * a * x[0]) / (a @ a), rtol=1e-12, atol=1e-14)


def _drop_rank_one(A, y, x, v, l=None, u=None, tau=1e-9):
    dy, dA, F, w = O.backward(A, y, x, v, l, u, tau)
    return dy, dA + np.outer(dy, x), F, w


def _wrong_sign(A, y, x, v, l=None, u=None, tau=1e-9):
    dy, dA, F, w = O.backward(A, y, x, v, l, u, tau)
    return -dy, dA, F, w


def _all_columns(A, y, x, v, l=None, u=None, tau=1e-9):
    dy, dA, F, w = O.backward(A, y, x, v, l, u, tau)
    wa = np.linalg.lstsq(A.T @ A + 1e-9 * np.eye(A.shape[1]), v, rcond=None)[0]
    return A @ wa, dA, F, w


@pytest.mark.parametrize("mutant", [_drop_rank_one, _wrong_sign, _all_columns])
def test_planted_backward_slips_are_caught(mutant):
    name, A, y, l, u = instances()[0]
    with pytest.raises(AssertionError):
        fd_checks(mutant, name, A, y, l, u, n_entries=4)
