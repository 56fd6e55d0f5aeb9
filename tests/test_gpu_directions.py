"""The translation directions of Section 4.2 chosen by bvls_setup, against the oracle.

NNLS needs a direction t with a_j^T t < 0 on every column (Proposition 2) to translate
y - A x into the dual feasible set.  Setup tries, in the oracle's order, t = -1 (case 3),
minus the mean column and minus the column most correlated with all others (Section 5's
choices), then the least-squares solution of A^T t = -1 (case 1, n <= m).  Each test builds
a matrix on which the earlier candidates fail, checks with the oracle's choose_translation
which candidate is the first interior one, and then that the GPU picked the same one and
solves to the certified optimum with safe screens.
"""
import numpy as np
import pytest

import oracle as O

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


def heavy_rows(seed, m=60, n=90):
    """|N(0,1)| entries, six rows scaled up, the first three columns shifted down: their
    sums turn negative (t = -1 fails) while their correlation with the column sum may stay
    positive."""
    rng = np.random.default_rng(seed)
    w = np.ones(m)
    w[:6] = rng.uniform(5, 15)
    A = np.abs(rng.standard_normal((m, n))) * w[:, None]
    A[:, :3] -= rng.uniform(1.5, 4.0)
    return A


def oracle_choice(A):
    u = np.full(A.shape[1], np.inf)
    t = O.choose_translation(A, u)
    m, n = A.shape
    s = A.sum(axis=1)
    for k, c in enumerate([-np.ones(m), -s / n, -A[:, int(np.argmax(A.T @ s))]]):
        if np.allclose(t, c):
            return k + 1, t
    return 4, t


CASES = {
    "minus_mean_column": lambda: heavy_rows(0),
    "minus_most_correlated_column": lambda: heavy_rows(20),
    "least_squares_case1": lambda: np.random.default_rng(3).standard_normal((120, 50)),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_direction_candidates_match_the_oracle(P, name):
    A = CASES[name]()
    m, n = A.shape
    choice, t = oracle_choice(A)
    assert choice == {"minus_mean_column": 2, "minus_most_correlated_column": 3, "least_squares_case1": 4}[name]
    rng = np.random.default_rng(7)
    x0 = np.where(rng.random(n) < 0.15, rng.uniform(0, 1, n), 0.0)
    y = A @ x0 + rng.standard_normal(m)
    A32, y32 = A.astype(np.float32), y.astype(np.float32)
    A64, y64 = A32.astype(np.float64), y32.astype(np.float64)
    l, u = np.zeros(n), np.full(n, np.inf)
    L = 1.05 * float(np.linalg.norm(A64, 2) ** 2)
    dev = torch.device("cuda:0")
    s = P.Solver(torch.from_numpy(A32).to(dev), l, u)
    x, scr, info, st = s.solve(torch.from_numpy(y32).to(dev), tol=1e-8, lipschitz=L, refine=True)
    torch.cuda.synchronize()
    s.close()
    assert info["t_choice"] == choice and info["dual"] == "translation"
    assert st == P.BVLS_OK and info["gap"] < 1e-8
    # the oracle's own rounding floor of the translated gap lies near 1e-9 on these
    # unnormalised matrices; its polished optimum is certified by the optimality conditions
    ref = O.solve(A64, y64, l, u, tol=1e-8, L=L)
    assert ref.converged and ref.dual_mode == "translation"
    x, scr = x.cpu().numpy(), scr.cpu().numpy()
    xs = O.polish(A64, y64, ref.x, l, u, tau=1e-7)
    assert O.kkt_residual(A64, y64, xs, l, u) < 1e-9 * (1 + np.abs(A64.T @ y64).max())
    g = A64.T @ (y64 - A64 @ xs)
    low = scr == 1
    assert low.sum() > 0
    assert np.all(xs[low] == 0.0) and np.all(g[low] < 0)
    if info["refined"]:
        assert float(np.abs(x - xs).max()) <= 1e-7 * max(1.0, float(np.abs(xs).max()))
    assert O.primal_objective(A64, y64, x) - O.primal_objective(A64, y64, xs) <= 1e-8 * 1.01 + 1e-12
