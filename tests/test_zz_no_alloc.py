"""bvls_solve_static -- the entry point for callers that cannot allocate device memory.

Some callers run where cudaMalloc is off limits (in a memory pool or allocator they do not
own, or under a host application that fixes its allocations at start-up).
bvls_solve_static serves them from a static device array.  These tests call it
through the C ABI twice in a row (the array keeps the previous call's contents, so the
second call checks that everything that must start at zero is cleared) and compare it with
bvls_setup + bvls_solve.  The file sorts last so that a run stopping at the first failure has
already run every other test.
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


def _padded_device_A(A, lda):
    """Column-major device copy with leading dimension lda; rows m..lda-1 are zero."""
    m, n = A.shape
    buf = torch.zeros(n, lda, dtype=torch.float32, device="cuda")
    buf[:, :m] = torch.from_numpy(np.ascontiguousarray(A.T))
    return buf


@pytest.mark.parametrize("make", [lambda: W.nnls_abs_gaussian(250, 700, 0.05, 1.0, 3),
                                  lambda: W.bvls_table2(190, 480, 6)])
def test_static_matches_handle_path_twice(P, make):
    from paper_2202_07258_gb300 import _capi
    p = make()
    m, n = p.m, p.n
    lda = (m + 31) // 32 * 32
    A64 = p.A.astype(np.float64)
    L = 1.05 * float(np.linalg.norm(A64, 2) ** 2)
    opts = P.make_opts(tol=1e-8, screen_every=10, lipschitz=L)
    l = np.ascontiguousarray(p.l)
    u = np.ascontiguousarray(p.u)
    y = torch.from_numpy(p.y).cuda()

    solver = P.Solver(torch.from_numpy(p.A).cuda(), p.l, p.u)
    x_ref, s_ref, info_ref, st_ref = solver.solve(y, opts=opts)
    torch.cuda.synchronize()
    solver.close()
    assert st_ref == P.BVLS_OK
    x_ref = x_ref.cpu().numpy()

    A_dev = _padded_device_A(p.A, lda)
    for call in range(2):
        x = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
        s = torch.full((n,), 255, dtype=torch.uint8, device="cuda")
        st, info = _capi.bvls_solve_static(A_dev.data_ptr(), m, n, lda, l.ctypes.data, u.ctypes.data,
                                           y.data_ptr(), None, opts, 0, x.data_ptr(), s.data_ptr())
        torch.cuda.synchronize()
        assert st == P.BVLS_OK, (call, _capi.bvls_last_error())
        assert info.converged and info.gap < 1e-8
        xs = x.cpu().numpy()
        scale = max(1.0, float(np.abs(x_ref).max()))
        assert float(np.abs(xs - x_ref).max()) <= 1e-9 * scale, call
        assert abs(info.iters - info_ref["iters"]) <= 10
        assert np.array_equal(s.cpu().numpy() > 0, s_ref.cpu().numpy() > 0) or \
            abs(int((s.cpu().numpy() > 0).sum()) - int((s_ref.cpu().numpy() > 0).sum())) <= 2


def test_static_default_step_constant_and_wide_lda(P):
    """opts.lipschitz = 0: the call estimates L itself (power steps on the static scratch);
    a leading dimension 32 rows beyond the padding changes the pass's tiling and stage
    layout.  The handle path then runs with the same L and must agree."""
    from paper_2202_07258_gb300 import _capi
    p = W.nnls_abs_gaussian(230, 610, 0.05, 1.0, 11)
    m, n = p.m, p.n
    lda = (m + 31) // 32 * 32 + 32
    A64 = p.A.astype(np.float64)
    normA2 = float(np.linalg.norm(A64, 2) ** 2)
    l = np.ascontiguousarray(p.l)
    u = np.ascontiguousarray(p.u)
    y = torch.from_numpy(p.y).cuda()
    A_dev = _padded_device_A(p.A, lda)
    opts0 = P.make_opts(tol=1e-8, screen_every=10)
    solver = P.Solver(torch.from_numpy(p.A).cuda(), p.l, p.u)
    Ls = []
    for call in range(2):
        x = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
        st, info = _capi.bvls_solve_static(A_dev.data_ptr(), m, n, lda, l.ctypes.data, u.ctypes.data,
                                           y.data_ptr(), None, opts0, 0, x.data_ptr(), None)
        torch.cuda.synchronize()
        assert st == P.BVLS_OK, (call, _capi.bvls_last_error())
        assert info.L >= normA2, (info.L, normA2)
        assert info.L <= 1.06 * normA2
        Ls.append(info.L)
        # the power steps sum with atomics, so L may differ in its last digits between
        # calls: the handle path runs with this call's own L
        x_ref, _, _, st_ref = solver.solve(y, opts=P.make_opts(tol=1e-8, screen_every=10, lipschitz=info.L))
        torch.cuda.synchronize()
        assert st_ref == P.BVLS_OK
        x_ref = x_ref.cpu().numpy()
        scale = max(1.0, float(np.abs(x_ref).max()))
        assert float(np.abs(x.cpu().numpy() - x_ref).max()) <= 1e-9 * scale, call
    solver.close()
    assert abs(Ls[0] - Ls[1]) <= 1e-6 * Ls[0]


def test_static_rejects_what_it_cannot_hold(P):
    from paper_2202_07258_gb300 import _capi
    A = torch.zeros(8, 64, dtype=torch.float32, device="cuda")   # lda = 64 columns of length 64
    y = torch.zeros(40, dtype=torch.float32, device="cuda")
    x = torch.empty(8, dtype=torch.float64, device="cuda")
    st, _ = _capi.bvls_solve_static(A.data_ptr(), 40, 8, 40, None, None, y.data_ptr(), None, None, 0,
                                    x.data_ptr(), None)
    assert st == P.BVLS_EINVAL and "multiple of 32" in _capi.bvls_last_error()
    st, _ = _capi.bvls_solve_static(A.data_ptr(), 5000, 8, 5024, None, None, y.data_ptr(), None, None, 0,
                                    x.data_ptr(), None)
    assert st == _capi.BVLS_ENOTSUP and "4096" in _capi.bvls_last_error()
    A = torch.zeros(8, 64, dtype=torch.float32, device="cuda")
    st, _ = _capi.bvls_solve_static(A.data_ptr(), 40, 8, 64, None, None, y.data_ptr(), None,
                                    P.make_opts(algorithm="cp"), 0, x.data_ptr(), None)
    assert st == _capi.BVLS_ENOTSUP and "FISTA" in _capi.bvls_last_error()
    o = P.make_opts()
    o.single_pass = 3
    st, _ = _capi.bvls_solve_static(A.data_ptr(), 40, 8, 64, None, None, y.data_ptr(), None, o, 0,
                                    x.data_ptr(), None)
    assert st == P.BVLS_EINVAL
