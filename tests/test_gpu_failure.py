"""Failure detection on the GPU without a GPU fault: a bounded device wait that runs out.

The persistent pass of bvls_solve synchronises its CTAs with grid barriers whose waits are
bounded (about 2 s by default).  bvls_set_grid_wait lowers that bound to a few cycles, so a
CTA that reaches a barrier before the others gives up at once: it records the error, the CTAs
leave their loops at their next barrier once the copies they issued have landed, and the call
returns BVLS_ETIMEOUT without touching its outputs.  Restoring the bound, the same handle
solves again and matches a fresh solve bit for bit.  Nothing here faults, traps or hangs: every
wait stays bounded and the kernel returns a status the host reads.
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


@pytest.mark.parametrize("profile", [0, 2])
def test_grid_barrier_timeout_is_reported_and_the_handle_recovers(P, profile):
    from paper_2202_07258_gb300 import _capi
    p = W.nnls_abs_gaussian(600, 3000, 0.05, 1.0, 7)
    dev = torch.device("cuda:0")
    s = P.Solver(torch.from_numpy(p.A).to(dev), p.l, p.u)
    y = torch.from_numpy(p.y).to(dev)
    ref_x, ref_s, ref_info, ref_st = s.solve(y, tol=1e-7, profile=profile)
    torch.cuda.synchronize()
    assert ref_st == P.BVLS_OK and ref_info["single_pass"] == 2      # the persistent form ran
    assert _capi.bvls_set_grid_wait(s.handle, 1) == P.BVLS_OK
    x = torch.full((p.n,), 12345.0, dtype=torch.float64, device=dev)
    scr = torch.full((p.n,), 77, dtype=torch.uint8, device=dev)
    x, scr, info, st = s.solve(y, tol=1e-7, profile=profile, x_out=x, screened_out=scr, check=False)
    torch.cuda.synchronize()
    assert st == _capi.BVLS_ETIMEOUT, (st, _capi.bvls_last_error())
    assert "wait" in _capi.bvls_last_error()
    assert bool(torch.all(x == 12345.0)) and bool(torch.all(scr == 77))   # outputs untouched
    assert _capi.bvls_set_grid_wait(s.handle, 0) == P.BVLS_OK
    x2, s2, info2, st2 = s.solve(y, tol=1e-7, profile=profile)
    torch.cuda.synchronize()
    assert st2 == P.BVLS_OK and info2["iters"] == ref_info["iters"]
    assert torch.equal(x2, ref_x) and torch.equal(s2, ref_s)
    s.close()
