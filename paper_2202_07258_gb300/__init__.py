"""GB300 (sm_103a) solver for box-constrained least squares with dynamic Gap safe screening.

    x* in argmin 1/2 ||y - A x||^2  s.t.  l <= x <= u      (NNLS: l = 0, u = +inf; BVLS)

Dantas, Soubies and Fevotte, "Accelerating Non-Negative and Bounded-Variable Linear
Regression Algorithms with Safe Screening": accelerated projected gradient with the
screening of Algorithm 1 fused into the CUDA kernels of the C ABI (include/bvls_gb300.h).

``_capi`` holds the C entry points under their C names; ``Solver`` marshals numpy arrays
or torch tensors into them.  Nothing here computes: every step runs in the CUDA kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _capi
from ._capi import (BVLS_DUAL_SCALING, BVLS_DUAL_TRANSLATION, BVLS_DUAL_ZERO, BVLS_EINVAL,
                    BVLS_EMAXITER, BVLS_ENONFINITE, BVLS_ENOTSUP, BVLS_OK, BVLS_PREC_FP32, BVLS_PREC_MIXED,
                    BVLS_PREC_FP32X2, DUAL_NAMES, STATUS_NAMES, bvls_default_opts, bvls_destroy,
                    bvls_backward, bvls_backward_default_opts, bvls_backward_info, bvls_backward_opts,
                    bvls_batch_info, bvls_info, bvls_last_error, bvls_opts, bvls_setup, bvls_solve,
                    bvls_solve_batched)

__all__ = ["Solver", "BVLSError", "bvls_setup", "bvls_solve", "bvls_destroy", "bvls_default_opts",
           "bvls_last_error", "bvls_opts", "bvls_info", "bvls_batch_info", "bvls_solve_batched", "make_opts",
           "bvls_backward", "bvls_backward_opts", "bvls_backward_info", "solve_batched_autograd",
           "solve_ragged"]


class BVLSError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _is_torch(x) -> bool:
    try:
        import torch
    except ImportError:  # pragma: no cover
        return False
    return isinstance(x, torch.Tensor)


def _host_f64(v, n):
    if v is None:
        return None
    return np.ascontiguousarray(np.broadcast_to(np.asarray(v, dtype=np.float64), (n,)))


def make_opts(tol=1e-6, screen_every=10, max_iter=100000, screening=True, precision="fp32x2",
              restart=True, lipschitz=0.0, profile=False, single_pass=True, algorithm="fista",
              refine=False) -> bvls_opts:
    o = bvls_default_opts()
    o.tol = float(tol)
    o.screen_every = int(screen_every)
    o.max_iter = int(max_iter)
    o.screening = 1 if screening else 0
    o.precision = {"fp32x2": BVLS_PREC_FP32X2, "fp32": BVLS_PREC_FP32, "mixed": BVLS_PREC_MIXED}[precision]
    o.restart = 1 if restart else 0
    o.lipschitz = float(lipschitz)
    o.profile = int(profile)            # 0 graphs, 1 event-timed chunk graph, 2 direct launches
    o.single_pass = int(single_pass)   # 0 two passes, 1 single pass (persistent), 2 single pass, two launches
    o.algorithm = {"fista": _capi.BVLS_ALG_FISTA, "cp": _capi.BVLS_ALG_CHAMBOLLE_POCK,
                   "chambolle_pock": _capi.BVLS_ALG_CHAMBOLLE_POCK}[algorithm]
    o.refine = 1 if refine else 0
    return o


class Solver:
    """One handle of the C ABI: the matrix A, the box [l, u] and the device workspace.

    A is (m, n): a torch tensor (any device) or a numpy array.  l, u are scalars or length-n
    arrays (u may hold inf); t optionally gives the translation direction (length m).
    """

    def __init__(self, A, l=None, u=None, t=None, stream=None):
        if _is_torch(A):
            import torch
            m, n = A.shape
            At = A.detach().to(dtype=torch.float32).t().contiguous()   # column-major A
            self._A_keep = At
            a_ptr = At.data_ptr()
            if stream is None and At.is_cuda:
                stream = torch.cuda.current_stream(At.device).cuda_stream
        else:
            A = np.asarray(A)
            m, n = A.shape
            Af = np.asfortranarray(A, dtype=np.float32)
            self._A_keep = Af
            a_ptr = Af.ctypes.data
        self.m, self.n = int(m), int(n)
        l_h, u_h = _host_f64(l, self.n), _host_f64(u, self.n)
        t_h = None if t is None else np.ascontiguousarray(np.asarray(t, dtype=np.float64).reshape(self.m))
        st, h = bvls_setup(a_ptr, self.m, self.n, self.m,
                           None if l_h is None else l_h.ctypes.data,
                           None if u_h is None else u_h.ctypes.data,
                           None if t_h is None else t_h.ctypes.data, stream)
        self._A_keep = None
        if st != BVLS_OK:
            raise BVLSError(st, bvls_last_error())
        self.handle = h

    def close(self):
        bvls_destroy(getattr(self, "handle", None))
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, y, x0=None, *, opts: bvls_opts | None = None, x_out=None, screened_out=None,
              check: bool = True, **kw):
        """Run bvls_solve.  Returns (x, screened, info_dict, status).

        Outputs follow y: a CUDA tensor y gives CUDA tensors (float64 x, uint8 screened),
        a numpy y gives numpy arrays.  ``kw`` builds the options (see ``make_opts``).
        With check=True a status other than OK / EMAXITER raises BVLSError.
        """
        dual_point = kw.pop("dual_point", None)
        if opts is None:
            opts = make_opts(**kw)
        keep = None
        if dual_point is not None:
            # a fixed dual point for every screening step (the oracle-dual-point experiment)
            if _is_torch(dual_point):
                import torch
                keep = dual_point.detach().to(dtype=torch.float64).contiguous()
                opts.dual_point = keep.data_ptr()
            else:
                keep = np.ascontiguousarray(np.asarray(dual_point, dtype=np.float64).reshape(self.m))
                opts.dual_point = keep.ctypes.data
        if _is_torch(y):
            import torch
            dev = y.device
            yk = y.detach().to(dtype=torch.float32).contiguous()
            x0k = None if x0 is None else x0.detach().to(device=dev, dtype=torch.float64).contiguous()
            x = x_out if x_out is not None else torch.empty(self.n, dtype=torch.float64, device=dev)
            s = screened_out if screened_out is not None else torch.empty(self.n, dtype=torch.uint8, device=dev)
            ptrs = (yk.data_ptr(), None if x0k is None else x0k.data_ptr(), x.data_ptr(), s.data_ptr())
        else:
            yk = np.ascontiguousarray(np.asarray(y, dtype=np.float32).reshape(self.m))
            x0k = None if x0 is None else np.ascontiguousarray(np.asarray(x0, dtype=np.float64).reshape(self.n))
            x = x_out if x_out is not None else np.empty(self.n, dtype=np.float64)
            s = screened_out if screened_out is not None else np.empty(self.n, dtype=np.uint8)
            ptrs = (yk.ctypes.data, None if x0k is None else x0k.ctypes.data, x.ctypes.data, s.ctypes.data)
        st, info = bvls_solve(self.handle, ptrs[0], ptrs[1], opts, ptrs[2], ptrs[3])
        del keep
        if check and st not in (BVLS_OK, BVLS_EMAXITER):
            raise BVLSError(st, bvls_last_error())
        d = info.as_dict()
        d["status"] = STATUS_NAMES.get(st, st)
        d["dual"] = DUAL_NAMES.get(info.dual_mode, info.dual_mode)
        return x, s, d, st

    def solve_batched(self, Y, X0=None, *, opts: bvls_opts | None = None, check: bool = True, **kw):
        """Run bvls_solve_batched on the rows of Y (B x m).

        Returns (X, screened, gaps, iters, status, info_dict, st): X (B x n float64),
        screened (B x n uint8), per-instance gap bounds, iteration indices and statuses.
        Outputs follow Y (CUDA tensors for a CUDA tensor Y, numpy arrays otherwise).
        """
        if opts is None:
            opts = make_opts(**kw)
        if _is_torch(Y):
            import torch
            dev = Y.device
            Yk = Y.detach().to(dtype=torch.float32).contiguous()
            B = int(Yk.shape[0])
            X0k = None if X0 is None else X0.detach().to(device=dev, dtype=torch.float64).contiguous()
            X = torch.empty((B, self.n), dtype=torch.float64, device=dev)
            S = torch.empty((B, self.n), dtype=torch.uint8, device=dev)
            gaps = torch.empty(B, dtype=torch.float64, device=dev)
            its = torch.empty(B, dtype=torch.int32, device=dev)
            sts = torch.empty(B, dtype=torch.int32, device=dev)
            ptr = lambda t: None if t is None else t.data_ptr()
        else:
            Yk = np.ascontiguousarray(np.asarray(Y, dtype=np.float32).reshape(-1, self.m))
            B = int(Yk.shape[0])
            X0k = None if X0 is None else np.ascontiguousarray(np.asarray(X0, dtype=np.float64).reshape(B, self.n))
            X = np.empty((B, self.n), dtype=np.float64)
            S = np.empty((B, self.n), dtype=np.uint8)
            gaps = np.empty(B, dtype=np.float64)
            its = np.empty(B, dtype=np.int32)
            sts = np.empty(B, dtype=np.int32)
            ptr = lambda t: None if t is None else t.ctypes.data
        st, info = bvls_solve_batched(self.handle, B, ptr(Yk), self.m, ptr(X0k), opts, ptr(X), ptr(S), ptr(gaps),
                                      ptr(its), ptr(sts))
        if check and st not in (BVLS_OK, BVLS_EMAXITER):
            raise BVLSError(st, bvls_last_error())
        d = info.as_dict()
        d["status"] = STATUS_NAMES.get(st, st)
        d["dual"] = DUAL_NAMES.get(info.dual_mode, info.dual_mode)
        return X, S, gaps, its, sts, d, st

    def backward(self, X, Y, dLdX, *, want_dA: bool = True, free_tol: float = 1e-9, cg_tol: float = 1e-12,
                 cg_max_iter: int = 4000, check: bool = True):
        """Run bvls_backward: gradients of L(x*) through the solution map.

        X (B x n solutions), Y (B x m right-hand sides) and dLdX (B x n) as CUDA tensors or
        numpy arrays.  Returns (dLdY (B x m), dLdA (m x n, summed over the batch, or None),
        status (B), info_dict), following the type of X.
        """
        o = bvls_backward_default_opts()
        o.free_tol, o.cg_tol, o.cg_max_iter = float(free_tol), float(cg_tol), int(cg_max_iter)
        if _is_torch(X):
            import torch
            dev = X.device
            Xk = X.detach().to(dtype=torch.float64).contiguous()
            B = int(Xk.shape[0])
            Yk = Y.detach().to(device=dev, dtype=torch.float32).contiguous()
            Vk = dLdX.detach().to(device=dev, dtype=torch.float64).contiguous()
            dY = torch.empty((B, self.m), dtype=torch.float64, device=dev)
            dA = torch.empty((self.n, self.m), dtype=torch.float64, device=dev) if want_dA else None
            sts = torch.empty(B, dtype=torch.int32, device=dev)
            ptr = lambda t: None if t is None else t.data_ptr()
        else:
            Xk = np.ascontiguousarray(np.asarray(X, dtype=np.float64).reshape(-1, self.n))
            B = int(Xk.shape[0])
            Yk = np.ascontiguousarray(np.asarray(Y, dtype=np.float32).reshape(B, self.m))
            Vk = np.ascontiguousarray(np.asarray(dLdX, dtype=np.float64).reshape(B, self.n))
            dY = np.empty((B, self.m), dtype=np.float64)
            dA = np.empty((self.n, self.m), dtype=np.float64) if want_dA else None
            sts = np.empty(B, dtype=np.int32)
            ptr = lambda t: None if t is None else t.ctypes.data
        st, info = bvls_backward(self.handle, B, ptr(Xk), ptr(Yk), self.m, ptr(Vk), o, ptr(dY), ptr(dA), ptr(sts))
        if check and st != BVLS_OK:
            raise BVLSError(st, bvls_last_error())
        # the C ABI writes dL/dA column-major (m x n): as a row-major (n x m) array, transpose
        return dY, (dA.T if dA is not None else None), sts, info.as_dict()


def _autograd_function():
    import torch

    class _SolveBatched(torch.autograd.Function):
        """x* = argmin_{l <= x <= u} 1/2 ||y_b - A x||^2 for every row y_b of Y, with gradients
        to A and Y from the free-set normal equations (bvls_backward)."""

        @staticmethod
        def forward(ctx, A, Y, l, u, opts_kw):
            solver = Solver(A.detach(), l, u)
            X, S, gaps, its, sts, info, st = solver.solve_batched(Y.detach(), **opts_kw)
            ctx.solver = solver
            ctx.save_for_backward(X, Y.detach())
            ctx.mark_non_differentiable(S)
            return X, S

        @staticmethod
        def backward(ctx, dX, dS):
            X, Y = ctx.saved_tensors
            solver = ctx.solver
            want_dA = ctx.needs_input_grad[0]
            dY, dA, sts, info = solver.backward(X, Y, dX, want_dA=want_dA)
            solver.close()
            ctx.solver = None
            gA = dA.to(dtype=torch.float32) if want_dA else None
            gY = dY.to(dtype=Y.dtype) if ctx.needs_input_grad[1] else None
            return gA, gY, None, None, None

    return _SolveBatched


_FN = None


def solve_batched_autograd(A, Y, l=None, u=None, **opts_kw):
    """Differentiable batched solve: returns (X, screened) with X (B x n, float64) carrying
    gradients to A (m x n) and Y (B x m) through the solution map."""
    global _FN
    if _FN is None:
        _FN = _autograd_function()
    return _FN.apply(A, Y, l, u, opts_kw)


def solve_ragged(problems, *, opts: bvls_opts | None = None, stream=None, check: bool = True, **kw):
    """bvls_solve_ragged on a list of (A, y, l, u) with A (m_k x n_k) and y (m_k) as numpy
    arrays or CUDA tensors and l, u as None, scalars or length-n_k arrays (host).

    Returns (xs, screened, gaps, iters, statuses, info_dict, status): per-instance numpy
    arrays x (float64) and screened flags (uint8), and per-instance gaps, iteration counts
    and statuses.
    """
    if opts is None:
        opts = make_opts(**kw)
    keep, descs, xs, ss = [], [], [], []
    for A, y, l, u in problems:
        if _is_torch(A):
            import torch
            At = A.detach().to(dtype=torch.float32).t().contiguous()   # column-major
            yt = y.detach().to(device=A.device, dtype=torch.float32).contiguous()
            a_ptr, y_ptr = At.data_ptr(), yt.data_ptr()
            m, n = int(A.shape[0]), int(A.shape[1])
        else:
            At = np.asfortranarray(np.asarray(A, dtype=np.float32))
            yt = np.ascontiguousarray(np.asarray(y, dtype=np.float32).reshape(-1))
            a_ptr, y_ptr = At.ctypes.data, yt.ctypes.data
            m, n = At.shape
        lh, uh = _host_f64(l, n), _host_f64(u, n)
        keep += [At, yt, lh, uh]
        x = np.empty(n, dtype=np.float64)
        sc = np.empty(n, dtype=np.uint8)
        xs.append(x)
        ss.append(sc)
        descs.append(_capi.bvls_problem(a_ptr, m, n, m, y_ptr, None if lh is None else lh.ctypes.data,
                                        None if uh is None else uh.ctypes.data))
    B = len(descs)
    gaps = np.empty(B, dtype=np.float64)
    its = np.empty(B, dtype=np.int32)
    sts = np.empty(B, dtype=np.int32)
    st, info = _capi.bvls_solve_ragged(descs, opts, stream, [x.ctypes.data for x in xs],
                                       [s.ctypes.data for s in ss], gaps.ctypes.data, its.ctypes.data,
                                       sts.ctypes.data)
    del keep
    if check and st not in (BVLS_OK, BVLS_EMAXITER):
        raise BVLSError(st, bvls_last_error())
    return xs, ss, gaps, its, sts, info.as_dict(), st

