"""ctypes binding of the C ABI declared in include/bvls_gb300.h (argument marshalling only).

The functions keep the C names.  Pointers are passed as integers (device pointers from
torch tensors, or host addresses from numpy arrays); the CUDA path does all the work.
Loading fails loudly when the extension is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbvls_gb300.so")

BVLS_OK, BVLS_EINVAL, BVLS_ENOMEM, BVLS_ECUDA, BVLS_EMAXITER, BVLS_ENONFINITE, BVLS_ENOTSUP, BVLS_ETIMEOUT = range(8)
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EMAXITER", 5: "ENONFINITE", 6: "ENOTSUP",
                7: "ETIMEOUT"}
BVLS_PREC_FP32X2, BVLS_PREC_FP32, BVLS_PREC_MIXED = 0, 1, 2
BVLS_ALG_FISTA, BVLS_ALG_CHAMBOLLE_POCK = 0, 1
BVLS_DUAL_SCALING, BVLS_DUAL_TRANSLATION, BVLS_DUAL_ZERO = 0, 1, 2
DUAL_NAMES = {0: "scaling", 1: "translation", 2: "zero"}

# Every symbol the header declares; tests check that the library exports all of them.
EXPORTED = ("bvls_default_opts", "bvls_setup", "bvls_solve", "bvls_destroy", "bvls_last_error",
            "bvls_solve_static", "bvls_solve_batched", "bvls_backward_default_opts", "bvls_backward",
            "bvls_solve_ragged", "bvls_set_grid_wait")


class bvls_opts(ctypes.Structure):
    _fields_ = [
        ("tol", ctypes.c_double),
        ("screen_every", ctypes.c_int),
        ("max_iter", ctypes.c_int),
        ("screening", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("restart", ctypes.c_int),
        ("lipschitz", ctypes.c_double),
        ("profile", ctypes.c_int),
        ("single_pass", ctypes.c_int),
        ("dual_point", ctypes.c_void_p),
        ("algorithm", ctypes.c_int),
        ("refine", ctypes.c_int),
    ]


class bvls_info(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int),
        ("converged", ctypes.c_int),
        ("n_preserved", ctypes.c_int),
        ("dual_mode", ctypes.c_int),
        ("gap_evals", ctypes.c_int),
        ("gap", ctypes.c_double),
        ("primal", ctypes.c_double),
        ("radius", ctypes.c_double),
        ("L", ctypes.c_double),
        ("sum_preserved", ctypes.c_double),
        ("sum_nonzero", ctypes.c_double),
        ("fwd_ms", ctypes.c_double),
        ("tr_ms", ctypes.c_double),
        ("fwd_launches", ctypes.c_int),
        ("tr_launches", ctypes.c_int),
        ("kernel_launches", ctypes.c_double),
        ("single_pass", ctypes.c_int),
        ("refined", ctypes.c_int),
        ("refine_rounds", ctypes.c_int),
        ("n_free", ctypes.c_int),
        ("refine_cg_iters", ctypes.c_int),
        ("kkt", ctypes.c_double),
        ("refine_ms", ctypes.c_double),
        ("refine_reason", ctypes.c_int),
        ("t_choice", ctypes.c_int),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class bvls_batch_info(ctypes.Structure):
    _fields_ = [
        ("iters_max", ctypes.c_int),
        ("n_converged", ctypes.c_int),
        ("gap_evals", ctypes.c_int),
        ("dual_mode", ctypes.c_int),
        ("L", ctypes.c_double),
        ("sum_step", ctypes.c_double),
        ("sum_eval", ctypes.c_double),
        ("sum_preserved", ctypes.c_double),
        ("step_ms", ctypes.c_double),
        ("eval_ms", ctypes.c_double),
        ("step_launches", ctypes.c_int),
        ("eval_launches", ctypes.c_int),
        ("kernel_launches", ctypes.c_double),
        ("n_refined", ctypes.c_int),
        ("refine_free_max", ctypes.c_int),
        ("kkt_max", ctypes.c_double),
        ("refine_ms", ctypes.c_double),
        ("refine_out_of_rounds", ctypes.c_int),
        ("refine_not_unique", ctypes.c_int),
        ("steps_persistent", ctypes.c_int),
        ("pad0", ctypes.c_int),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class bvls_backward_opts(ctypes.Structure):
    _fields_ = [
        ("free_tol", ctypes.c_double),
        ("cg_tol", ctypes.c_double),
        ("cg_max_iter", ctypes.c_int),
    ]


class bvls_backward_info(ctypes.Structure):
    _fields_ = [
        ("n_converged", ctypes.c_int),
        ("n_iter_limit", ctypes.c_int),
        ("n_too_large", ctypes.c_int),
        ("n_not_unique", ctypes.c_int),
        ("max_free", ctypes.c_int),
        ("max_cg_iters", ctypes.c_int),
        ("cg_work", ctypes.c_double),
        ("kernel_ms", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class bvls_problem(ctypes.Structure):
    _fields_ = [
        ("A", ctypes.c_void_p),
        ("m", ctypes.c_int),
        ("n", ctypes.c_int),
        ("lda", ctypes.c_int),
        ("y", ctypes.c_void_p),
        ("l", ctypes.c_void_p),
        ("u", ctypes.c_void_p),
    ]


class bvls_ragged_info(ctypes.Structure):
    _fields_ = [
        ("iters_max", ctypes.c_int),
        ("n_converged", ctypes.c_int),
        ("n_translation", ctypes.c_int),
        ("n_zero", ctypes.c_int),
        ("chunks", ctypes.c_int),
        ("tiles_max", ctypes.c_int),
        ("setup_ms", ctypes.c_double),
        ("solve_ms", ctypes.c_double),
        ("tile_cols", ctypes.c_int),
        ("screen_every", ctypes.c_int),
        ("tuned", ctypes.c_int),
        ("tune_ms", ctypes.c_double),
        ("n_refined", ctypes.c_int),
        ("refine_free_max", ctypes.c_int),
        ("kkt_max", ctypes.c_double),
        ("refine_ms", ctypes.c_double),
        ("refine_out_of_rounds", ctypes.c_int),
        ("refine_not_unique", ctypes.c_int),
        ("sum_rows_cols", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the extension (once).  Raises ImportError if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"CUDA extension not built: {path} is missing "
                          "(run `python -c 'import __graft_entry__ as g; g.build()'`)")
    lib = ctypes.CDLL(path)
    vp, ci, cd = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.bvls_default_opts.argtypes = [ctypes.POINTER(bvls_opts)]
    lib.bvls_default_opts.restype = None
    lib.bvls_setup.argtypes = [vp, ci, ci, ci, vp, vp, vp, vp, ctypes.POINTER(vp)]
    lib.bvls_setup.restype = ci
    lib.bvls_solve.argtypes = [vp, vp, vp, ctypes.POINTER(bvls_opts), vp, vp, ctypes.POINTER(bvls_info)]
    lib.bvls_solve.restype = ci
    lib.bvls_destroy.argtypes = [vp]
    lib.bvls_destroy.restype = None
    lib.bvls_last_error.argtypes = []
    lib.bvls_last_error.restype = ctypes.c_char_p
    lib.bvls_solve_static.argtypes = [vp, ci, ci, ci, vp, vp, vp, vp, ctypes.POINTER(bvls_opts), vp, vp, vp,
                                      ctypes.POINTER(bvls_info)]
    lib.bvls_solve_static.restype = ci
    lib.bvls_solve_batched.argtypes = [vp, ci, vp, ci, vp, ctypes.POINTER(bvls_opts), vp, vp, vp, vp, vp,
                                       ctypes.POINTER(bvls_batch_info)]
    lib.bvls_solve_batched.restype = ci
    lib.bvls_backward_default_opts.argtypes = [ctypes.POINTER(bvls_backward_opts)]
    lib.bvls_backward_default_opts.restype = None
    lib.bvls_backward.argtypes = [vp, ci, vp, vp, ci, vp, ctypes.POINTER(bvls_backward_opts), vp, vp, vp,
                                  ctypes.POINTER(bvls_backward_info)]
    lib.bvls_backward.restype = ci
    lib.bvls_solve_ragged.argtypes = [ci, ctypes.POINTER(bvls_problem), ctypes.POINTER(bvls_opts), vp,
                                      ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p), vp, vp, vp,
                                      ctypes.POINTER(bvls_ragged_info)]
    lib.bvls_solve_ragged.restype = ci
    lib.bvls_set_grid_wait.argtypes = [vp, ctypes.c_longlong]
    lib.bvls_set_grid_wait.restype = ci
    _lib = lib
    return lib


def bvls_set_grid_wait(h: int, cycles: int) -> int:
    return load().bvls_set_grid_wait(h, int(cycles))


def bvls_default_opts() -> bvls_opts:
    o = bvls_opts()
    load().bvls_default_opts(ctypes.byref(o))
    return o


def bvls_last_error() -> str:
    return load().bvls_last_error().decode()


def bvls_setup(A_ptr: int, m: int, n: int, lda: int, l_ptr: int | None, u_ptr: int | None,
               t_ptr: int | None, stream: int | None) -> tuple[int, int | None]:
    h = ctypes.c_void_p()
    st = load().bvls_setup(A_ptr, m, n, lda, l_ptr, u_ptr, t_ptr, stream or 0, ctypes.byref(h))
    return st, h.value


def bvls_solve(h: int, y_ptr: int, x0_ptr: int | None, opts: bvls_opts | None, x_out_ptr: int,
               screened_ptr: int | None) -> tuple[int, bvls_info]:
    info = bvls_info()
    st = load().bvls_solve(h, y_ptr, x0_ptr, ctypes.byref(opts) if opts is not None else None,
                           x_out_ptr, screened_ptr, ctypes.byref(info))
    return st, info


def bvls_solve_static(A_ptr: int, m: int, n: int, lda: int, l_ptr: int | None, u_ptr: int | None,
                      y_ptr: int, x0_ptr: int | None, opts: bvls_opts | None, stream: int | None,
                      x_out_ptr: int, screened_ptr: int | None) -> tuple[int, bvls_info]:
    info = bvls_info()
    st = load().bvls_solve_static(A_ptr, m, n, lda, l_ptr, u_ptr, y_ptr, x0_ptr,
                                  ctypes.byref(opts) if opts is not None else None, stream or 0,
                                  x_out_ptr, screened_ptr, ctypes.byref(info))
    return st, info


def bvls_solve_batched(h: int, B: int, Y_ptr: int, ldy: int, X0_ptr: int | None, opts: bvls_opts | None,
                       X_out_ptr: int, screened_ptr: int | None, gaps_ptr: int | None, iters_ptr: int | None,
                       status_ptr: int | None) -> tuple[int, bvls_batch_info]:
    info = bvls_batch_info()
    st = load().bvls_solve_batched(h, B, Y_ptr, ldy, X0_ptr, ctypes.byref(opts) if opts is not None else None,
                                   X_out_ptr, screened_ptr, gaps_ptr, iters_ptr, status_ptr, ctypes.byref(info))
    return st, info


def bvls_backward_default_opts() -> bvls_backward_opts:
    o = bvls_backward_opts()
    load().bvls_backward_default_opts(ctypes.byref(o))
    return o


def bvls_backward(h: int, B: int, X_ptr: int, Y_ptr: int, ldy: int, dLdX_ptr: int,
                  opts: bvls_backward_opts | None, dLdY_ptr: int | None, dLdA_ptr: int | None,
                  status_ptr: int | None) -> tuple[int, bvls_backward_info]:
    info = bvls_backward_info()
    st = load().bvls_backward(h, B, X_ptr, Y_ptr, ldy, dLdX_ptr, ctypes.byref(opts) if opts is not None else None,
                              dLdY_ptr, dLdA_ptr, status_ptr, ctypes.byref(info))
    return st, info


def bvls_solve_ragged(probs, opts: bvls_opts | None, stream: int | None, x_ptrs, screened_ptrs, gaps_ptr,
                      iters_ptr, status_ptr) -> tuple[int, bvls_ragged_info]:
    B = len(probs)
    arr = (bvls_problem * B)(*probs)
    xp = (ctypes.c_void_p * B)(*x_ptrs)
    sp = (ctypes.c_void_p * B)(*screened_ptrs) if screened_ptrs is not None else None
    info = bvls_ragged_info()
    st = load().bvls_solve_ragged(B, arr, ctypes.byref(opts) if opts is not None else None, stream or 0, xp,
                                  sp, gaps_ptr, iters_ptr, status_ptr, ctypes.byref(info))
    return st, info


def bvls_destroy(h: int | None) -> None:
    if h:
        load().bvls_destroy(h)
