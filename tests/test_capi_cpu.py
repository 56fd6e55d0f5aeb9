"""CPU checks of the C ABI: the library builds, loads and exports every declared symbol.

No GPU is touched: only host-side argument validation paths are called.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2202_07258_gb300 import build, _capi
    build.build()
    return _capi.load()


def _declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            names |= set(re.findall(r"BVLS_API\s+[\w\s\*]+?\b(bvls_\w+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(lib):
    from paper_2202_07258_gb300 import _capi
    declared = _declared_symbols()
    assert declared, "no declarations found"
    assert declared == set(_capi.EXPORTED), (declared, _capi.EXPORTED)
    for name in declared:
        assert hasattr(lib, name), name


def test_default_opts_host_only(lib):
    from paper_2202_07258_gb300 import _capi
    o = _capi.bvls_default_opts()
    assert o.tol == 1e-6 and o.screen_every == 10 and o.screening == 1
    assert o.precision == _capi.BVLS_PREC_FP32X2 and o.restart == 1 and o.profile == 0


def test_enum_constants_match_header():
    """Every BVLS_* enumerator of the header has the same value in the Python binding."""
    from paper_2202_07258_gb300 import _capi
    txt = "".join(open(os.path.join(ROOT, "include", f)).read()
                  for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h"))
    consts = dict((k, int(v)) for k, v in re.findall(r"\b(BVLS_[A-Z0-9_]+)\s*=\s*(-?\d+)", txt))
    for k in ("BVLS_PREC_FP32X2", "BVLS_PREC_FP32", "BVLS_PREC_MIXED", "BVLS_ALG_FISTA",
              "BVLS_ALG_CHAMBOLLE_POCK", "BVLS_OK", "BVLS_EINVAL"):
        assert k in consts and getattr(_capi, k) == consts[k], k
    for k, v in consts.items():
        if hasattr(_capi, k):
            assert getattr(_capi, k) == v, k


def test_setup_rejects_bad_sizes_before_touching_the_device(lib):
    from paper_2202_07258_gb300 import _capi
    buf = (ctypes.c_float * 4)()
    st, h = _capi.bvls_setup(ctypes.addressof(buf), 0, 2, 2, None, None, None, 0)
    assert st == _capi.BVLS_EINVAL and h is None
    assert "m >= 1" in _capi.bvls_last_error()
    st, h = _capi.bvls_setup(ctypes.addressof(buf), 2, 2, 1, None, None, None, 0)
    assert st == _capi.BVLS_EINVAL
    st, h = _capi.bvls_setup(ctypes.addressof(buf), 30000, 2, 30000, None, None, None, 0)
    assert st == _capi.BVLS_ENOTSUP
    st, _ = _capi.bvls_solve(None, None, None, None, None, None)
    assert st == _capi.BVLS_EINVAL
    st, _ = _capi.bvls_solve_batched(None, 4, None, 2, None, None, None, None, None, None, None)
    assert st == _capi.BVLS_EINVAL
    st, _ = _capi.bvls_backward(None, 4, None, None, 2, None, None, None, None, None)
    assert st == _capi.BVLS_EINVAL
    o = _capi.bvls_backward_default_opts()
    assert o.free_tol == 1e-9 and o.cg_tol == 1e-12 and o.cg_max_iter == 4000
    st, _ = _capi.bvls_solve_ragged([], None, 0, [], None, None, None, None)
    assert st == _capi.BVLS_EINVAL
    bad = _capi.bvls_problem(ctypes.addressof(buf), 2000, 2, 2000, ctypes.addressof(buf), None, None)
    st, _ = _capi.bvls_solve_ragged([bad], None, 0, [ctypes.addressof(buf)], None, None, None, None)
    assert st == _capi.BVLS_ENOTSUP     # m above the ragged path's limit, rejected before any device work


def test_struct_layouts_match_header(tmp_path):
    """ctypes mirrors of bvls_opts / bvls_info / bvls_batch_info have the C compiler's sizes and offsets."""
    import shutil
    import subprocess
    from paper_2202_07258_gb300 import _capi
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    classes = {"bvls_opts": _capi.bvls_opts, "bvls_info": _capi.bvls_info,
               "bvls_batch_info": _capi.bvls_batch_info, "bvls_backward_opts": _capi.bvls_backward_opts,
               "bvls_backward_info": _capi.bvls_backward_info, "bvls_problem": _capi.bvls_problem,
               "bvls_ragged_info": _capi.bvls_ragged_info}
    fields = {k: [f for f, _ in c._fields_] for k, c in classes.items()}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "bvls_gb300.h"', "int main(void){"]
    for st, fl in fields.items():
        lines.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for f in fl:
            lines.append(f'printf("{st}.{f} %zu\\n", offsetof({st}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for st, cls in classes.items():
        assert int(out[st]) == ctypes.sizeof(cls), st
        for f in fields[st]:
            assert int(out[f"{st}.{f}"]) == getattr(cls, f).offset, (st, f)
