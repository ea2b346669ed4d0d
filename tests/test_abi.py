"""C-ABI checks that need no GPU: the library loads, exports every symbol that
include/rbicg.h declares, and rejects invalid arguments before touching the device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rbicg.h")
LIB = os.path.join(ROOT, "paper_1010_0762_gb300", "librbicg.so")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rbicg_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_1010_0762_gb300 import build
        build.build()
    return C.CDLL(LIB)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["rbicg_create", "rbicg_update_recycle", "rbicg_solve_pair", "rbicg_destroy",
              "rbicg_solve_batch", "rbicg_op_dual_spmv_project", "rbicg_op_gram", "rbicg_op_eig_select",
              "rbicg_op_svd", "rbicg_bilinear_form", "rbicg_irka", "rbicg_set_refresh"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_default_params_and_argument_errors(lib):
    from paper_1010_0762_gb300 import rbicg as R
    p = R.default_params()
    assert (p.k, p.s, p.max_itn, p.tol, p.svd_tol) == (10, 40, 20000, 1e-8, 1e-6)
    h = C.c_void_p()
    bad = R.default_params(k=0)
    assert R.lib.rbicg_create(C.byref(bad), 100, R.R64, None, C.byref(h)) == R.ERR_ARG
    bad = R.default_params(k=30, s=60)
    assert R.lib.rbicg_create(C.byref(bad), 100, R.R64, None, C.byref(h)) == R.ERR_ARG
    assert b"80" in R.lib.rbicg_last_error(None)
    assert R.lib.rbicg_create(C.byref(p), 0, R.R64, None, C.byref(h)) == R.ERR_ARG
    assert R.lib.rbicg_create(C.byref(p), 100, R.R64, None, C.byref(h)) == R.OK
    r = R.Result()
    # null vectors and a missing operator are argument errors (no device work)
    assert R.lib.rbicg_solve_pair(h, None, None, None, None, None, C.byref(r)) == R.ERR_ARG
    one = C.c_void_p(1)
    assert R.lib.rbicg_solve_pair(h, None, one, one, one, one, C.byref(r)) == R.ERR_ARG
    assert b"operator" in R.lib.rbicg_last_error(h)
    csr = R.CSRStruct()
    csr.n = 99
    assert R.lib.rbicg_update_recycle(h, C.byref(csr)) == R.ERR_ARG   # n mismatch
    assert R.lib.rbicg_destroy(h) == R.OK
    assert R.lib.rbicg_op_gram(R.R64, 10, None, 1, 1, None, 1, 1, 0, None, None) == R.ERR_ARG
    assert R.lib.rbicg_op_eig_select(R.R64, 100, None, None, 4, None, None, None, None, None) == R.ERR_ARG
    assert R.lib.rbicg_bilinear_form(None, R.R64, None, None, None, None, None, None) == R.ERR_ARG
    ip = R.IrkaParams()
    R.lib.rbicg_irka_default_params(C.byref(ip))
    assert (ip.r, ip.max_steps, ip.shift_tol, ip.strategy, ip.refresh_every, ip.batched) == (8, 10, 1e-6, 1, 1, 1)
    res = R.IrkaResult()
    assert R.lib.rbicg_irka(C.byref(p), C.byref(ip), None, None, None, None, None, None, None, None, None,
                            None, None, C.byref(res)) == R.ERR_ARG
    one = C.c_void_p(1)
    csr = R.CSRStruct()
    csr.n, csr.nnz, csr.row_ptr, csr.col_idx, csr.val = 4, 4, 1, 1, 1
    ip.strategy = 7
    sh = (C.c_double * 16)()
    assert R.lib.rbicg_irka(C.byref(p), C.byref(ip), C.byref(csr), one, one, sh, None, sh, None, None, None,
                            None, None, C.byref(res)) == R.ERR_ARG
    assert b"strategy" in R.lib.rbicg_last_error(None)
    ip.strategy = 1
    csr.has_shift = 1
    assert R.lib.rbicg_irka(C.byref(p), C.byref(ip), C.byref(csr), one, one, sh, None, sh, None, None, None,
                            None, None, C.byref(res)) == R.ERR_ARG
    h2 = C.c_void_p()
    assert R.lib.rbicg_create(C.byref(p), 100, R.R64, None, C.byref(h2)) == R.OK
    assert R.lib.rbicg_set_refresh(h2, 2) == R.ERR_ARG
    assert R.lib.rbicg_set_refresh(h2, 0) == R.OK
    assert R.lib.rbicg_destroy(h2) == R.OK
