"""rbicg_op_gram_noalloc, the allocation-free Gram entry point for callers that must not
allocate device memory, against the allocating rbicg_op_gram on two consecutive calls.

Kept in a file that pytest collects last; it passes alone in a fresh process and after the
other tests (the entry point keeps no state other than its shared scratch array)."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1010_0762_gb300 import rbicg as R
    f = R.lib.rbicg_op_gram_noalloc
    f.restype = C.c_int
    f.argtypes = [C.c_int, C.c_int64, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_int,
                  C.c_void_p, C.c_void_p]
    return R, f


def test_gram_noalloc_matches_allocating_gram_on_two_calls():
    R, f = _lib()
    stream = torch.cuda.current_stream()
    cases = [(False, False, 70001, 64, 40), (True, False, 9001, 17, 64), (False, True, 70001, 64, 64)]
    for cx, fp32, n, mx, my in cases:
        rng = np.random.default_rng(mx * 1000 + my)
        X = rng.standard_normal((n, mx)) + (1j * rng.standard_normal((n, mx)) if cx else 0)
        Y = rng.standard_normal((n, my)) + (1j * rng.standard_normal((n, my)) if cx else 0)
        Xd = torch.as_tensor(X, device="cuda")
        Yd = torch.as_tensor(Y, device="cuda")
        ref = R.op_gram(Xd, Yd, fp32=fp32)            # existing (allocating) entry point
        scale = np.sqrt(np.outer((abs(X) ** 2).sum(0), (abs(Y) ** 2).sum(0)))
        tol = 2e-6 if fp32 else 1e-13                  # the tolerances of the Gram parity tests
        for _ in range(2):                             # two calls in a row share the scratch
            G = torch.full((mx, my), float("nan"), dtype=Xd.dtype, device="cuda")
            st = f(R.C128 if cx else R.R64, n, Xd.data_ptr(), mx, Xd.stride(0), Yd.data_ptr(), my,
                   Yd.stride(0), int(fp32), G.data_ptr(), stream.cuda_stream)
            stream.synchronize()
            assert st == R.OK
            err = (abs(G.cpu().numpy() - ref) / scale).max()
            assert err < tol, err
            # and against X^H Y formed on the host
            err = (abs(G.cpu().numpy() - X.conj().T @ Y) / scale).max()
            assert err < tol, err


def test_gram_noalloc_rejects_sizes_beyond_its_scratch():
    R, f = _lib()
    X = torch.zeros(100, 65, dtype=torch.float64, device="cuda")
    G = torch.zeros(65, 65, dtype=torch.float64, device="cuda")
    st = f(R.R64, 100, X.data_ptr(), 65, 65, X.data_ptr(), 65, 65, 0, G.data_ptr(),
           torch.cuda.current_stream().cuda_stream)
    assert st == R.ERR_ARG
    assert b"1..64" in R.lib.rbicg_last_error(None)
