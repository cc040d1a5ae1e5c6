"""The no-allocation contraction entry point (lno_ot_gemm_sliced_noalloc).

It serves callers that cannot allocate device memory (their HBM belongs to
their own pool, or a cudaMalloc is not allowed where they call us); its
scratch is a static device array.  Two calls in a row, with different sizes
and slice counts (the second smaller, so any stale scratch would show), must
each agree with the allocating entry point lno_ot_selftest_gemm within the
slice-precision tolerance the other contraction tests use.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _bind(lib):
    for name in ("lno_ot_selftest_gemm", "lno_ot_gemm_sliced_noalloc"):
        f = getattr(lib, name)
        f.argtypes = [ctypes.c_int] * 5 + [ctypes.c_void_p] * 4
        f.restype = ctypes.c_int
    return lib


def _call(fn, S, A, B):
    M, K = A.shape
    N = B.shape[0]
    dA = torch.as_tensor(A, dtype=torch.float64).cuda().contiguous()
    dB = torch.as_tensor(B, dtype=torch.float64).cuda().contiguous()
    dC = torch.full((N, M), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    rc = fn(0, S, M, N, K, ctypes.c_void_p(dA.data_ptr()), ctypes.c_void_p(dB.data_ptr()),
            ctypes.c_void_p(dC.data_ptr()), None)
    assert rc == 0, rc
    return dC.cpu().numpy()


def test_noalloc_matches_allocating_entry_point_on_two_calls(lib):
    L = _bind(lib)
    cases = [(4, 260, 500, 300, 3), (3, 300, 700, 600, 1), (2, 200, 300, 40, 2)]
    for S, M, N, K, seed in cases:
        rng = np.random.default_rng(seed)
        A = rng.standard_normal((M, K))
        B = rng.standard_normal((N, K))
        ref = _call(L.lno_ot_selftest_gemm, S, A, B)
        got = _call(L.lno_ot_gemm_sliced_noalloc, S, A, B)
        scale = np.abs(A).max() * np.abs(B).max() * np.sqrt(K)
        tol = 2.0 ** (-8 * S + 4)
        assert np.isfinite(got).all()
        assert np.abs(got - ref).max() / scale < tol
        assert np.abs(got - B @ A.T).max() / scale < tol


def test_noalloc_rejects_host_pointers_and_restores_device(lib):
    L = _bind(lib)
    dA = torch.zeros((64, 32), dtype=torch.float64, device="cuda")
    dC = torch.zeros((64, 64), dtype=torch.float64, device="cuda")
    host = np.zeros((64, 32))
    dev0 = torch.cuda.current_device()
    rc = L.lno_ot_gemm_sliced_noalloc(0, 2, 64, 64, 32, ctypes.c_void_p(dA.data_ptr()),
                                      ctypes.c_void_p(host.ctypes.data),
                                      ctypes.c_void_p(dC.data_ptr()), None)
    assert rc == -2   # LNO_OT_EDEVICE: nothing was launched
    assert torch.cuda.current_device() == dev0
    # a bad device ordinal is rejected too
    rc = L.lno_ot_gemm_sliced_noalloc(1 << 20, 2, 64, 64, 32, ctypes.c_void_p(dA.data_ptr()),
                                      ctypes.c_void_p(dA.data_ptr()),
                                      ctypes.c_void_p(dC.data_ptr()), None)
    assert rc == -2


def test_noalloc_rejects_oversized_operands(lib):
    L = _bind(lib)
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    # 4 slices of 8192 x 8192 rows per operand need far more than 64 MiB
    assert L.lno_ot_gemm_sliced_noalloc(0, 4, 8192, 8192, 1024, p, p, p, None) == -1
    assert b"limit" in L.lno_ot_last_error()
