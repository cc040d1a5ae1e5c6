"""The tcgen05 contraction kernel on its own (diagnostic C entry point).

Checks the shared-memory layouts, TMA boxes, MMA descriptors and the slice
bookkeeping: integer inputs must come out bit-exact, random inputs within
the slice precision, for tile-aligned and ragged shapes.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2311_10048_gb300 import lno_ot

pytestmark = pytest.mark.gpu


def run(lib, S, A, B):
    M, K = A.shape
    N = B.shape[0]
    dA = torch.as_tensor(A, dtype=torch.float64).cuda().contiguous()
    dB = torch.as_tensor(B, dtype=torch.float64).cuda().contiguous()
    dC = torch.full((N, M), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    rc = lib.lno_ot_selftest_gemm(0, S, M, N, K, ctypes.c_void_p(dA.data_ptr()),
                                  ctypes.c_void_p(dB.data_ptr()), ctypes.c_void_p(dC.data_ptr()),
                                  None)
    assert rc == 0, lib.lno_ot_strerror(rc)
    return dC.cpu().numpy()


@pytest.fixture(scope="module")
def L(lib):
    lib.lno_ot_selftest_gemm.argtypes = [ctypes.c_int] * 5 + [ctypes.c_void_p] * 4
    lib.lno_ot_selftest_gemm.restype = ctypes.c_int
    return lib


@pytest.mark.parametrize("shape", [(128, 256, 32), (200, 300, 40), (5, 7, 3), (384, 512, 416),
                                   (130, 1000, 64)])
def test_integer_inputs_are_exact(L, shape):
    M, N, K = shape
    rng = np.random.default_rng(M * 7 + N)
    A = rng.integers(-128, 129, size=(M, K)).astype(np.float64)
    B = rng.integers(-128, 129, size=(N, K)).astype(np.float64)
    A[0, 0] = 128.0   # pins the power-of-two scale to 128 (integer slices)
    B[0, 0] = -128.0
    C = run(L, 1, A, B)
    assert np.array_equal(C, B @ A.T)


@pytest.mark.parametrize("S", [1, 2, 3, 4, 5])
def test_random_inputs_within_slice_precision(L, S):
    M, N, K = 300, 700, 600
    rng = np.random.default_rng(S)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((N, K))
    ref = B @ A.T
    C = run(L, S, A, B)
    scale = np.abs(A).max() * np.abs(B).max() * np.sqrt(K)
    err = np.abs(C - ref).max() / scale
    # each operand carries about 8 S - 1 bits relative to its largest element;
    # the dropped slice products (p + q >= S) bound the error at that level
    assert err < 2.0 ** (-8 * S + 4), err
    if S == 4:
        assert np.abs(C - ref).max() / np.abs(ref).max() < 1e-8
    if S == 5:
        assert np.abs(C - ref).max() / np.abs(ref).max() < 1e-10


def test_negative_and_zero_matrices(L):
    A = np.zeros((64, 16))
    B = np.ones((33, 16))
    assert np.array_equal(run(L, 2, A, B), np.zeros((33, 64)))
    A = -np.ones((64, 16)) * 0.75
    C = run(L, 3, A, B)
    assert np.allclose(C, -12.0, atol=0, rtol=0)
