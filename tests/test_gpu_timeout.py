"""Bounded device waits of the contraction and energy kernels, exercised
without a fault.

lno_ot_selftest_timeout runs one tile with the contraction kernel's test hook
that issues no copy, so the MMA thread's first wait for operand data can only
end by its time limit (a flag that nothing sets).  The call must come back
with LNO_OT_ETIMEOUT and the code of a wait for work, twice in a row, and the
device must then still compute the small domain c0 correctly (stored oracle
values) and a plain product on the same kernel.  lno_ot_selftest_energy_timeout
does the same for the TMA staging of the energy kernel (code 7).
"""
import ctypes
import json
import os

import numpy as np
import pytest
import torch

from paper_2311_10048_gb300 import lno_ot
from paper_2311_10048_gb300.synth import config_domain

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")
CASES = ("aaa", "aab", "abb", "bbb")


def test_bounded_wait_gives_up_and_device_recovers(lib):
    lno_ot.load_library()
    for _ in range(2):
        code = ctypes.c_int(-1)
        rc = lib.lno_ot_selftest_timeout(0, 2_000_000, ctypes.byref(code), None)
        assert rc == lno_ot.ETIMEOUT, lib.lno_ot_strerror(rc)
        assert code.value in (3, 6), code.value   # MMA thread or epilogue gave up
    assert lib.lno_ot_selftest_timeout(0, 10, None, None) == lno_ot.EINVAL

    g = json.load(open(os.path.join(GOLD, "c0_energy.json")))
    dd = lno_ot.to_device(config_domain("c0"))
    for prec, tol in (("bf16x10", 1e-8), ("fp64", 1e-8)):
        ctx = lno_ot.Context(0, prec)
        out = ctx.energy(dd)
        ctx.close()
        for c in CASES:
            assert abs(out[c] - g["cases"][c]["sum"]) <= tol, (prec, c)

    rng = np.random.default_rng(5)
    A = rng.standard_normal((200, 96))
    B = rng.standard_normal((300, 96))
    dA, dB = torch.as_tensor(A).cuda(), torch.as_tensor(B).cuda()
    dC = torch.full((300, 200), float("nan"), dtype=torch.float64, device="cuda")
    rc = lib.lno_ot_selftest_gemm(0, 4, 200, 300, 96, ctypes.c_void_p(dA.data_ptr()),
                                  ctypes.c_void_p(dB.data_ptr()), ctypes.c_void_p(dC.data_ptr()),
                                  None)
    assert rc == 0
    ref = B @ A.T
    assert np.abs(dC.cpu().numpy() - ref).max() / np.abs(ref).max() < 1e-8


def test_energy_stage_wait_gives_up_and_device_recovers(lib):
    lno_ot.load_library()
    for _ in range(2):
        code = ctypes.c_int(-1)
        rc = lib.lno_ot_selftest_energy_timeout(0, 2_000_000, ctypes.byref(code), None)
        assert rc == lno_ot.ETIMEOUT, lib.lno_ot_strerror(rc)
        assert code.value == 7, code.value
    assert lib.lno_ot_selftest_energy_timeout(0, 10, None, None) == lno_ot.EINVAL

    g = json.load(open(os.path.join(GOLD, "c0_energy.json")))
    dd = lno_ot.to_device(config_domain("c0"))
    ctx = lno_ot.Context(0, "bf16x10")
    out = ctx.energy(dd)
    ctx.close()
    for c in CASES:
        assert abs(out[c] - g["cases"][c]["sum"]) <= 1e-8, c
