"""C-ABI library: builds, loads without a GPU, exports what the header declares.

No compute calls here (no GPU on the CPU runner).
"""
import ctypes
import os
import subprocess
import textwrap

import pytest

from paper_2311_10048_gb300 import lno_ot

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_header_function(lib):
    names = lno_ot.exported_names()
    assert {"lno_ot_init", "lno_ot_energy", "lno_ot_energy_batched", "lno_ot_backward",
            "lno_ot_destroy", "lno_ot_strerror"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n


def test_strerror_and_version(lib):
    for code in (0, -1, -2, -3, -4, -5, -6, 99):
        assert lib.lno_ot_strerror(code)
    assert lib.lno_ot_version().decode().startswith("lno_ot")


def test_null_arguments_rejected_without_device(lib):
    assert lib.lno_ot_init(None, None) == lno_ot.EINVAL
    r = lno_ot.Result()
    assert lib.lno_ot_energy(None, None, ctypes.byref(r)) == lno_ot.EINVAL
    assert lib.lno_ot_energy_batched(None, 0, None, None) == lno_ot.EINVAL
    st = lno_ot.Stats()
    assert lib.lno_ot_last_stats(None, ctypes.byref(st)) == lno_ot.EINVAL


def test_ctypes_struct_layouts_match_c(tmp_path):
    """sizeof/offsetof of every public struct, C compiler vs the binding."""
    src = tmp_path / "sz.c"
    src.write_text(textwrap.dedent("""
        #include <stdio.h>
        #include <stddef.h>
        #include "lno_ot.h"
        int main(void) {
          printf("%zu %zu %zu %zu %zu\\n", sizeof(lno_ot_options), sizeof(lno_ot_domain),
                 sizeof(lno_ot_result), sizeof(lno_ot_grad), sizeof(lno_ot_stats));
          printf("%zu %zu %zu %zu %zu %zu %zu\\n", offsetof(lno_ot_domain, t2ab),
                 offsetof(lno_ot_domain, e_trip), offsetof(lno_ot_domain, n_sel),
                 offsetof(lno_ot_stats, elements), offsetof(lno_ot_domain, fov),
                 offsetof(lno_ot_domain, e_orb), offsetof(lno_ot_grad, dfov));
          printf("%zu %zu %zu %zu\\n", sizeof(lno_ot_central), offsetof(lno_ot_central, spin),
                 offsetof(lno_ot_central, U), offsetof(lno_ot_central, dE));
          return 0;
        }
    """))
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    got = [int(x) for x in out]
    C = ctypes
    want = [C.sizeof(lno_ot.Options), C.sizeof(lno_ot.Domain), C.sizeof(lno_ot.Result),
            C.sizeof(lno_ot.Grad), C.sizeof(lno_ot.Stats),
            lno_ot.Domain.t2ab.offset, lno_ot.Domain.e_trip.offset, lno_ot.Domain.n_sel.offset,
            lno_ot.Stats.elements.offset, lno_ot.Domain.fov.offset, lno_ot.Domain.e_orb.offset,
            lno_ot.Grad.dfov.offset, C.sizeof(lno_ot.Central), lno_ot.Central.spin.offset,
            lno_ot.Central.U.offset, lno_ot.Central.dE.offset]
    assert got == want


def test_build_is_sm103a_only():
    from paper_2311_10048_gb300 import build as b
    assert b.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_enum_values_match_binding():
    """Status codes and precision modes: header enums vs the binding's constants."""
    import re
    text = open(os.path.join(ROOT, "include", "lno_ot.h")).read()
    enums = {m.group(1): int(m.group(2))
             for m in re.finditer(r"\b(LNO_OT_[A-Z0-9]+)\s*=\s*(-?\d+)", text)}
    want = {"LNO_OT_OK": lno_ot.OK, "LNO_OT_EINVAL": lno_ot.EINVAL,
            "LNO_OT_EDEVICE": lno_ot.EDEVICE, "LNO_OT_ENOMEM": lno_ot.ENOMEM,
            "LNO_OT_ECUDA": lno_ot.ECUDA, "LNO_OT_ETIMEOUT": lno_ot.ETIMEOUT,
            "LNO_OT_EUNSUPPORTED": lno_ot.EUNSUPPORTED, "LNO_OT_FP64": lno_ot.FP64,
            "LNO_OT_BF16X3": lno_ot.BF16X3, "LNO_OT_TF32": lno_ot.TF32,
            "LNO_OT_BF16X6": lno_ot.BF16X6, "LNO_OT_BF16X10": lno_ot.BF16X10,
            "LNO_OT_BF16X15": lno_ot.BF16X15}
    for k, v in want.items():
        assert enums.get(k) == v, (k, enums.get(k), v)
    assert set(lno_ot.PRECISIONS.values()) == {0, 1, 2, 3, 4, 5}


def test_laplace_quadrature_meets_its_tolerance():
    """Host-only routine: the returned exponential sum bounds the relative
    error of 1/x on the range by tol (checked on a dense grid here), with
    3-4 points at the paper's laptol = 1e-2 on a (T) denominator range."""
    import numpy as np
    for lo, hi, tol, nmax_pts in ((1.2, 21.0, 1e-2, 4), (3.9, 16.1, 1e-2, 4), (0.5, 40.0, 1e-2, 8),
                                  (1.2, 21.0, 1e-3, 10), (1.2, 21.0, 1e-4, 14)):
        s, w = lno_ot.laplace_quadrature(lo, hi, tol)
        x = np.geomspace(lo, hi, 20000)
        err = np.abs(1.0 - x * (np.exp(-np.outer(x, s)) @ w)).max()
        assert err <= tol, (lo, hi, tol, err)
        assert len(s) <= nmax_pts and (s > 0).all() and (np.diff(s) > 0).all()
    with pytest.raises(lno_ot.LnoError):
        lno_ot.laplace_quadrature(2.0, 1.0, 1e-2)
