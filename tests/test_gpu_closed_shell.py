"""Closed-shell domains: the spin-flip shortcut (only aaa and aab computed when
both spins share their arrays) against the full four-case path and the
closed-shell (T) formula of the oracle (pin P2)."""
import numpy as np
import pytest
import torch

from oracle.closed_shell import rhf_energy
from paper_2311_10048_gb300 import lno_ot
from paper_2311_10048_gb300.synth import make_domain

pytestmark = pytest.mark.gpu
CASES = ("aaa", "aab", "abb", "bbb")


def shared(dd):
    """The same device arrays for both spins (the closed-shell calling form)."""
    return dict(dd, B=[dd["B"][0]] * 2, eps=[dd["eps"][0]] * 2, t1=[dd["t1"][0]] * 2,
                t2bb=dd["t2aa"])


# float64: the two paths differ only by the rounding-level asymmetry of t2ab;
# BF16X6: each is within the 1e-7 Eh bar of the exact value
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("bf16x6", 1e-7)])
@pytest.mark.parametrize("shape", [(24, 4, 48, 21), (40, 6, 120, 22), (37, 5, 70, 23)])
def test_spin_flip_shortcut_equals_full_path(lib, prec, tol, shape):
    nbas, n, naux, seed = shape
    d = make_domain(nbas, (n, n), naux=naux, L=naux / 3, seed=seed, closed_shell=True)
    dd = lno_ot.to_device(d)
    ctx = lno_ot.Context(0, prec)
    na = n
    ntr = {"aaa": na * (na - 1) * (na - 2) // 6, "bbb": na * (na - 1) * (na - 2) // 6,
           "aab": na * (na - 1) // 2 * na, "abb": na * (na - 1) // 2 * na}
    et_s = [torch.zeros(ntr[c], dtype=torch.float64, device="cuda") for c in CASES]
    et_f = [torch.zeros(ntr[c], dtype=torch.float64, device="cuda") for c in CASES]
    short = ctx.energy(shared(dd), e_trip=et_s)
    n_short = ctx.stats()["triplets"]
    full = ctx.energy(dd, e_trip=et_f)           # separate (equal) arrays: all four cases
    n_full = ctx.stats()["triplets"]
    ctx.close()
    assert n_short == ntr["aaa"] + ntr["aab"] and n_full == sum(ntr.values())
    rel = prec == "fp64"
    for i, c in enumerate(CASES):
        scale = max(1.0, abs(full[c])) if rel else 1.0
        assert abs(short[c] - full[c]) <= tol * scale, (c, short[c], full[c])
        escale = max(1.0, float(et_f[i].abs().max())) if rel else 1.0
        assert float((et_s[i] - et_f[i]).abs().max()) <= tol * escale, c
    ref = rhf_energy(d)
    assert abs(short["total"] - ref) <= (1e-8 if prec == "fp64" else 1e-7) * max(1.0, abs(ref))


def test_asymmetric_t2ab_disables_the_shortcut(lib):
    d = make_domain(24, (4, 4), naux=48, L=16.0, seed=24, closed_shell=True)
    dd = lno_ot.to_device(d)
    t2ab = dd["t2ab"].clone()
    t2ab[0, 1, 2, 3] += 1e-3                     # breaks t2ab[i][J][a][B] == t2ab[J][i][B][a]
    ctx = lno_ot.Context(0, "fp64")
    out = ctx.energy(dict(shared(dd), t2ab=t2ab))
    n = ctx.stats()["triplets"]
    ref = ctx.energy(dict(dd, t2ab=t2ab))
    ctx.close()
    assert n == 2 * (4 + 4 * 6)                  # all four cases computed
    for c in CASES:
        assert abs(out[c] - ref[c]) <= 1e-12 * max(1.0, abs(ref[c]))
    assert out["aab"] != out["abb"]
