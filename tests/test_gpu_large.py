"""Full-size parity on sampled triplets (the oracle computes them one by one).

c1 (nbas 400): the whole domain runs exactly as bench.py times it (BF16X10,
20 steps, step s = block s of 20 of every case's restricted triplets); the
per-triplet contributions at the seeded sample stored by
tests/golden/make_golden.py must match the oracle within 1e-8 Eh.  The
float64 GPU path and BF16X6 (within 1e-7 Eh) run on the sampled triplets.

c2 (nbas 700, 80/78 occupied, naux 2100): the stored oracle values of a
seeded triplet sample (make_golden.py c2s) against the float64 path
(1e-8 Eh), BF16X15 and BF16X10 (1e-8 Eh) and BF16X6 (1e-7 Eh) on the same
triplets.  Needs ~80 GB of host memory for the inputs.
"""
import json
import math
import os

import numpy as np
import pytest
import torch

from paper_2311_10048_gb300 import lno_ot
from paper_2311_10048_gb300.synth import config_domain

pytestmark = pytest.mark.gpu
CASES = ("aaa", "aab", "abb", "bbb")
GOLD = os.path.join(os.path.dirname(__file__), "golden")
BENCH_STEPS = 20


def n_trip(case, na, nb):
    c2 = lambda n: n * (n - 1) // 2
    c3 = lambda n: n * (n - 1) * (n - 2) // 6
    return {"aaa": c3(na), "bbb": c3(nb), "aab": c2(na) * nb, "abb": c2(nb) * na}[case]


def golden(name):
    p = os.path.join(GOLD, f"{name}_energy.json")
    if not os.path.exists(p):
        pytest.skip(f"stored oracle values {p} not generated")
    return json.load(open(p))


@pytest.fixture(scope="module")
def c1_device():
    d = config_domain("c1")
    dd = lno_ot.to_device(d)
    yield d, dd
    del dd
    torch.cuda.empty_cache()


def sampled(ctx, dd, g, tol, label):
    sel = [np.array(g["cases"][c]["index"], dtype=np.int64) for c in CASES]
    et = [torch.zeros(max(len(s), 1), dtype=torch.float64, device="cuda") for s in sel]
    out = ctx.energy(dd, e_trip=et, trip_sel=sel)
    worst = 0.0
    for ci, c in enumerate(CASES):
        got = et[ci][:len(sel[ci])].cpu().numpy()
        ref = np.array(g["cases"][c]["e"])
        err = np.abs(got - ref)
        worst = max(worst, float(err.max()) if err.size else 0.0)
        assert (err <= tol).all(), (label, c, err.max())
        assert abs(out[c] - math.fsum(ref.tolist())) <= tol * max(1, len(ref)), (label, c)
    return worst


def test_c1_bench_launch_configuration_sampled_parity(lib, c1_device):
    g = golden("c1s")
    d, dd = c1_device
    na, nb = d["nocc"]
    ntr = [n_trip(c, na, nb) for c in CASES]
    et = [torch.zeros(n, dtype=torch.float64, device="cuda") for n in ntr]
    ctx = lno_ot.Context(0, "bf16x10")
    tot = {c: [] for c in CASES}
    for s in range(BENCH_STEPS):
        sel = [np.arange(n * s // BENCH_STEPS, n * (s + 1) // BENCH_STEPS, dtype=np.int64)
               for n in ntr]
        views = [et[ci][sel[ci][0]:sel[ci][-1] + 1] if len(sel[ci]) else None for ci in range(4)]
        out = ctx.energy(dd, e_trip=views, trip_sel=sel)
        for c in CASES:
            tot[c].append(out[c])
    ctx.close()
    worst = 0.0
    for ci, c in enumerate(CASES):
        got = et[ci].cpu().numpy()
        for q, ref in zip(g["cases"][c]["index"], g["cases"][c]["e"]):
            err = abs(float(got[q]) - ref)
            worst = max(worst, err)
            assert err <= 1e-8, (c, q, got[q], ref)
        # the blocks cover every triplet once: the step sums add up to the
        # sum of the per-triplet contributions
        assert abs(math.fsum(tot[c]) - math.fsum(got.tolist())) <= 1e-9 * abs(math.fsum(tot[c]))
    print("c1 bf16x10 (bench launch configuration) worst per-triplet |dE| =", worst)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-8), ("bf16x6", 1e-7)])
def test_c1_sampled_parity_other_paths(lib, c1_device, prec, tol):
    g = golden("c1s")
    _, dd = c1_device
    ctx = lno_ot.Context(0, prec)
    worst = sampled(ctx, dd, g, tol, prec)
    ctx.close()
    print("c1", prec, "worst per-triplet |dE| =", worst)


def test_c2_sampled_parity_all_paths(lib):
    g = golden("c2s")
    d = config_domain("c2")
    dd = lno_ot.to_device(d)
    del d
    res = {}
    for prec, tol in (("fp64", 1e-8), ("bf16x15", 1e-8), ("bf16x10", 1e-8), ("bf16x6", 1e-7)):
        ctx = lno_ot.Context(0, prec)
        res[prec] = sampled(ctx, dd, g, tol, prec)
        ctx.close()
    del dd
    torch.cuda.empty_cache()
    print("c2 worst per-triplet |dE|:", res)
