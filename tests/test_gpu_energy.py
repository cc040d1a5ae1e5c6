"""GPU path vs the CPU oracle, element by element (per-triplet contributions).

Float64 path: |dE| <= 1e-8 Eh on every case sum and 1e-10 Eh per triplet.
Tensor-core paths: |dE| <= 1e-7 Eh at the small configuration (BF16X6).
"""
import json
import math
import os

import numpy as np
import pytest
import torch

from oracle import triples as T
from paper_2311_10048_gb300 import lno_ot
from paper_2311_10048_gb300.synth import config_domain, make_domain

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")
CASES = ("aaa", "aab", "abb", "bbb")


def golden(name):
    p = os.path.join(GOLD, f"{name}_energy.json")
    if not os.path.exists(p):
        pytest.skip(f"stored oracle values {p} not generated")
    return json.load(open(p))


@pytest.fixture(scope="module")
def ctx64(lib):
    c = lno_ot.Context(0, "fp64")
    yield c
    c.close()


@pytest.fixture(scope="module")
def ctx6(lib):
    c = lno_ot.Context(0, "bf16x6")
    yield c
    c.close()


@pytest.fixture(scope="module")
def ctx3(lib):
    c = lno_ot.Context(0, "bf16x3")
    yield c
    c.close()


def run_with_trip(ctx, dom_np, sel=None):
    dd = lno_ot.to_device(dom_np)
    na, nb = dd["nocc"]
    n = [T.n_triplets(c, na, nb) if sel is None or sel[i] is None else len(sel[i])
         for i, c in enumerate(CASES)]
    et = [torch.zeros(max(k, 1), dtype=torch.float64, device="cuda") for k in n]
    out = ctx.energy(dd, e_trip=et, trip_sel=sel)
    return out, [e[:k].cpu().numpy() for e, k in zip(et, n)]


def test_c0_fp64_per_triplet_matches_stored_oracle(ctx64):
    g = golden("c0")
    out, et = run_with_trip(ctx64, config_domain("c0"))
    for i, c in enumerate(CASES):
        ref = np.array(g["cases"][c]["e"])
        assert et[i].shape == ref.shape
        assert np.abs(et[i] - ref).max() <= 1e-10, c
        assert abs(out[c] - g["cases"][c]["sum"]) <= 1e-8, c
    assert abs(out["total"] - g["total"]) <= 1e-8


SHAPES = [  # nbas, na, nb, naux, seed -- ragged tiles, tiny and degenerate spaces
    (7, 3, 2, 14, 1), (9, 3, 3, 20, 2), (20, 5, 1, 40, 3), (37, 4, 3, 70, 4),
    (50, 7, 4, 90, 5), (23, 6, 6, 46, 6), (18, 3, 0, 30, 7), (40, 2, 1, 64, 8),
    (33, 16, 14, 48, 9),
]


@pytest.mark.parametrize("shape", SHAPES)
def test_shapes_fp64_vs_oracle(ctx64, shape):
    nbas, na, nb, naux, seed = shape
    d = make_domain(nbas, (na, nb), naux=naux, L=naux / 3, seed=seed, t1_sd=0.02)
    out, et = run_with_trip(ctx64, d)
    ev = T.Evaluator(d)
    for i, c in enumerate(CASES):
        ref = [float(ev.triplet_energy(c, t)) for t in T.triplets(c, na, nb)]
        if ref:
            assert np.abs(et[i] - np.array(ref)).max() <= 1e-11 * max(1.0, np.abs(ref).max()), c
        assert abs(out[c] - math.fsum(ref)) <= 1e-9 * max(1.0, abs(out[c])), c


def test_no_virtuals_and_no_triplets(ctx64):
    d = make_domain(5, (5, 3), naux=10, L=4.0, seed=11)   # spin up has no virtual
    out = ctx64.energy(lno_ot.to_device(d))
    ref = T.energy(d)
    for c in CASES:
        assert abs(out[c] - ref[c]) <= 1e-12
    d = make_domain(12, (2, 1), naux=20, L=6.0, seed=12)  # aaa, bbb, abb empty
    out = ctx64.energy(lno_ot.to_device(d))
    assert out["aaa"] == 0.0 and out["bbb"] == 0.0 and out["abb"] == 0.0
    assert abs(out["aab"] - T.energy(d)["aab"]) <= 1e-12


def test_triplet_subset(ctx64):
    d = config_domain("c0")
    g = golden("c0")
    sel = [np.array([0, 5, 19]), np.array([59, 1, 30]), None, np.array([3])]
    out, et = run_with_trip(ctx64, d, sel)
    for i, c in enumerate(CASES):
        ref = np.array(g["cases"][c]["e"])
        want = ref if sel[i] is None else ref[sel[i]]
        assert np.abs(et[i] - want).max() <= 1e-10
        assert abs(out[c] - math.fsum(want)) <= 1e-9


def test_c0_bf16x6_within_1e7(ctx6):
    g = golden("c0")
    out, et = run_with_trip(ctx6, config_domain("c0"))
    for i, c in enumerate(CASES):
        assert abs(out[c] - g["cases"][c]["sum"]) <= 1e-7, (c, out[c], g["cases"][c]["sum"])
    assert abs(out["total"] - g["total"]) <= 1e-7


def test_c0_bf16x3_close(ctx3):
    g = golden("c0")
    out, _ = run_with_trip(ctx3, config_domain("c0"))
    assert abs(out["total"] - g["total"]) <= 1e-4 * abs(g["total"])


@pytest.mark.parametrize("shape", SHAPES[:5])
def test_shapes_bf16x6_vs_oracle(ctx6, shape):
    nbas, na, nb, naux, seed = shape
    d = make_domain(nbas, (na, nb), naux=naux, L=naux / 3, seed=seed, t1_sd=0.02)
    out, _ = run_with_trip(ctx6, d)
    ref = T.energy(d)
    for c in CASES:
        assert abs(out[c] - ref[c]) <= 1e-7 + 1e-7 * abs(ref[c]), c


def test_error_codes(ctx64, lib):
    import ctypes
    d = config_domain("c0")
    dd = lno_ot.to_device(d)
    s, keep = lno_ot.make_domain_struct(dd)
    s.nocc[1] = s.nocc[0] + 1
    assert ctx64.energy_raw(s)[0] == lno_ot.EINVAL
    s, keep = lno_ot.make_domain_struct(dd)
    s.B[0] = None
    assert ctx64.energy_raw(s)[0] == lno_ot.EINVAL
    host = torch.zeros(10, dtype=torch.float64)
    s, keep = lno_ot.make_domain_struct(dd)
    s.eps[1] = host.data_ptr()
    assert ctx64.energy_raw(s)[0] == lno_ot.EDEVICE
    s, keep = lno_ot.make_domain_struct(dd, trip_sel=[np.array([10 ** 6]), None, None, None])
    assert ctx64.energy_raw(s)[0] == lno_ot.EINVAL
    with pytest.raises(lno_ot.LnoError):
        lno_ot.Context(0, 99)                     # no such precision
    # the context stays usable after errors
    assert abs(ctx64.energy(dd)["total"] - golden("c0")["total"]) <= 1e-8


def test_c4_fp64_matches_stored_oracle(ctx64):
    g = golden("c4")
    out, et = run_with_trip(ctx64, config_domain("c4"))
    for i, c in enumerate(CASES):
        ref = np.array(g["cases"][c]["e"])
        assert np.abs(et[i] - ref).max() <= 1e-10 * max(1.0, np.abs(ref).max()), c
        assert abs(out[c] - g["cases"][c]["sum"]) <= 1e-8, c
    assert abs(out["total"] - g["total"]) <= 1e-8


def test_batched_equals_single_domain_calls(lib):
    doms = [make_domain(*s[:1], (s[1], s[2]), naux=s[3], L=s[3] / 3, seed=s[4], t1_sd=0.02)
            for s in SHAPES[:4]]
    dds = [lno_ot.to_device(d) for d in doms]
    for prec in ("fp64", "bf16x6"):
        ctx = lno_ot.Context(0, prec)
        rc, res = ctx.energy_batched(dds)
        assert rc == 0
        singles = [ctx.energy(dd) for dd in dds]
        ctx.close()
        for r, s1, d in zip(res, singles, doms):
            assert r["status"] == 0
            for c in CASES + ("total",):
                assert r[c] == s1[c]            # same kernels, same order: bitwise
            ref = T.energy(d)
            assert abs(r["total"] - ref["total"]) <= (1e-9 if prec == "fp64" else 1e-7)


def test_batched_reports_per_domain_errors(lib):
    good = lno_ot.to_device(make_domain(12, (3, 2), naux=24, L=8.0, seed=3))
    ctx = lno_ot.Context(0, "fp64")
    import ctypes
    s_good, _ = lno_ot.make_domain_struct(good)
    s_bad, _ = lno_ot.make_domain_struct(good)
    s_bad.nocc[1] = 7          # nocc[1] > nocc[0]
    arr = (lno_ot.Domain * 3)(s_good, s_bad, s_good)
    res = (lno_ot.Result * 3)()
    rc = ctx.lib.lno_ot_energy_batched(ctx.h, 3, arr, res)
    assert rc == lno_ot.EINVAL
    assert res[0].status == 0 and res[1].status == lno_ot.EINVAL and res[2].status == 0
    assert res[0].e[4] == res[2].e[4] != 0.0
    ctx.close()


def test_tuning_table_is_read(lib, tmp_path):
    d = lno_ot.to_device(make_domain(40, (6, 4), naux=80, L=20.0, seed=1))
    ref = None
    for rows in ("1000 0 4\n", "1000 64 64\n", "# comment\n20 64 1\n1000 0 2\n"):
        p = tmp_path / "t.txt"
        p.write_text(rows)
        ctx = lno_ot.Context(0, "bf16x6", tune_cache=str(p))
        e = ctx.energy(d)["total"]
        ctx.close()
        ref = e if ref is None else ref
        assert e == ref                          # schedule changes never change the result
    with pytest.raises(lno_ot.LnoError):
        lno_ot.Context(0, "bf16x6", tune_cache=str(tmp_path / "missing.txt"))


@pytest.fixture(scope="module")
def ctx10(lib):
    c = lno_ot.Context(0, "bf16x10")
    yield c
    c.close()


def test_c0_bf16x10_within_1e8(ctx10):
    g = golden("c0")
    out, et = run_with_trip(ctx10, config_domain("c0"))
    for i, c in enumerate(CASES):
        assert np.abs(et[i] - np.array(g["cases"][c]["e"])).max() <= 1e-9, c
    assert abs(out["total"] - g["total"]) <= 1e-8


def test_c4_bf16x10_matches_stored_oracle(ctx10):
    # 4 BF16 slices per operand: per triplet ~40x closer to the oracle than BF16X6
    g = golden("c4")
    out, et = run_with_trip(ctx10, config_domain("c4"))
    for i, c in enumerate(CASES):
        assert np.abs(et[i] - np.array(g["cases"][c]["e"])).max() <= 2e-9, c
    assert abs(out["total"] - g["total"]) <= 1e-8


@pytest.mark.parametrize("shape", SHAPES[:5])
def test_shapes_bf16x10_vs_oracle(ctx10, shape):
    nbas, na, nb, naux, seed = shape
    d = make_domain(nbas, (na, nb), naux=naux, L=naux / 3, seed=seed, t1_sd=0.02)
    out, _ = run_with_trip(ctx10, d)
    ref = T.energy(d)
    for c in CASES:
        assert abs(out[c] - ref[c]) <= 1e-9 + 1e-9 * abs(ref[c]), c


@pytest.mark.parametrize("prec,widths", [("bf16x3", (256, 128)), ("bf16x6", (128, 64)),
                                         ("bf16x10", (128, 64)), ("bf16x10", (128, 96))])
def test_tile_widths_give_bitwise_equal_results(lib, tmp_path, prec, widths):
    # several n-tiles per problem (154 virtuals: 11781 pairs) and a ragged m edge
    d = lno_ot.to_device(make_domain(160, (6, 4), naux=120, L=30.0, seed=2))
    res = []
    for bn in widths:
        p = tmp_path / f"t{prec}{bn}.txt"
        p.write_text(f"100000 {bn} 16\n")
        ctx = lno_ot.Context(0, prec, tune_cache=str(p))
        res.append(ctx.energy(d))
        ctx.close()
    for c in CASES + ("total",):
        assert res[0][c] == res[1][c], (prec, c)


@pytest.fixture(scope="module")
def ctx15(lib):
    c = lno_ot.Context(0, "bf16x15")
    yield c
    c.close()


# BF16X15 removes the slicing error almost entirely; what is left per triplet
# is the float32 rounding of the W intermediates and of the energy arithmetic
# (about 1e-8 of e_t at c0), the same floor as BF16X10's
def test_c0_bf16x15_per_triplet(ctx15):
    g = golden("c0")
    out, et = run_with_trip(ctx15, config_domain("c0"))
    for i, c in enumerate(CASES):
        assert np.abs(et[i] - np.array(g["cases"][c]["e"])).max() <= 1e-9, c
    assert abs(out["total"] - g["total"]) <= 1e-8


def test_c4_bf16x15_per_triplet(ctx15):
    g = golden("c4")
    out, et = run_with_trip(ctx15, config_domain("c4"))
    worst = 0.0
    for i, c in enumerate(CASES):
        err = np.abs(et[i] - np.array(g["cases"][c]["e"])).max()
        worst = max(worst, err)
        assert err <= 2e-9, c
    # the per-triplet float32 rounding (~1e-10 Eh, unbiased) adds up as
    # sqrt(8436) over the domain
    assert abs(out["total"] - g["total"]) <= 3e-8
    print("c4 bf16x15 worst per-triplet |dE| =", worst)


def test_kept_operands_give_the_whole_domain_per_triplet_values(lib):
    # blocks of triplets through a context that keeps the operands equal, bit
    # for bit, one uncached call over the whole domain; release and a new
    # domain rebuild them
    d = make_domain(60, (7, 5), naux=100, L=25.0, seed=12, t1_sd=0.02)
    dd = lno_ot.to_device(d)
    na, nb = dd["nocc"]
    n = [T.n_triplets(c, na, nb) for c in CASES]
    for prec in ("bf16x10", "fp64"):
        ref_ctx = lno_ot.Context(0, prec)
        ref = [torch.zeros(k, dtype=torch.float64, device="cuda") for k in n]
        tot = ref_ctx.energy(dd, e_trip=ref)["total"]
        ref_ctx.close()
        ctx = lno_ot.Context(0, prec, keep_operands=True)
        for rep in range(2):
            got = [torch.full((k,), float("nan"), dtype=torch.float64, device="cuda") for k in n]
            K = 3
            for s in range(K):
                sel = [np.arange(k * s // K, k * (s + 1) // K, dtype=np.int64) for k in n]
                views = [got[ci][sel[ci][0]:sel[ci][-1] + 1] if len(sel[ci]) else None
                         for ci in range(4)]
                ctx.energy(dd, e_trip=views, trip_sel=sel)
            for ci in range(4):
                assert torch.equal(got[ci], ref[ci]), (prec, rep, CASES[ci])
            assert ctx.energy(dd)["total"] == tot
            ctx.release()
        other = lno_ot.to_device(config_domain("c0"))
        e0 = ctx.energy(other)["total"]
        ctx.close()
        g = golden("c0")
        assert abs(e0 - g["total"]) <= 1e-8


def test_tf32_path_against_oracle(lib):
    # TF32 slices with rounding FP32 accumulation: measured, not exact
    g0, g4 = golden("c0"), golden("c4")
    ctx = lno_ot.Context(0, "tf32")
    out0, et0 = run_with_trip(ctx, config_domain("c0"))
    out4 = ctx.energy(lno_ot.to_device(config_domain("c4")))
    ctx.close()
    err0 = max(abs(out0[c] - g0["cases"][c]["sum"]) for c in CASES)
    err4 = abs(out4["total"] - g4["total"])
    print("tf32: c0 worst case |dE| =", err0, " c4 total |dE| =", err4)
    assert err0 <= 1e-6
    assert err4 <= 1e-5 * abs(g4["total"])
