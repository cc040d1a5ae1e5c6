"""Restricted open-shell f_ov term and orbital contributions: GPU vs the oracle.

f_ov: the occupied-virtual Fock block of an RO reference (Sec. 3.3, eq
off_diagonal_fock) enters V like the T1 term.  Orbital contributions: eq
cim_pt_energy (1/3 same spin; 1/4, 1/4, 1/2 mixed).  Float64 path within
1e-10 Eh per triplet / orbital, BF16X6 within 1e-7 Eh.
"""
import json
import math
import os

import numpy as np
import pytest
import torch

from oracle import triples as T
from paper_2311_10048_gb300 import lno_ot
from paper_2311_10048_gb300.synth import add_fov, config_domain, make_domain

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")
CASES = ("aaa", "aab", "abb", "bbb")


def golden(name):
    return json.load(open(os.path.join(GOLD, f"{name}_energy.json")))


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


def run(ctx, d_np, sel=None):
    dd = lno_ot.to_device(d_np)
    na, nb = dd["nocc"]
    n = [T.n_triplets(c, na, nb) if sel is None or sel[i] is None else len(sel[i])
         for i, c in enumerate(CASES)]
    et = [torch.zeros(max(k, 1), dtype=torch.float64, device="cuda") for k in n]
    eo = [torch.full((max(na, 1),), np.nan, dtype=torch.float64, device="cuda"),
          torch.full((max(nb, 1),), np.nan, dtype=torch.float64, device="cuda")]
    out = ctx.energy(dd, e_trip=et, trip_sel=sel, e_orb=eo)
    return out, [e[:k].cpu().numpy() for e, k in zip(et, n)], \
        [eo[0][:na].cpu().numpy(), eo[1][:nb].cpu().numpy()]


def c0f():
    g = golden("c0f")
    return add_fov(config_domain("c0"), sd=g["fov"]["sd"], seed=g["fov"]["seed"]), g


def test_c0_fov_fp64_matches_stored_oracle(ctx64):
    d, g = c0f()
    out, et, eo = run(ctx64, d)
    for i, c in enumerate(CASES):
        ref = np.array(g["cases"][c]["e"])
        assert np.abs(et[i] - ref).max() <= 1e-10, c
        assert abs(out[c] - g["cases"][c]["sum"]) <= 1e-8, c
    assert abs(out["total"] - g["total"]) <= 1e-8
    for s, key in enumerate(("alpha", "beta")):
        assert np.abs(eo[s] - np.array(g["orbital"][key])).max() <= 1e-10, key
    # the term is present: differs from the closed-shell-Fock result
    assert abs(out["total"] - golden("c0")["total"]) > 1e-5


def test_c0_fov_bf16x6_within_1e7(ctx6):
    d, g = c0f()
    out, _, eo = run(ctx6, d)
    for c in CASES:
        assert abs(out[c] - g["cases"][c]["sum"]) <= 1e-7, c
    assert abs(out["total"] - g["total"]) <= 1e-7
    for s, key in enumerate(("alpha", "beta")):
        assert np.abs(eo[s] - np.array(g["orbital"][key])).max() <= 1e-7, key


def test_c0_orbital_contributions_without_fov(ctx64, ctx6):
    g = golden("c0")
    for ctx, tol in ((ctx64, 1e-10), (ctx6, 1e-7)):
        out, _, eo = run(ctx, config_domain("c0"))
        for s, key in enumerate(("alpha", "beta")):
            assert np.abs(eo[s] - np.array(g["orbital"][key])).max() <= tol, key
        assert abs(math.fsum(list(eo[0]) + list(eo[1])) - out["total"]) <= 1e-9


SHAPES = [  # nbas, na, nb, naux, seed: ragged tiles, tiny and degenerate spaces
    (7, 3, 2, 14, 1), (20, 5, 1, 40, 3), (37, 4, 3, 70, 4), (18, 3, 0, 30, 7),
    (33, 16, 14, 48, 9),
]


@pytest.mark.parametrize("shape", SHAPES)
def test_shapes_fov_fp64_vs_oracle(ctx64, shape):
    nbas, na, nb, naux, seed = shape
    d = add_fov(make_domain(nbas, (na, nb), naux=naux, L=naux / 3, seed=seed, t1_sd=0.02),
                sd=0.03, seed=seed)
    if nb == 0:
        d["fov"][1] = None
    out, et, eo = run(ctx64, d)
    ev = T.Evaluator(d)
    for i, c in enumerate(CASES):
        ref = [float(ev.triplet_energy(c, t)) for t in T.triplets(c, na, nb)]
        if ref:
            assert np.abs(et[i] - np.array(ref)).max() <= 1e-11 * max(1.0, np.abs(ref).max()), c
        assert abs(out[c] - math.fsum(ref)) <= 1e-9 * max(1.0, abs(out[c])), c
    o = T.orbital_energies(d)
    scale = max(1.0, abs(out["total"]))
    assert np.abs(eo[0] - np.array(o["alpha"])).max() <= 1e-11 * scale
    if nb:
        assert np.abs(eo[1] - np.array(o["beta"])).max() <= 1e-11 * scale


@pytest.mark.parametrize("shape", SHAPES[:3])
def test_shapes_fov_bf16x6_vs_oracle(ctx6, shape):
    nbas, na, nb, naux, seed = shape
    d = add_fov(make_domain(nbas, (na, nb), naux=naux, L=naux / 3, seed=seed, t1_sd=0.02),
                sd=0.03, seed=seed)
    out, _, _ = run(ctx6, d)
    ref = T.energy(d)
    for c in CASES:
        assert abs(out[c] - ref[c]) <= 1e-7 + 1e-7 * abs(ref[c]), c


def test_one_spin_block_null_counts_as_zero(ctx64):
    base = make_domain(20, (5, 3), naux=40, L=13.0, seed=17, t1_sd=0.02)
    d = add_fov(base, sd=0.03, seed=17)
    d_gpu = dict(d, fov=[d["fov"][0], None])
    d_ref = dict(d, fov=[d["fov"][0], np.zeros_like(d["fov"][1])])
    out, _, _ = run(ctx64, d_gpu)
    ref = T.energy(d_ref)
    assert abs(out["total"] - ref["total"]) <= 1e-9 * max(1.0, abs(ref["total"]))


def test_subset_orbital_contributions(ctx64):
    d, _ = c0f()
    sel = [np.array([0, 5, 19]), np.array([59, 1, 30]), None, np.array([3])]
    _, _, eo = run(ctx64, d, sel)
    o = T.orbital_energies(d, trip_sel={c: (None if sel[i] is None else list(sel[i]))
                                        for i, c in enumerate(CASES)})
    assert np.abs(eo[0] - np.array(o["alpha"])).max() <= 1e-10
    assert np.abs(eo[1] - np.array(o["beta"])).max() <= 1e-10


def test_c4_fov_sampled_fp64(ctx64):
    d = add_fov(config_domain("c4"), sd=0.02, seed=4)
    na, nb = d["nocc"]
    rng = np.random.default_rng(404)
    sel = [np.sort(rng.choice(T.n_triplets(c, na, nb), size=2, replace=False)).astype(np.int64)
           for c in CASES]
    _, et, _ = run(ctx64, d, sel)
    ev = T.Evaluator(d)
    with torch.no_grad():
        for i, c in enumerate(CASES):
            allt = T.triplets(c, na, nb)
            ref = np.array([float(ev.triplet_energy(c, allt[int(q)])) for q in sel[i]])
            assert np.abs(et[i] - ref).max() <= 1e-10 * max(1.0, np.abs(ref).max()), c


def test_batched_with_fov_equals_single(lib):
    doms = [add_fov(make_domain(s[0], (s[1], s[2]), naux=s[3], L=s[3] / 3, seed=s[4],
                                t1_sd=0.02), sd=0.03, seed=s[4]) for s in SHAPES[:3]]
    dds = [lno_ot.to_device(x) for x in doms]
    ctx = lno_ot.Context(0, "bf16x6")
    rc, res = ctx.energy_batched(dds)
    assert rc == 0
    singles = [ctx.energy(x) for x in dds]
    ctx.close()
    for r, s1 in zip(res, singles):
        for c in CASES + ("total",):
            assert r[c] == s1[c]


def test_fov_on_spin_without_virtuals_is_rejected(ctx64):
    d = make_domain(5, (5, 3), naux=10, L=4.0, seed=11)    # spin up: no virtual
    dd = lno_ot.to_device(d)
    dd["fov"] = [torch.zeros((5, 1), dtype=torch.float64, device="cuda"), None]
    s, keep = lno_ot.make_domain_struct(dd)
    assert ctx64.energy_raw(s)[0] == lno_ot.EINVAL
