"""Central-LMO share of E(T) in the Laplace form (Sec. 3.7, eqs
laplace_transform and local_pt) through lno_ot_energy_central, against the
oracle and against properties that hold at any size.

* oracle parity: random orthonormal central orbitals of both spins, the
  oracle's laptol = 1e-2 quadrature given to both sides; float64 path within
  1e-11 Eh, BF16X10 / BF16X15 within 1e-9 Eh, BF16X6 within 1e-8 Eh, on
  shapes with ragged tiles;
* semicanonical limit: with central orbitals = the semicanonical ones and an
  accurate quadrature, each share is 1/3 of the E(T) contribution of every
  triplet the orbital belongs to (per-triplet values of lno_ot_energy);
* a complete orthonormal set: the shares add up to the same total for every
  rotation (a trace) and to E(T) within the quadrature's error, at the
  differentiation domain's size (nbas 200, 20/18 occupied).
"""
import numpy as np
import pytest
import torch

from oracle import laplace as L
from oracle import triples as T
from paper_2311_10048_gb300 import lno_ot
from paper_2311_10048_gb300.synth import config_domain, make_domain

pytestmark = pytest.mark.gpu
CASES = ("aaa", "aab", "abb", "bbb")


def orth(n, seed, rows=None):
    q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((n, n)))
    return q.T[: (n if rows is None else rows)].copy()


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64).cuda()


SHAPES = [(11, 3, 2, 24, 3), (20, 5, 3, 40, 5), (37, 4, 3, 70, 6), (23, 6, 6, 46, 7)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("bf16x10", 1e-9), ("bf16x15", 1e-9),
                                      ("bf16x6", 1e-8)])
def test_central_share_matches_oracle(lib, shape, prec, tol):
    nbas, na, nb, naux, seed = shape
    d = make_domain(nbas, (na, nb), naux=naux, L=naux / 3, seed=seed, t1_sd=0.02)
    lo, hi = L.denominator_range(d)
    s, w = L.quadrature(lo, hi, 1e-2)
    Ua, Ub = orth(na, seed, max(1, na - 1)), orth(nb, seed + 1)
    ref = L.central_energies(d, Ua, Ub, s, w)
    dd = lno_ot.to_device(d)
    ctx = lno_ot.Context(0, prec)
    got = (ctx.energy_central(dd, 0, dev(Ua), s, w), ctx.energy_central(dd, 1, dev(Ub), s, w))
    ctx.close()
    for x in (0, 1):
        np.testing.assert_allclose(got[x], ref[x], rtol=0, atol=tol)


def third_partition(nocc, et):
    na, nb = nocc
    out = [np.zeros(na), np.zeros(nb)]
    trips = {c: T.triplets(c, na, nb) for c in CASES}
    sp = {"aaa": (0, 0, 0), "aab": (0, 0, 1), "abb": (1, 1, 0), "bbb": (1, 1, 1)}
    for ci, c in enumerate(CASES):
        for (i, j, k), e in zip(trips[c], et[ci]):
            for p, x in zip((i, j, k), sp[c]):
                out[x][p] += e / 3.0
    return out


def test_semicanonical_limit_is_one_third_of_each_triplet(lib):
    d = config_domain("c0")
    na, nb = d["nocc"]
    lo, hi = L.denominator_range(d)
    s, w = L.trapezoid_rule(lo, hi, 1e-11)
    assert L.quad_error(s, w, lo, hi) < 1e-10
    dd = lno_ot.to_device(d)
    ctx = lno_ot.Context(0, "fp64")
    et = [torch.zeros(max(T.n_triplets(c, na, nb), 1), dtype=torch.float64, device="cuda")
          for c in CASES]
    ctx.energy(dd, e_trip=et)
    ref = third_partition((na, nb), [e[:T.n_triplets(c, na, nb)].cpu().numpy()
                                     for e, c in zip(et, CASES)])
    got = (ctx.energy_central(dd, 0, dev(np.eye(na)), s, w),
           ctx.energy_central(dd, 1, dev(np.eye(nb)), s, w))
    ctx.close()
    for x in (0, 1):
        np.testing.assert_allclose(got[x], ref[x], rtol=1e-9, atol=1e-14)


def test_complete_set_is_a_trace_at_c4_size(lib):
    d = config_domain("c4")
    na, nb = d["nocc"]
    lo, hi = L.denominator_range(d)
    s, w = lno_ot.laplace_quadrature(lo, hi, 1e-2)
    qe = L.quad_error(s, w, lo, hi)
    dd = lno_ot.to_device(d)
    ctx = lno_ot.Context(0, "bf16x10")
    E = ctx.energy(dd)["total"]
    tots = []
    for seed in (None, 11):
        Ua = np.eye(na) if seed is None else orth(na, seed)
        Ub = np.eye(nb) if seed is None else orth(nb, seed + 1)
        tots.append(ctx.energy_central(dd, 0, dev(Ua), s, w).sum()
                    + ctx.energy_central(dd, 1, dev(Ub), s, w).sum())
    ctx.close()
    assert abs(tots[0] - tots[1]) <= 1e-10 * abs(E), tots
    assert abs(tots[0] - E) <= 1.5 * qe * abs(E), (tots[0], E, qe)
    print("c4 Laplace total", tots, "E(T)", E, "quadrature error", qe, "points", len(s))
