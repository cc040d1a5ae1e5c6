"""Pins of the Laplace-transformed central-LMO oracle (Sec. 3.7, eqs
laplace_transform and local_pt) against independent statements:

* the quadrature really bounds the relative error of 1/x on the range;
* the spin-case restricted sums equal the spin-orbital definition (first
  occupied index of the 1/36 sum) for rotated central orbitals;
* in the semicanonical basis with an accurate quadrature, each orbital's share
  is 1/3 of every triplet it belongs to (per-triplet values of the triples
  oracle, itself pinned by spin-orbital brute force);
* over a complete orthonormal set the shares add up to the same number for
  every rotation (a trace), and to E(T) as the quadrature gets accurate;
* a planted mistake in the bars or in the share fails the pins.
"""
import math

import numpy as np
import pytest

from oracle import laplace as L
from oracle import triples as T
from oracle.spinorbital import central_energy_brute
from paper_2311_10048_gb300.synth import config_domain, make_domain

CASES = ("aaa", "aab", "abb", "bbb")


def tiny(nbas, na, nb, seed):
    return make_domain(nbas, (na, nb), naux=20, L=10.0, seed=seed, t1_sd=0.05)


def orth(n, seed):
    if n == 0:
        return np.zeros((0, 0))
    q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((n, n)))
    return q.T


def third_partition(d):
    """1/3 of every restricted triplet to each of its orbitals."""
    na, nb = d["nocc"]
    out = [np.zeros(na), np.zeros(nb)]
    for c in CASES:
        for (i, j, k), e in zip(T.triplets(c, na, nb), T.triplet_energies(d, c)):
            sp = {"aaa": (0, 0, 0), "aab": (0, 0, 1), "abb": (1, 1, 0), "bbb": (1, 1, 1)}[c]
            for p, x in zip((i, j, k), sp):
                out[x][p] += e / 3.0
    return out


@pytest.mark.parametrize("rng_", [(1.2, 21.0), (0.5, 40.0), (3.9, 16.1)])
@pytest.mark.parametrize("tol", [1e-2, 1e-3])
def test_quadrature_bounds_the_relative_error(rng_, tol):
    lo, hi = rng_
    s, w = L.quadrature(lo, hi, tol)
    assert L.quad_error(s, w, lo, hi) <= tol
    assert (s > 0).all() and (w > 0).all()
    if tol == 1e-2 and hi / lo < 20:
        assert len(s) <= 4          # the paper's "3(-4) points" at laptol = 1e-2


@pytest.mark.parametrize("eps", [1e-4, 1e-8, 1e-12])
def test_trapezoid_rule_accuracy(eps):
    s, w = L.trapezoid_rule(1.2, 21.0, eps)
    assert L.quad_error(s, w, 1.2, 21.0) <= 10 * eps


@pytest.mark.parametrize("shape", [(9, 3, 2, 5), (8, 3, 1, 6), (9, 2, 2, 7)])
def test_spin_case_sums_equal_spin_orbital_definition(shape):
    nbas, na, nb, seed = shape
    d = tiny(nbas, na, nb, seed)
    lo, hi = L.denominator_range(d)
    s, w = L.quadrature(lo, hi, 1e-2)
    for spin, n in ((0, na), (1, nb)):
        U = orth(n, seed + spin)[: max(1, n - 1)]
        got = L.central_energy(d, spin, U, s, w)
        ref = central_energy_brute(d, spin, U, s, w)
        for g, r in zip(got, ref):
            assert abs(g - r) <= 1e-13 + 1e-11 * abs(r), (spin, got, ref)


@pytest.mark.parametrize("shape", [(11, 3, 2, 3), (10, 4, 2, 4)])
def test_semicanonical_limit_is_one_third_of_each_triplet(shape):
    nbas, na, nb, seed = shape
    d = make_domain(nbas, (na, nb), naux=24, L=8.0, seed=seed, t1_sd=0.02)
    lo, hi = L.denominator_range(d)
    s, w = L.trapezoid_rule(lo, hi, 1e-12)
    got = L.central_energies(d, np.eye(na), np.eye(nb), s, w)
    ref = third_partition(d)
    for x in (0, 1):
        np.testing.assert_allclose(got[x], ref[x], rtol=1e-9, atol=1e-15)


def test_complete_set_is_a_trace_and_converges_to_full_energy():
    d = make_domain(11, (3, 2), naux=24, L=8.0, seed=3, t1_sd=0.02)
    E = T.energy(d)["total"]
    lo, hi = L.denominator_range(d)
    prev = None
    for eps in (1e-2, 1e-5, 1e-10):
        s, w = L.trapezoid_rule(lo, hi, eps)
        qe = L.quad_error(s, w, lo, hi)
        a0, b0 = L.central_energies(d, np.eye(3), np.eye(2), s, w)
        a1, b1 = L.central_energies(d, orth(3, 1), orth(2, 2), s, w)
        tot0, tot1 = a0.sum() + b0.sum(), a1.sum() + b1.sum()
        assert abs(tot0 - tot1) <= 1e-12 * abs(tot0)          # invariant to the rotation
        assert abs(tot0 - E) <= 1.5 * qe * abs(E)            # quadrature error bound
        if prev is not None:
            assert abs(tot0 - E) < prev
        prev = abs(tot0 - E)
    assert prev <= 1e-9 * abs(E)


@pytest.mark.parametrize("mistake", ["no_occupied_bar", "share_quarter"])
def test_planted_mistakes_are_caught(mistake, monkeypatch):
    d = tiny(9, 3, 2, 5)
    lo, hi = L.denominator_range(d)
    s, w = L.quadrature(lo, hi, 1e-2)
    U = orth(3, 9)
    ref = central_energy_brute(d, 0, U, s, w)
    if mistake == "no_occupied_bar":
        old = L._bars

        def bars(eps, no, sq):
            ho, hv = old(eps, no, sq)
            return [x * 0 + 1 for x in ho], hv
        monkeypatch.setattr(L, "_bars", bars)
    else:
        monkeypatch.setattr(L, "_SHARE", 0.25)
    got = L.central_energy(d, 0, U, s, w)
    assert max(abs(g - r) / abs(r) for g, r in zip(got, ref)) > 1e-3
