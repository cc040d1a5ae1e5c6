"""Pins of the NAF oracle (Sec. 3.6, eq naf_w) against independent facts:

* W^s is the sum over p <= q written out by explicit loops (tiny case);
* closed-shell limit: identical spin-up and spin-down factors give the NAFs of
  W^up itself (the 1/2 in the spin average), as the paper notes;
* eps_naf = 0 keeps everything and the four-index integrals, hence E(T), are
  unchanged; the trace of W equals sum_{p<=q} sum_X B^2;
* truncation: the four-index integrals are a projection (idempotent), their
  error is bounded through the dropped eigenvalues, and E(T) of the
  compressed domain approaches E(T) as eps_naf decreases.
"""
import numpy as np
import pytest

from oracle import naf as N
from oracle import triples as T
from paper_2311_10048_gb300.synth import make_domain


def dom(seed=1, nbas=10, nocc=(3, 2), naux=24, L=4.0):
    return make_domain(nbas, nocc, naux=naux, L=L, seed=seed, t1_sd=0.02)


def test_w_equals_explicit_pair_sum():
    d = dom()
    B = d["B"][0]
    naux, n, _ = B.shape
    W = np.zeros((naux, naux))
    for p in range(n):
        for q in range(p, n):
            W += np.outer(B[:, p, q], B[:, p, q])
    np.testing.assert_allclose(N.naf_w(B), W, rtol=1e-13, atol=1e-15)
    assert abs(np.trace(W) - sum((B[:, p, q] ** 2).sum() for p in range(n)
                                 for q in range(p, n))) < 1e-12 * np.trace(W)


def test_closed_shell_limit_uses_the_spin_up_nafs():
    d = make_domain(10, (3, 3), naux=24, L=4.0, seed=2, closed_shell=True)
    lam, V, _, _ = N.naf(d["B"][0], d["B"][1], 1e-3)
    lam1, U1 = np.linalg.eigh(N.naf_w(d["B"][0]))
    lam1 = np.sort(lam1)[::-1]
    np.testing.assert_allclose(lam, lam1, rtol=1e-12, atol=1e-14)
    keep = lam1 > 1e-3
    P = V @ V.T
    U1 = U1[:, np.argsort(np.linalg.eigh(N.naf_w(d["B"][0]))[0])[::-1]][:, keep]
    np.testing.assert_allclose(P, U1 @ U1.T, atol=1e-10)


def test_zero_threshold_keeps_the_integrals_and_energy():
    d = dom(3)
    c, lam = N.compressed_domain(d, 0.0)
    assert c["naux"] == d["naux"]
    for s in (0, 1):
        B, Bc = d["B"][s], c["B"][s]
        g = np.einsum("Xpq,Xrs->pqrs", B, B)
        gc = np.einsum("Xpq,Xrs->pqrs", Bc, Bc)
        np.testing.assert_allclose(gc, g, atol=1e-12)
    assert abs(T.energy(c)["total"] - T.energy(d)["total"]) < 1e-12 * abs(T.energy(d)["total"])


def test_truncation_is_a_projection_and_converges():
    d = dom(4, naux=30, L=3.0)
    E = T.energy(d)["total"]
    prev = None
    for eps in (1e-1, 1e-3, 1e-6):
        c, lam = N.compressed_domain(d, eps)
        assert c["naux"] == int((lam > eps).sum()) and c["naux"] < d["naux"]
        # (pq|rs) with the kept NAFs: sum_XY B (V V^T) B; V V^T idempotent
        _, V, _, _ = N.naf(d["B"][0], d["B"][1], eps)
        P = V @ V.T
        np.testing.assert_allclose(P @ P, P, atol=1e-12)
        # the discarded part of W^avg is bounded by the dropped eigenvalues
        W = 0.5 * (N.naf_w(d["B"][0]) + N.naf_w(d["B"][1]))
        R = W - P @ W @ P
        assert np.linalg.norm(R, 2) <= lam[lam <= eps].max() * (1 + 1e-9)
        err = abs(T.energy(c)["total"] - E)
        if prev is not None:
            assert err < prev
        prev = err
    assert prev < 1e-6 * abs(E)
