"""Natural auxiliary functions (NAF) of a domain -- plain CPU oracle.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module; the library never
does.  It shares no code with the CUDA path.

What it computes (arXiv 2311.10048, Sec. 3.6, eq naf_w): for each spin the
matrix of the three-centre integrals over the orbital pairs p <= q of the
domain,

    W^s_XY = sum_{p <= q} (pq|X) (pq|Y),      here (pq|X) = B^X_pq,

their spin average W = (W^up + W^down) / 2 (one auxiliary basis for both
spins, as the mixed-spin integrals need), its eigenvectors with eigenvalues
above eps_naf as the NAFs, and the compressed factors

    B'^{X'}_pq = sum_X V_{X X'} B^X_pq    (X' over the kept eigenvectors),

so that sum_{X'} B'_pq B'_rs = sum_{XY} B_pq (V V^T)_{XY} B_rs approximates
(pq|rs).  The eigen-decomposition is numpy's (a library routine as one step).
"""
from __future__ import annotations

import numpy as np


def naf_w(B):
    """W_XY = sum_{p<=q} B^X_pq B^Y_pq for one spin, B [naux][n][n] symmetric."""
    naux, n, _ = B.shape
    iu = np.triu_indices(n)
    J = B[:, iu[0], iu[1]]                # [naux][pairs p <= q]
    return J @ J.T


def naf(B_up, B_down, eps_naf):
    """(eigenvalues descending, V [naux][nkept], B' up, B' down) of Sec. 3.6."""
    W = 0.5 * (naf_w(B_up) + naf_w(B_down))
    lam, U = np.linalg.eigh(W)
    order = np.argsort(lam)[::-1]
    lam, U = lam[order], U[:, order]
    keep = lam > eps_naf
    V = U[:, keep]
    naux, n, _ = B_up.shape

    def compress(B):
        return (V.T @ B.reshape(naux, -1)).reshape(V.shape[1], n, n)
    return lam, V, compress(B_up), compress(B_down)


def compressed_domain(dom, eps_naf):
    """Copy of a domain dict with both B factors replaced by their NAF
    compression (naux -> the number of kept NAFs)."""
    lam, V, Bu, Bd = naf(np.asarray(dom["B"][0]), np.asarray(dom["B"][1]), eps_naf)
    out = dict(dom)
    out["B"] = [Bu, Bd]
    out["naux"] = int(V.shape[1])
    return out, lam
