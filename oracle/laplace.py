"""Laplace-transformed (T) share of one central LMO -- plain CPU oracle.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module; the library never
does.  It shares no code with the CUDA path.

What it computes (arXiv 2311.10048, Sec. 3.7, eqs laplace_transform and
local_pt).  With Delta = -D = e_a + e_b + e_c - e_i - e_j - e_k > 0 the
denominator is replaced by a quadrature of its Laplace integral,

    1/Delta = int_0^inf exp(-Delta s) ds  ~  sum_q w_q exp(-Delta s_q),

so that W (W + V) / D ~ -sum_q w_q Wbar_q (Wbar_q + Vbar_q), where the bar
multiplies every occupied index p of W and V by exp(+e_p s_q / 2) and every
virtual index x by exp(-e_x s_q / 2).  After that factorisation the sum over
the first occupied index is a trace and can be taken in any orthonormal
occupied basis; the share of a central localized orbital u (coefficients
u_i in the semicanonical occupied orbitals of its spin) is eq local_pt:

    dE_u = -(1/3) sum_q w_q [ sum_{j<k, a<b<c}  Wbar_ujk (Wbar_ujk + Vbar_ujk)
                             + sum_{j, K, a<b, C} (u and j the same spin)
                             + sum_{J<K, A<B, c}  (u the single spin) ]

with Wbar_u.. = sum_i u_i exp(e_i s_q / 2) Wbar_i.. (W is linear in its first
occupied index; the i-factor of the bar goes with the coefficient).  This
module evaluates exactly that: the semicanonical W and V of every needed
(i, j, k) from ``oracle.triples`` (pinned against the spin-orbital
definition), the linear combination over i, the bar factors and the
restricted sums of eq local_pt.

The partition of a mixed triplet is eq local_pt's: 1/3 of it to each of its
three orbitals (eq cim_pt_energy's 1/8 prefactors would give 1/4, 1/4, 1/2;
both add up to E(T) over a complete set of orbitals).

The quadrature itself (``quadrature``) is not given by the paper beyond its
threshold laptol = 1e-2 (Table thresholds) and "3(-4) points": here it is the
smallest exponential sum whose largest relative error for 1/x on the
denominator range is at most the tolerance, found by least squares on the
relative error with Lawson reweighting towards the minimax fit.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .triples import Evaluator, as_tensors

_f64 = torch.float64


def quad_error(s, w, xmin, xmax, npts=4000):
    """Largest |1 - x sum_q w_q exp(-x s_q)| on a dense log grid of [xmin, xmax]."""
    x = np.geomspace(xmin, xmax, npts)
    r = 1.0 - x * (np.exp(-np.outer(x, np.asarray(s))) @ np.asarray(w))
    return float(np.abs(r).max())


def trapezoid_rule(xmin, xmax, eps):
    """(s, w) from the trapezoid rule on 1/x = int exp(t - x e^t) dt (s = e^t):
    nodes t_k = t_lo + k h, weights h e^{t_k}.  The step h = pi^2 / ln(4/eps)
    bounds the discretisation error by ~eps; t_lo = ln(eps / (2 xmax)) and
    t_hi = ln(ln(2/eps) / xmin) bound the two truncation errors.  Many points,
    but every accuracy is reachable (used for the convergence pins)."""
    h = math.pi ** 2 / math.log(4.0 / eps)
    lo = math.log(eps / (2.0 * xmax))
    hi = math.log(math.log(2.0 / eps) / xmin)
    n = int(math.ceil((hi - lo) / h)) + 1
    t = lo + h * np.arange(n)
    return np.exp(t), h * np.exp(t)


def quadrature(xmin, xmax, tol, nmax=12):
    """(s, w): the fewest-point exponential sum with relative error <= tol for
    1/x on [xmin, xmax] (0 < xmin < xmax); raises if nmax points do not reach
    it.  Meant for the laptol regime (tol >= ~1e-5)."""
    from scipy.optimize import least_squares
    R = xmax / xmin
    y = np.geomspace(1.0, R, 600)          # fit on [1, R], then rescale

    def resid(p, n, wt):
        q = np.clip(p, -60.0, 30.0)
        s, w = np.exp(q[:n]), np.exp(q[n:])
        return wt * (1.0 - y * (np.exp(-np.outer(y, s)) @ w))

    best = None
    for n in range(1, nmax + 1):
        # start: trapezoid rule of int exp(t - y e^t) dt on a grid of t = log s
        lo, hi = math.log(min(tol, 0.1) / (4.0 * R)), math.log(math.log(1.0 / min(tol, 0.1)) + 1.0)
        t = np.linspace(lo, hi, n) if n > 1 else np.array([0.5 * (lo + hi)])
        h = (hi - lo) / max(n - 1, 1)
        p = np.concatenate([t, t + math.log(h)])
        wt = np.ones_like(y)
        for _ in range(30):                 # Lawson: weights follow the error
            sol = least_squares(resid, p, args=(n, wt), method="lm", xtol=1e-15, ftol=1e-15,
                                max_nfev=2000)
            p = sol.x
            r = np.abs(resid(p, n, np.ones_like(y)))
            wt = wt * (r / r.max()) ** 0.5 + 1e-3
            wt = wt / wt.max()
        p = np.clip(p, -60.0, 30.0)
        s, w = np.exp(p[:n]) / xmin, np.exp(p[n:]) / xmin
        order = np.argsort(s)
        s, w = s[order], w[order]
        err = quad_error(s, w, xmin, xmax)
        if best is None or err < best[2]:
            best = (s, w, err)
        if err <= tol:
            return s, w
    raise ValueError(f"no {nmax}-point quadrature reaches {tol} (best {best[2]:.3g})")


def denominator_range(dom):
    """[Delta_min, Delta_max] over all triples of the domain (both spins)."""
    d = dom if isinstance(dom["B"][0], torch.Tensor) else as_tensors(dom)
    na, nb = d["nocc"]
    eo = torch.cat([d["eps"][0][:na], d["eps"][1][:nb]]).numpy()
    ev = torch.cat([d["eps"][0][na:], d["eps"][1][nb:]]).numpy()
    eo, ev = np.sort(eo), np.sort(ev)
    return float(ev[:3].sum() - eo[-3:].sum()), float(ev[-3:].sum() - eo[:3].sum())


# eq local_pt: every restricted term of a central orbital enters with 1/3
_SHARE = 1.0 / 3.0


def _bars(eps, no, sq):
    """Laplace bars of one quadrature point: exp(+e_p s/2) for the occupied
    orbitals, exp(-e_x s/2) for the virtual ones, per spin."""
    ho = [torch.exp(eps[x][:no[x]] * (sq / 2)) for x in (0, 1)]
    hv = [torch.exp(-eps[x][no[x]:] * (sq / 2)) for x in (0, 1)]
    return ho, hv


class _Central:
    """Semicanonical W, V of the domain (cached per (i, j, k)) and the bars."""

    def __init__(self, dom):
        self.ev = Evaluator(dom)
        self.d = self.ev.d
        self._w = {}

    def same(self, s, i, j, k):
        key = ("S", s, i, j, k)
        if key not in self._w:
            self._w[key] = self.ev.same_spin_wv(s, i, j, k)
        return self._w[key]

    def mixed(self, s, i, j, K):
        key = ("M", s, i, j, K)
        if key not in self._w:
            self._w[key] = self.ev.mixed_wv(s, i, j, K)
        return self._w[key]


def central_energy(dom, spin, U, s, w, _central=None):
    """dE of eq local_pt for each central LMO (row of U [nlmo][nocc[spin]])
    of spin ``spin``, with quadrature points s and weights w.  Returns a numpy
    array [nlmo]."""
    C = _central or _Central(dom)
    d = C.d
    sg, tg = spin, 1 - spin
    no = d["nocc"]
    eps = [d["eps"][0], d["eps"][1]]
    U = torch.as_tensor(np.asarray(U), dtype=_f64)
    out = np.zeros(U.shape[0])
    with torch.no_grad():
        for sq, wq in zip(np.asarray(s, dtype=np.float64), np.asarray(w, dtype=np.float64)):
            ho, hv = _bars(eps, no, sq)
            coef = U * ho[sg][None, :]                                     # u_i exp(e_i s/2)
            for l in range(U.shape[0]):
                c = coef[l]
                acc = 0.0
                # (1) u with two more orbitals of its spin: j < k, a < b < c
                nv = hv[sg].numel()
                ar = torch.arange(nv)
                m3 = (ar[:, None, None] < ar[None, :, None]) & (ar[None, :, None] < ar[None, None, :])
                for j in range(no[sg]):
                    for k in range(j + 1, no[sg]):
                        Wb = torch.zeros(nv, nv, nv, dtype=_f64)
                        Vb = torch.zeros_like(Wb)
                        for i in range(no[sg]):
                            if i in (j, k) or c[i] == 0:
                                continue
                            W, V = C.same(sg, i, j, k)
                            Wb += c[i] * W
                            Vb += c[i] * V
                        f = ho[sg][j] * ho[sg][k] * hv[sg][:, None, None] * hv[sg][None, :, None] \
                            * hv[sg][None, None, :]
                        Wb, Vb = Wb * f, Vb * f
                        acc += float((Wb * (Wb + Vb))[m3].sum())
                # (2) u and j of its spin, K of the other: a < b (spin sg), C
                nvs, nvt = hv[sg].numel(), hv[tg].numel()
                ar = torch.arange(nvs)
                m2 = (ar[:, None] < ar[None, :])[:, :, None].expand(nvs, nvs, nvt)
                for j in range(no[sg]):
                    for K in range(no[tg]):
                        Wb = torch.zeros(nvs, nvs, nvt, dtype=_f64)
                        Vb = torch.zeros_like(Wb)
                        for i in range(no[sg]):
                            if i == j or c[i] == 0:
                                continue
                            W, V = C.mixed(sg, i, j, K)
                            Wb += c[i] * W
                            Vb += c[i] * V
                        f = ho[sg][j] * ho[tg][K] * hv[sg][:, None, None] * hv[sg][None, :, None] \
                            * hv[tg][None, None, :]
                        Wb, Vb = Wb * f, Vb * f
                        acc += float((Wb * (Wb + Vb))[m2].sum())
                # (3) u the single orbital of its spin with J < K of the other: A < B, c
                ar = torch.arange(nvt)
                m2t = (ar[:, None] < ar[None, :])[:, :, None].expand(nvt, nvt, nvs)
                for J in range(no[tg]):
                    for K in range(J + 1, no[tg]):
                        Wb = torch.zeros(nvt, nvt, nvs, dtype=_f64)
                        Vb = torch.zeros_like(Wb)
                        for i in range(no[sg]):
                            if c[i] == 0:
                                continue
                            W, V = C.mixed(tg, J, K, i)
                            Wb += c[i] * W
                            Vb += c[i] * V
                        f = ho[tg][J] * ho[tg][K] * hv[tg][:, None, None] * hv[tg][None, :, None] \
                            * hv[sg][None, None, :]
                        Wb, Vb = Wb * f, Vb * f
                        acc += float((Wb * (Wb + Vb))[m2t].sum())
                out[l] += -wq * acc * _SHARE
    return out


def central_energies(dom, Ua, Ub, s, w):
    """dE of every row of Ua (spin up LMOs) and Ub (spin down LMOs)."""
    C = _Central(dom)
    return (central_energy(dom, 0, Ua, s, w, C), central_energy(dom, 1, Ub, s, w, C))
