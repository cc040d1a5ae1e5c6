"""Spin-orbital (T) energy by explicit enumeration -- tiny inputs only.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

This is the definition behind eq cim_pt_energy of arXiv 2311.10048 (Sec. 2.1,
"conventional unrestricted ... (T) energy expressions" with W = t D), written
out over spin orbitals with no spin-case algebra at all:

  <pq||rs> = <pq|rs> - <pq|sr>,  <pq|rs> = (pr|qs) delta(s_p,s_r) delta(s_q,s_s)
  W^{abc}_{ijk} = P(i/jk) P(a/bc) [ sum_e t^{ae}_{jk} <ei||bc>
                                    - sum_m t^{bc}_{im} <ma||jk> ]
  V^{abc}_{ijk} = P(i/jk) P(a/bc) [ t^a_i <jk||bc> + f_ia t^{bc}_{jk} ]
  E = 1/36 sum_{ijkabc} W (W + V) / D

(f_ia: the optional occupied-virtual Fock block of an RO reference, zero
when the domain has no ``fov``.)  ``orbital_partition`` applies the
prefactors of eq cim_pt_energy (1/36 same spin, 1/8 mixed) to these
spin-orbital tensors.

All occupied (i,j,k) and virtual (a,b,c) spin orbitals are enumerated, so the
tensors hold n_occ^3 n_vir^3 numbers: keep nbas <= 12.
"""
from __future__ import annotations

import torch

from .triples import as_tensors

_f64 = torch.float64


def _orbitals(d):
    """Spin orbitals as (spin, spatial index) lists: occupied, then virtual."""
    na, nb = d["nocc"]
    n = d["nbas"]
    occ = [(0, p) for p in range(na)] + [(1, p) for p in range(nb)]
    vir = [(0, p) for p in range(na, n)] + [(1, p) for p in range(nb, n)]
    return occ, vir


def _chem(d, P, Q, R, S):
    """(pq|rs) over spin-orbital lists with the spin deltas of <pr|qs>.

    Returns g[p][q][r][s] = (pq|rs) if spin(p)==spin(q) and spin(r)==spin(s),
    else 0.
    """
    g = torch.zeros(len(P), len(Q), len(R), len(S), dtype=_f64)
    B = d["B"]
    for a, (sp, p) in enumerate(P):
        for b, (sq, q) in enumerate(Q):
            if sp != sq:
                continue
            lhs = B[sp][:, p, q]
            for c, (sr, r) in enumerate(R):
                for e, (ss, s) in enumerate(S):
                    if sr != ss:
                        continue
                    g[a, b, c, e] = lhs @ B[sr][:, r, s]
    return g


def _anti(d, P, Q, R, S):
    """<pq||rs> = (pr|qs) - (ps|qr), as a [p][q][r][s] tensor."""
    pr_qs = _chem(d, P, R, Q, S).permute(0, 2, 1, 3)    # [p][q][r][s]
    ps_qr = _chem(d, P, S, Q, R).permute(0, 2, 3, 1)    # [p][q][r][s]
    return pr_qs - ps_qr


def _amplitudes(d, occ, vir):
    """Spin-orbital T1 [i][a] and antisymmetric T2 [i][j][a][b]."""
    na, nb = d["nocc"]
    no, nv = len(occ), len(vir)
    t1 = torch.zeros(no, nv, dtype=_f64)
    t2 = torch.zeros(no, no, nv, nv, dtype=_f64)
    for I, (si, i) in enumerate(occ):
        for A, (sa, a) in enumerate(vir):
            if si == sa:
                t1[I, A] = d["t1"][si][i, a - d["nocc"][si]]
    for I, (si, i) in enumerate(occ):
        for J, (sj, j) in enumerate(occ):
            for A, (sa, a) in enumerate(vir):
                for Bv, (sb, b) in enumerate(vir):
                    va = a - d["nocc"][sa]
                    vb = b - d["nocc"][sb]
                    if si == sj == sa == sb == 0:
                        v = d["t2aa"][i, j, va, vb]
                    elif si == sj == sa == sb == 1:
                        v = d["t2bb"][i, j, va, vb]
                    elif (si, sj, sa, sb) == (0, 1, 0, 1):
                        v = d["t2ab"][i, j, va, vb]
                    elif (si, sj, sa, sb) == (1, 0, 1, 0):
                        v = d["t2ab"][j, i, vb, va]
                    elif (si, sj, sa, sb) == (0, 1, 1, 0):
                        v = -d["t2ab"][i, j, vb, va]
                    elif (si, sj, sa, sb) == (1, 0, 0, 1):
                        v = -d["t2ab"][j, i, va, vb]
                    else:
                        continue
                    t2[I, J, A, Bv] = v
    return t1, t2


def _fock_ov(d, occ, vir):
    """Spin-orbital f_ia [i][a] (zero across spins, zero without ``fov``)."""
    f = torch.zeros(len(occ), len(vir), dtype=_f64)
    if d.get("fov") is None:
        return f
    for I, (si, i) in enumerate(occ):
        for A, (sa, a) in enumerate(vir):
            if si == sa:
                f[I, A] = d["fov"][si][i, a - d["nocc"][si]]
    return f


def _p3(x, axes):
    """P(p/qr) on three axes of x: f(pqr) - f(qpr) - f(rqp)."""
    p, q, r = axes
    return x - x.transpose(p, q) - x.transpose(p, r)


def brute_force(dom, return_tensors=False):
    """E(T) from the spin-orbital definition, split by the spin of (ijk).

    Returns {"aaa","aab","abb","bbb","total"}: the occupied-spin pattern with
    0, 1, 2, 3 spin-down orbitals among i,j,k (spin conservation makes the
    virtual pattern match).
    """
    d = dom if isinstance(dom["B"][0], torch.Tensor) else as_tensors(dom)
    with torch.no_grad():
        occ, vir = _orbitals(d)
        t1, t2 = _amplitudes(d, occ, vir)
        ei_bc = _anti(d, vir, occ, vir, vir)          # <ei||bc> [e][i][b][c]
        ma_jk = _anti(d, occ, vir, occ, occ)          # <ma||jk> [m][a][j][k]
        jk_bc = _anti(d, occ, occ, vir, vir)          # <jk||bc> [j][k][b][c]
        # indices of the 6-index tensors: [i][j][k][a][b][c]
        c = torch.einsum("jkae,eibc->ijkabc", t2, ei_bc) \
            - torch.einsum("imbc,majk->ijkabc", t2, ma_jk)
        W = _p3(_p3(c, (0, 1, 2)), (3, 4, 5))
        v = torch.einsum("ia,jkbc->ijkabc", t1, jk_bc) \
            + torch.einsum("ia,jkbc->ijkabc", _fock_ov(d, occ, vir), t2)
        V = _p3(_p3(v, (0, 1, 2)), (3, 4, 5))
        eo = torch.stack([d["eps"][s][p] for s, p in occ])
        ev = torch.stack([d["eps"][s][p] for s, p in vir])
        D = (eo[:, None, None, None, None, None] + eo[None, :, None, None, None, None]
             + eo[None, None, :, None, None, None] - ev[None, None, None, :, None, None]
             - ev[None, None, None, None, :, None] - ev[None, None, None, None, None, :])
        E = W * (W + V) / D / 36.0
        spin = torch.tensor([s for s, _ in occ])
        nbeta = spin[:, None, None] + spin[None, :, None] + spin[None, None, :]
        out = {}
        for nb_, name in enumerate(("aaa", "aab", "abb", "bbb")):
            out[name] = float(E[nbeta == nb_].sum())
        out["total"] = float(E.sum())
        if return_tensors:
            return out, dict(W=W, V=V, D=D, occ=occ, vir=vir)
        return out


def orbital_partition(dom):
    """Orbital contributions written out from eq cim_pt_energy over spin
    orbitals: for an occupied orbital p of spin s (t the other spin),

      dE_p = 1/36 sum_{jk abc, all spin s} E6[p,j,k,a,b,c]
           + 1/8 sum_{a (s); J,K,B,C (t)} E6[p,J,K,a,B,C]
           + 1/8 sum_{j,a,b (s); K,C (t)} E6[p,j,K,a,b,C]

    with E6 = W (W + V) / D over unrestricted spin-orbital indices.
    Returns {"alpha": [...], "beta": [...]} (floats).
    """
    d = dom if isinstance(dom["B"][0], torch.Tensor) else as_tensors(dom)
    _, t = brute_force(d, return_tensors=True)
    with torch.no_grad():
        E6 = t["W"] * (t["W"] + t["V"]) / t["D"]
        occ, vir = t["occ"], t["vir"]
        os_ = torch.tensor([s for s, _ in occ])
        vs_ = torch.tensor([s for s, _ in vir])
        res = {"alpha": [], "beta": []}
        for I, (s, p) in enumerate(occ):
            o_s, o_t = os_ == s, os_ != s
            v_s, v_t = vs_ == s, vs_ != s
            e = E6[I]                                        # [j][k][a][b][c]
            same = e[o_s][:, o_s][:, :, v_s][:, :, :, v_s][:, :, :, :, v_s].sum() / 36.0
            two_t = e[o_t][:, o_t][:, :, v_s][:, :, :, v_t][:, :, :, :, v_t].sum() / 8.0
            one_t = e[o_s][:, o_t][:, :, v_s][:, :, :, v_s][:, :, :, :, v_t].sum() / 8.0
            res["alpha" if s == 0 else "beta"].append(float(same + two_t + one_t))
        return res


def central_energy_brute(dom, spin, U, s, w):
    """eq local_pt written out over spin orbitals (tiny inputs only).

    For a central orbital u = sum_i U[l, i] phi_i (i over the occupied
    orbitals of ``spin``) and the quadrature (s_q, w_q) of eq laplace_transform:

      dE_u = -sum_q w_q (1/36) sum_{jkabc} Wbar_u (Wbar_u + Vbar_u),
      Wbar_u[jkabc] = sum_i U[l,i] e^{e_i s_q/2} W[ijkabc] e^{(e_j+e_k) s_q/2}
                      e^{-(e_a+e_b+e_c) s_q/2}

    over unrestricted spin-orbital j, k, a, b, c (the first-index share of the
    1/36 sum of the definition, whose denominators the quadrature replaces).
    Returns a list [nlmo].
    """
    d = dom if isinstance(dom["B"][0], torch.Tensor) else as_tensors(dom)
    _, t = brute_force(d, return_tensors=True)
    W, V, occ, vir = t["W"], t["V"], t["occ"], t["vir"]
    U = torch.as_tensor(U, dtype=_f64)
    eo = torch.stack([d["eps"][x][p] for x, p in occ])
    ev = torch.stack([d["eps"][x][p] for x, p in vir])
    rows = [I for I, (x, _) in enumerate(occ) if x == spin]   # occupied spin orbitals of `spin`
    out = [0.0] * U.shape[0]
    with torch.no_grad():
        for sq, wq in zip(s, w):
            sq, wq = float(sq), float(wq)
            f = (torch.exp(eo * sq / 2)[:, None, None, None, None]
                 * torch.exp(eo * sq / 2)[None, :, None, None, None]
                 * torch.exp(-ev * sq / 2)[None, None, :, None, None]
                 * torch.exp(-ev * sq / 2)[None, None, None, :, None]
                 * torch.exp(-ev * sq / 2)[None, None, None, None, :])
            for l in range(U.shape[0]):
                Wb = torch.zeros_like(W[0])
                Vb = torch.zeros_like(V[0])
                for q, I in enumerate(rows):
                    c = U[l, q] * torch.exp(eo[I] * sq / 2)
                    Wb = Wb + c * W[I]
                    Vb = Vb + c * V[I]
                Wb, Vb = Wb * f, Vb * f
                out[l] += -wq * float((Wb * (Wb + Vb)).sum()) / 36.0
    return out
