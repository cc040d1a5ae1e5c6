"""Closed-shell (RHF) (T) energy -- independent formula for the closed-shell pin.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

arXiv 2311.10048 states that the open-shell method is identical to its
closed-shell counterpart for closed-shell systems (Sec. 8, Summary) and that
the NAF step reduces to the closed-shell one in that limit (Sec. 3.6).  The
closed-shell (T) energy used here is the textbook spin-adapted expression
(the CCSD(T) reference of eq cim_pt_energy) in spatial orbitals:

  W^{abc}_{ijk} = P [ sum_d (bd|ai) t^{cd}_{kj} - sum_l (ck|jl) t^{ab}_{il} ]
  V^{abc}_{ijk} = W^{abc}_{ijk} + (bj|ck) t^a_i + (ai|ck) t^b_j + (ai|bj) t^c_k
  E = 1/3 sum_{ijkabc} (4 W_abc + W_bca + W_cab)(V_abc - V_cba) / D

where P sums the six simultaneous permutations of the pairs (ai),(bj),(ck),
t^{ab}_{ij} are the spin-adapted (alpha-beta) doubles, and all index sums run
over all occupied / virtual orbitals.  No spin-orbital or spin-case algebra
is shared with ``oracle.triples``.
"""
from __future__ import annotations

import itertools

import torch

from .triples import as_tensors

_f64 = torch.float64


def rhf_energy(dom):
    """Closed-shell E(T) of a domain whose two spins carry identical data.

    Uses the spin-up factors/energies/T1 and t2ab as the closed-shell doubles.
    """
    d = dom if isinstance(dom["B"][0], torch.Tensor) else as_tensors(dom)
    na, nb = d["nocc"]
    if na != nb:
        raise ValueError("closed-shell formula needs nocc[0] == nocc[1]")
    with torch.no_grad():
        B, eps, t1, t2 = d["B"][0], d["eps"][0], d["t1"][0], d["t2ab"]
        no = na
        o, v = slice(0, no), slice(no, B.shape[1])

        def eri(p, q, r, s):
            L, R = B[:, p, q], B[:, r, s]
            return torch.einsum("Qpq,Qrs->pqrs", L, R)

        g_vvvo = eri(v, v, v, o)     # (bd|ai) -> [b][d][a][i]
        g_vooo = eri(v, o, o, o)     # (ck|jl) -> [c][k][j][l]
        g_vovo = eri(v, o, v, o)     # (ai|bj) -> [a][i][b][j]
        # w0[i,j,k,a,b,c] = sum_d (bd|ai) t^{cd}_{kj} - sum_l (ck|jl) t^{ab}_{il}
        w0 = torch.einsum("bdai,kjcd->ijkabc", g_vvvo, t2) \
            - torch.einsum("ckjl,ilab->ijkabc", g_vooo, t2)
        W = torch.zeros_like(w0)
        for p in itertools.permutations(range(3)):
            W = W + w0.permute(*p, *(3 + q for q in p))
        V = W + torch.einsum("bjck,ia->ijkabc", g_vovo, t1) \
              + torch.einsum("aick,jb->ijkabc", g_vovo, t1) \
              + torch.einsum("aibj,kc->ijkabc", g_vovo, t1)
        eo, ev = eps[o], eps[v]
        D = (eo[:, None, None, None, None, None] + eo[None, :, None, None, None, None]
             + eo[None, None, :, None, None, None] - ev[None, None, None, :, None, None]
             - ev[None, None, None, None, :, None] - ev[None, None, None, None, None, :])
        Wbca = W.permute(0, 1, 2, 5, 3, 4)     # [..,a,b,c] -> W[..,b,c,a]
        Wcab = W.permute(0, 1, 2, 4, 5, 3)     # [..,a,b,c] -> W[..,c,a,b]
        Vcba = V.permute(0, 1, 2, 5, 4, 3)     # [..,a,b,c] -> V[..,c,b,a]
        E = ((4.0 * W + Wbca + Wcab) * (V - Vcba) / D).sum() / 3.0
        return float(E)
