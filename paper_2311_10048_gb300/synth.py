"""Seeded synthetic LNO-domain inputs for the open-shell (T) energy.

This module only builds inputs. It holds none of the (T) arithmetic, and both
the GPU path (through its callers) and the CPU oracle receive its arrays as
plain data.

What a domain is (arXiv 2311.10048, Sec. 3.7 "Correlation energy calculation
in the LIS"): semicanonical spin-up / spin-down orbitals of one local
interacting subspace, DF three-centre integrals B^Q_pq with one auxiliary index
shared by both spins (Sec. 3.6, NAF paragraph), orbital energies, and CCSD
T1/T2 amplitudes.  Real amplitudes come from an iterative CCSD solver; here T2
is MP2-like, built from the same B and orbital energies, so that the sizes,
signs and value distributions are those of a real LIS.

Recipe (the same for every configuration; seeds and sizes in ``CONFIGS``):

* ``rng = numpy.random.default_rng(seed)`` (PCG64).  Draw order: spin up
  (B, eps, T1), then spin down (B, eps, T1).
* B^Q_pq: N(0,1) for p <= q (``numpy.triu_indices`` order), mirrored to q < p,
  then scaled by exp(-Q/L)/sqrt(naux).  Orbitals are ordered occupied first,
  then virtual.
* eps: occupied U(-2.0, -0.3), virtual U(0.1, 5.0), each sorted ascending.
* T1 ~ N(0, 1e-3) (standard deviation 1e-3).
* T2 (MP2-like; D2 = e_i + e_j - e_a - e_b < 0):
  t^{ab}_{ij} = [(ia|jb) - (ib|ja)] / D2 for both same-spin blocks and
  t^{aB}_{iJ} = (ia|JB) / D2 for the mixed block, (pq|rs) = sum_Q B_pq B_rs.

Array layouts (all float64, C order):
  B[s]    [naux][nbas][nbas]      s = 0 spin up, 1 spin down
  eps[s]  [nbas]
  t1[s]   [nocc[s]][nvir[s]]
  t2aa    [na][na][nva][nva]      antisymmetric in (i,j) and in (a,b)
  t2bb    [nb][nb][nvb][nvb]
  t2ab    [na][nb][nva][nvb]      t2ab[i][J][a][B] = t^{aB}_{iJ}
"""
from __future__ import annotations

import math

import numpy as np

# Single-domain workloads.  L is the decay length of B along Q.
CONFIGS = {
    # small single domain (runs everywhere in seconds)
    "c0": dict(nbas=40, nocc=(6, 4), naux=120, L=40.0, seed=0),
    # medium single domain
    "c1": dict(nbas=400, nocc=(40, 38), naux=1200, L=300.0, seed=1),
    # large single domain (precision study)
    "c2": dict(nbas=700, nocc=(80, 78), naux=2100, L=525.0, seed=2),
    # differentiation domain
    "c4": dict(nbas=200, nocc=(20, 18), naux=600, L=150.0, seed=4),
}

C3_SEED = 3
C3_NDOM = 2000


def c3_shapes(ndom: int = C3_NDOM, seed: int = C3_SEED):
    """Shapes of the 2000-domain batch (LIS statistics of the paper's large runs).

    n_a = clip(round(lognormal(ln 25, 0.5)), 8, 60); n_b = n_a - U{1,2,3};
    nvir = clip(round(8 n_a U(0.8, 1.2)), 60, 400); nbas = n_a + nvir;
    naux = 3 (n_a + nvir); L = naux / 4; domain d uses seed 3*10^6 + d.
    """
    rng = np.random.default_rng(seed)
    out = []
    for d in range(ndom):
        na = int(np.clip(round(rng.lognormal(math.log(25.0), 0.5)), 8, 60))
        nb = na - int(rng.integers(1, 4))
        nvir = int(np.clip(round(8 * na * rng.uniform(0.8, 1.2)), 60, 400))
        nbas = na + nvir
        naux = 3 * (na + nvir)
        out.append(dict(nbas=nbas, nocc=(na, nb), naux=naux, L=naux / 4.0,
                        seed=3_000_000 + d))
    return out


def _draw_spin(rng, nbas, nocc, naux, L, t1_sd):
    iu = np.triu_indices(nbas)
    B = np.empty((naux, nbas, nbas))
    vals = rng.standard_normal((naux, iu[0].size))
    B[:, iu[0], iu[1]] = vals
    B[:, iu[1], iu[0]] = vals
    B *= (np.exp(-np.arange(naux) / L) / math.sqrt(naux))[:, None, None]
    eo = np.sort(rng.uniform(-2.0, -0.3, nocc))
    ev = np.sort(rng.uniform(0.1, 5.0, nbas - nocc))
    eps = np.concatenate([eo, ev])
    t1 = rng.standard_normal((nocc, nbas - nocc)) * t1_sd
    return B, eps, t1


def _ovov(Bp, op, Bq, oq):
    """(ia|JB) for i,a of spin p and J,B of spin q, shape [op][vp][oq][vq]."""
    naux, nbas, _ = Bp.shape
    L = np.ascontiguousarray(Bp[:, :op, op:]).reshape(naux, -1)
    R = np.ascontiguousarray(Bq[:, :oq, oq:]).reshape(naux, -1)
    return (L.T @ R).reshape(op, nbas - op, oq, nbas - oq)


def make_domain(nbas, nocc, naux, L, seed, t1_sd=1e-3, closed_shell=False):
    """Build one synthetic domain (dict of float64 arrays, layouts above).

    ``closed_shell=True`` (requires nocc[0] == nocc[1]) copies the spin-up
    draws to spin down, which gives a closed-shell (RHF-like) domain.
    """
    na, nb = int(nocc[0]), int(nocc[1])
    if not (0 <= nb <= na <= nbas):
        raise ValueError("need 0 <= nocc[1] <= nocc[0] <= nbas")
    rng = np.random.default_rng(seed)
    Ba, ea, t1a = _draw_spin(rng, nbas, na, naux, L, t1_sd)
    if closed_shell:
        if na != nb:
            raise ValueError("closed_shell needs nocc[0] == nocc[1]")
        Bb, eb, t1b = Ba.copy(), ea.copy(), t1a.copy()
    else:
        Bb, eb, t1b = _draw_spin(rng, nbas, nb, naux, L, t1_sd)
    return dict(nbas=nbas, naux=naux, nocc=(na, nb), B=[Ba, Bb], eps=[ea, eb],
                t1=[t1a, t1b], **mp2_like_t2(Ba, ea, na, Bb, eb, nb))


def add_fov(dom, sd=0.02, seed=0):
    """Copy of ``dom`` with an off-diagonal Fock block per spin.

    ``fov[s]`` [nocc[s]][nvir[s]] ~ N(0, sd), drawn from a generator of its
    own (PCG64 seeded with (seed, 7)) so that every other input of the domain
    stays bit for bit what ``make_domain`` gave.  Stands in for the f_ia of a
    restricted open-shell reference in the semicanonical basis.
    """
    rng = np.random.default_rng([int(seed), 7])
    na, nb = dom["nocc"]
    n = dom["nbas"]
    out = dict(dom)
    out["fov"] = [rng.normal(0.0, sd, size=(na, n - na)), rng.normal(0.0, sd, size=(nb, n - nb))]
    return out


def mp2_like_t2(Ba, ea, na, Bb, eb, nb):
    """MP2-like doubles from B and eps (input recipe, see module docstring).

    The element-wise part runs one first occupied index at a time, so the
    peak host memory is the (ia|jb) block plus the outputs.
    """
    out = {}
    for key, (Bp, ep, op) in (("t2aa", (Ba, ea, na)), ("t2bb", (Bb, eb, nb))):
        g = _ovov(Bp, op, Bp, op)                       # [i][a][j][b]
        eo, ev = ep[:op], ep[op:]
        nv = ev.size
        t2 = np.empty((op, op, nv, nv))
        for i in range(op):
            gi = g[i]                                    # [a][j][b]
            num = gi.transpose(1, 0, 2) - gi.transpose(1, 2, 0)   # [j][a][b]
            d2 = (eo[i] + eo)[:, None, None] - ev[None, :, None] - ev[None, None, :]
            t2[i] = num / d2
        out[key] = t2
        del g
    g = _ovov(Ba, na, Bb, nb)                            # [i][a][J][B]
    eoa, eva, eob, evb = ea[:na], ea[na:], eb[:nb], eb[nb:]
    t2 = np.empty((na, nb, eva.size, evb.size))
    for i in range(na):
        d2 = (eoa[i] + eob)[:, None, None] - eva[None, :, None] - evb[None, None, :]
        t2[i] = g[i].transpose(1, 0, 2) / d2
    out["t2ab"] = t2
    return out


def config_domain(name: str, **over):
    """The single-domain configuration ``name`` ("c0", "c1", "c2", "c4")."""
    cfg = dict(CONFIGS[name])
    cfg.update(over)
    return make_domain(**cfg)


def domain_bytes(nbas, nocc, naux):
    """Bytes of one domain's inputs in float64 (B, eps, T1, T2)."""
    na, nb = nocc
    va, vb = nbas - na, nbas - nb
    n = 2 * naux * nbas * nbas + 2 * nbas + na * va + nb * vb
    n += na * na * va * va + nb * nb * vb * vb + na * nb * va * vb
    return 8 * n
