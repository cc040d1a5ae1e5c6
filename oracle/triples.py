"""Spin-case (T) energy of one LNO domain -- plain CPU float64 oracle.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the library never
does.  It shares no code with the CUDA path.

What it computes (arXiv 2311.10048, Sec. 2.1, eq cim_pt_energy): the
open-shell perturbative triples energy split into the four spin cases
aaa, aab, abb, bbb, with the triples amplitude times denominator
W = t D and the standard (T) energy sum_{ijkabc} W (W + V) / D with the
T1-driven disconnected part V (the CCSD(T) and CrawfordRev references of that
equation).  In spin orbitals (``oracle.spinorbital`` writes this definition
out literally):

  W^{abc}_{ijk} = P(i/jk) P(a/bc) [ sum_e t^{ae}_{jk} <ei||bc>
                                    - sum_m t^{bc}_{im} <ma||jk> ]
  V^{abc}_{ijk} = P(i/jk) P(a/bc) [ t^a_i <jk||bc> + f_ia t^{bc}_{jk} ]
  E(T) = 1/36 sum_{ijkabc} W (W + V) / D,  D = e_i+e_j+e_k-e_a-e_b-e_c

with P(i/jk) f(ijk) = f(ijk) - f(jik) - f(kji).  This module evaluates the
same sum one restricted occupied triplet at a time with spatial orbitals:
same spin i<j<k with a<b<c, mixed spin i<j (spin s), K (spin t) with
a<b (s), C (t).  Mulliken integrals come from the DF factors,
(pq|rs) = sum_Q B^Q_pq B^Q_rs (Sec. 3.3, eq ed_df_int with B = I L^-T).

The f_ia term is the restricted open-shell one: with an RO reference the
semicanonical Fock matrix keeps an occupied-virtual block (Sec. 3.3, eq
off_diagonal_fock and the singles of eq cim_mp2_ed_energy); it enters V the
way t^a_i does, with the doubles amplitude in place of the integral.  It is
optional (``fov`` absent or None means zero).

Orbital contributions (eq cim_pt_energy): E(T) = sum_i dE_i + sum_I dE_I with
1/36 on the same-spin sum and 1/8 on each mixed sum over unrestricted
indices.  Per restricted triplet that gives each orbital of a same-spin
triplet 1/3 of e_t, and in a mixed triplet 1/4 to each of the two orbitals of
the same spin and 1/2 to the third (``orbital_energies``).

Conventions (readings of the paper, listed in the design notes):
* E = sum W (W+V)/D with the T1 term (and the f_ov term when given) in V.
* The full domain energy over all occupied orbitals is computed (not the
  central-LMO share of eq local_pt).
* Triplet enumeration order (also the order of per-triplet outputs):
  aaa: (i,j,k) i<j<k lexicographic; aab: (i,j,K) i<j lexicographic;
  abb: (I,J,k) I<J lexicographic; bbb: (I,J,K) I<J<K lexicographic.
"""
from __future__ import annotations

import math

import torch

CASES = ("aaa", "aab", "abb", "bbb")

_f64 = torch.float64


def as_tensors(dom, requires_grad=False):
    """Domain dict (numpy or torch) -> dict of CPU float64 torch tensors."""
    def t(x):
        y = torch.as_tensor(x, dtype=_f64).detach().clone()
        return y.requires_grad_(requires_grad)
    return dict(nbas=int(dom["nbas"]), naux=int(dom["naux"]),
                nocc=(int(dom["nocc"][0]), int(dom["nocc"][1])),
                B=[t(dom["B"][0]), t(dom["B"][1])],
                eps=[t(dom["eps"][0]), t(dom["eps"][1])],
                t1=[t(dom["t1"][0]), t(dom["t1"][1])],
                t2aa=t(dom["t2aa"]), t2bb=t(dom["t2bb"]), t2ab=t(dom["t2ab"]),
                fov=_fov_tensors(dom, t))


def _fov_tensors(dom, t):
    """[f spin up, f spin down] or None; a None spin block is zero."""
    f = dom.get("fov")
    if f is None:
        return None
    n = int(dom["nbas"])
    out = []
    for s in (0, 1):
        o = int(dom["nocc"][s])
        out.append(t(f[s]) if f[s] is not None else t(torch.zeros(o, n - o, dtype=_f64)))
    return out


def triplets(case, na, nb):
    """Restricted occupied triplets of one spin case, in output order."""
    if case == "aaa":
        n = na
        return [(i, j, k) for i in range(n) for j in range(i + 1, n)
                for k in range(j + 1, n)]
    if case == "bbb":
        n = nb
        return [(i, j, k) for i in range(n) for j in range(i + 1, n)
                for k in range(j + 1, n)]
    if case == "aab":
        return [(i, j, K) for i in range(na) for j in range(i + 1, na)
                for K in range(nb)]
    if case == "abb":
        return [(I, J, k) for I in range(nb) for J in range(I + 1, nb)
                for k in range(na)]
    raise ValueError(case)


def n_triplets(case, na, nb):
    c2 = lambda n: n * (n - 1) // 2
    c3 = lambda n: n * (n - 1) * (n - 2) // 6
    return {"aaa": c3(na), "bbb": c3(nb), "aab": c2(na) * nb,
            "abb": c2(nb) * na}[case]


class _Spin:
    """Orbital blocks of one spin: occupied o, virtual v, factors B, eps."""

    def __init__(self, B, eps, no):
        self.B, self.eps, self.no = B, eps, no
        self.nv = B.shape[1] - no
        self.o = slice(0, no)
        self.v = slice(no, B.shape[1])


def _eri(Sp, p, q, Sr, r, s):
    """(pq|rs) = sum_Q B^Q_pq B^Q_rs for index ranges/integers p,q,r,s."""
    L = Sp.B[:, p, q]
    R = Sr.B[:, r, s]
    lp = L.reshape(L.shape[0], -1)
    rp = R.reshape(R.shape[0], -1)
    return (lp.T @ rp).reshape(tuple(L.shape[1:]) + tuple(R.shape[1:]))


class Evaluator:
    """Per-triplet (T) contributions of one domain, integrals built lazily."""

    def __init__(self, dom):
        d = dom if isinstance(dom["B"][0], torch.Tensor) else as_tensors(dom)
        self.d = d
        na, nb = d["nocc"]
        self.S = [_Spin(d["B"][0], d["eps"][0], na),
                  _Spin(d["B"][1], d["eps"][1], nb)]
        self.t2ss = [d["t2aa"], d["t2bb"]]
        # t2st[s] = t^{a C}_{i K} with i,a of spin s and K,C of the other spin
        self.t2st = [d["t2ab"], d["t2ab"].permute(1, 0, 3, 2)]
        self.t1 = d["t1"]
        self.fov = d.get("fov")        # None or [f_ia spin up, f_IA spin down]
        self._cache = {}

    def _c(self, key, fn):
        v = self._cache.get(key)
        if v is None:
            v = fn()
            self._cache[key] = v
        return v

    # ---------------- same spin:  i<j<k, a<b<c ----------------------------
    def _abar(self, s, i):
        """A_i[e,b,c] = (eb|ic) - (ec|ib) = <ei||bc> (spin s)."""
        def f():
            S = self.S[s]
            g = _eri(S, S.v, S.v, S, i, S.v)            # (eb|ic) -> [e][b][c]
            return g - g.transpose(1, 2)
        return self._c(("A", s, i), f)

    def _hbar(self, s, j, k):
        """H_jk[m,a] = (mj|ak) - (mk|aj) = <ma||jk> (spin s)."""
        S = self.S[s]
        return _eri(S, S.o, j, S, S.v, k) - _eri(S, S.o, k, S, S.v, j)

    def _kbar(self, s, j, k):
        """K_jk[b,c] = (jb|kc) - (jc|kb) = <jk||bc> (spin s)."""
        S = self.S[s]
        g = _eri(S, j, S.v, S, k, S.v)
        return g - g.T

    def _z_same(self, s, i, j, k):
        """Z(i,j,k)_abc = sum_e t^{ae}_{jk} A_i[e,bc] - sum_m t^{bc}_{im} H_jk[m,a]."""
        t2 = self.t2ss[s]
        part = torch.einsum("ae,ebc->abc", t2[j, k], self._abar(s, i))
        hole = torch.einsum("mbc,ma->abc", t2[i], self._hbar(s, j, k))
        return part - hole

    def same_spin_wv(self, s, i, j, k):
        """W and V of one same-spin triplet, [a][b][c] over all virtuals."""
        X = self._z_same(s, i, j, k) - self._z_same(s, j, i, k) \
            - self._z_same(s, k, j, i)
        W = X - X.permute(1, 0, 2) - X.permute(2, 1, 0)
        t1 = self.t1[s]
        fv = None if self.fov is None else self.fov[s]

        def y(p, q, r):
            # t^a_p <qr||bc>  (+ f_pa t^{bc}_{qr})
            out = t1[p][:, None, None] * self._kbar(s, q, r)[None, :, :]
            if fv is not None:
                out = out + fv[p][:, None, None] * self.t2ss[s][q, r][None, :, :]
            return out
        Yb = y(i, j, k) - y(j, i, k) - y(k, j, i)
        V = Yb - Yb.permute(1, 0, 2) - Yb.permute(2, 1, 0)
        return W, V

    def same_spin_energy(self, s, i, j, k):
        S = self.S[s]
        W, V = self.same_spin_wv(s, i, j, k)
        ev = S.eps[S.v]
        D = (S.eps[i] + S.eps[j] + S.eps[k]) - ev[:, None, None] \
            - ev[None, :, None] - ev[None, None, :]
        n = S.nv
        ar = torch.arange(n)
        mask = (ar[:, None, None] < ar[None, :, None]) & \
               (ar[None, :, None] < ar[None, None, :])
        return (W * (W + V) / D)[mask].sum()

    # ---------------- mixed spin:  i<j (s), K (t); a<b (s), C (t) ----------
    def mixed_wv(self, s, i, j, K):
        """W and V of one mixed triplet, [a][b][C]."""
        t = 1 - s
        Ss, St = self.S[s], self.S[t]
        tss, tst = self.t2ss[s], self.t2st[s]

        def g_ov_vv(x):      # (xb|EC) -> [b][E][C]
            return self._c(("G", s, x), lambda: _eri(Ss, x, Ss.v, St, St.v, St.v))

        def z1(p, q):
            # -sum_E t^{aE}_{qK} (pb|EC) + sum_M t^{bC}_{pM} (qa|MK)
            part = torch.einsum("aE,bEC->abC", tst[q, K], g_ov_vv(p))
            jq = _eri(Ss, q, Ss.v, St, St.o, K)               # (qa|MK) -> [a][M]
            hole = torch.einsum("MbC,aM->abC", tst[p], jq)
            return -part + hole

        def z3():
            # sum_e t^{ae}_{ij} (be|KC) - sum_m t^{bC}_{mK} [(mj|ai) - (mi|aj)]
            f = self._c(("F", s, K), lambda: _eri(Ss, Ss.v, Ss.v, St, K, St.v))
            part = torch.einsum("ae,beC->abC", tss[i, j], f)
            h = _eri(Ss, Ss.o, j, Ss, Ss.v, i) - _eri(Ss, Ss.o, i, Ss, Ss.v, j)
            hole = torch.einsum("mbC,ma->abC", tst[:, K], h)
            return part - hole

        def z7(p, q):
            # sum_e t^{eC}_{qK} [(eb|pa) - (ea|pb)] + sum_m t^{ba}_{pm} (mq|CK)
            ab = self._abar(s, p)            # A_p[e,b,a] = (eb|pa) - (ea|pb)
            part = torch.einsum("eC,eba->abC", tst[q, K], ab)
            l = _eri(Ss, Ss.o, q, St, St.v, K)                # (mq|CK) -> [m][C]
            hole = torch.einsum("mba,mC->abC", tss[p], l)
            return part + hole

        Y = z1(i, j) - z1(j, i) + z3()
        W = Y - Y.permute(1, 0, 2) + z7(i, j) - z7(j, i)
        t1s, t1t = self.t1[s], self.t1[t]
        kjb = _eri(Ss, j, Ss.v, St, K, St.v)                  # (jb|KC) [b][C]
        kib = _eri(Ss, i, Ss.v, St, K, St.v)                  # (ib|KC)
        u = t1s[i][:, None, None] * kjb[None] - t1s[j][:, None, None] * kib[None]
        oo = _eri(Ss, i, Ss.v, Ss, j, Ss.v)                   # (ia|jb) [a][b]
        V = u - u.permute(1, 0, 2) + t1t[K][None, None, :] * (oo - oo.T)[:, :, None]
        if self.fov is not None:
            # the same terms with t^x_p -> f_px and the integral -> the doubles
            # amplitude of the same indices: (jb|KC) -> t^{bC}_{jK},
            # (ia|jb) - (ib|ja) -> t^{ab}_{ij}
            fs, ft = self.fov[s], self.fov[t]
            uf = fs[i][:, None, None] * tst[j, K][None] - fs[j][:, None, None] * tst[i, K][None]
            V = V + uf - uf.permute(1, 0, 2) + ft[K][None, None, :] * tss[i, j][:, :, None]
        return W, V

    def mixed_energy(self, s, i, j, K):
        t = 1 - s
        Ss, St = self.S[s], self.S[t]
        W, V = self.mixed_wv(s, i, j, K)
        es, et = Ss.eps[Ss.v], St.eps[St.v]
        D = (Ss.eps[i] + Ss.eps[j] + St.eps[K]) - es[:, None, None] \
            - es[None, :, None] - et[None, None, :]
        n = Ss.nv
        ar = torch.arange(n)
        mask = (ar[:, None] < ar[None, :])[:, :, None].expand(n, n, St.nv)
        return (W * (W + V) / D)[mask].sum()

    # ---------------- drivers --------------------------------------------
    def triplet_energy(self, case, trip):
        """e_t: the contribution of one restricted triplet (Eh)."""
        i, j, k = trip
        if case == "aaa":
            return self.same_spin_energy(0, i, j, k)
        if case == "bbb":
            return self.same_spin_energy(1, i, j, k)
        if case == "aab":
            return self.mixed_energy(0, i, j, k)
        if case == "abb":
            return self.mixed_energy(1, i, j, k)
        raise ValueError(case)

    def case_energies(self, case, trips=None):
        na, nb = self.d["nocc"]
        trips = triplets(case, na, nb) if trips is None else trips
        return [self.triplet_energy(case, t) for t in trips]


def energy(dom):
    """E(T) split by spin case: {"aaa","aab","abb","bbb","total"} (floats).

    Per-triplet contributions are summed with math.fsum, so the result does
    not depend on summation order.
    """
    ev = Evaluator(dom)
    out = {}
    with torch.no_grad():
        for c in CASES:
            out[c] = math.fsum(float(e) for e in ev.case_energies(c))
    out["total"] = math.fsum(out[c] for c in CASES)
    return out


def triplet_energies(dom, case, trips=None):
    """Per-triplet contributions (list of floats) in ``triplets`` order."""
    ev = Evaluator(dom)
    with torch.no_grad():
        return [float(e) for e in ev.case_energies(case, trips)]


def orbital_energies(dom, trip_sel=None):
    """Orbital contributions dE_i (spin up) and dE_I (spin down) of eq
    cim_pt_energy, from the per-triplet contributions: same-spin triplet
    1/3 to each orbital; mixed triplet 1/4 to each of its two same-spin
    orbitals and 1/2 to the other.  ``trip_sel`` (dict case -> list of
    triplet indices) restricts the sums to those triplets.

    Returns {"alpha": [na floats], "beta": [nb floats]}, each summed with
    math.fsum.
    """
    ev = Evaluator(dom)
    na, nb = ev.d["nocc"]
    parts = {0: [[] for _ in range(na)], 1: [[] for _ in range(nb)]}
    with torch.no_grad():
        for c in CASES:
            allt = triplets(c, na, nb)
            idx = range(len(allt)) if trip_sel is None or trip_sel.get(c) is None \
                else trip_sel[c]
            for q in idx:
                i, j, k = allt[q]
                e = float(ev.triplet_energy(c, (i, j, k)))
                if c in ("aaa", "bbb"):
                    s = 0 if c == "aaa" else 1
                    for p in (i, j, k):
                        parts[s][p].append(e / 3.0)
                else:
                    s = 0 if c == "aab" else 1
                    parts[s][i].append(e / 4.0)
                    parts[s][j].append(e / 4.0)
                    parts[1 - s][k].append(e / 2.0)
    return {"alpha": [math.fsum(x) for x in parts[0]],
            "beta": [math.fsum(x) for x in parts[1]]}


def energy_graph(dom_t):
    """Differentiable total E(T) (torch scalar) for tensors with requires_grad.

    Used for the oracle gradient: autograd through the same spin-case sums.
    """
    ev = Evaluator(dom_t)
    tot = torch.zeros((), dtype=_f64)
    for c in CASES:
        for e in ev.case_energies(c):
            tot = tot + e
    return tot
