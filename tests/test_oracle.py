"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each checks it against an
independent statement (spin-orbital definition, closed-shell formula, an
invariance, a symmetry, finite differences).
"""
import copy
import json
import math
import os

import numpy as np
import pytest
import torch

from oracle import triples as T
from oracle.closed_shell import rhf_energy
from oracle.spinorbital import brute_force
from paper_2311_10048_gb300.synth import config_domain, make_domain

CASES = ("aaa", "aab", "abb", "bbb")
TINY = [(9, 3, 2, 1), (10, 4, 4, 2), (9, 3, 3, 3), (8, 3, 1, 4), (10, 4, 1, 5),
        (9, 4, 2, 6), (7, 2, 2, 7)]


def tiny(nbas, na, nb, seed, **kw):
    kw.setdefault("t1_sd", 0.05)
    return make_domain(nbas, (na, nb), naux=20, L=10.0, seed=seed, **kw)


def close(a, b, rel=1e-12, abs_=1e-15):
    return abs(a - b) <= abs_ + rel * max(abs(a), abs(b))


@pytest.mark.parametrize("shape", TINY)
def test_p1_spin_cases_equal_spin_orbital_brute_force(shape):
    d = tiny(*shape)
    e, b = T.energy(d), brute_force(d)
    for k in CASES + ("total",):
        assert close(e[k], b[k]), (k, e[k], b[k])
    assert e["total"] < 0


def test_p2_closed_shell_limit_equals_rhf_formula():
    for seed in (11, 12, 13):
        d = tiny(9, 3, 3, seed, closed_shell=True)
        e = T.energy(d)
        ref = rhf_energy(d)
        assert close(e["total"], ref, rel=1e-12), (e["total"], ref)
        assert close(e["aaa"], e["bbb"]) and close(e["aab"], e["abb"])


def test_p2_closed_shell_at_larger_size():
    d = make_domain(24, (4, 4), naux=48, L=16.0, seed=21, closed_shell=True)
    assert close(T.energy(d)["total"], rhf_energy(d), rel=1e-12)


def test_p3_w_antisymmetry_spin_orbital_and_spin_case():
    d = tiny(9, 3, 2, 31)
    _, tens = brute_force(d, return_tensors=True)
    W, V = tens["W"], tens["V"]
    for X in (W, V):
        for p, q in ((0, 1), (1, 2), (0, 2), (3, 4), (4, 5), (3, 5)):
            assert torch.allclose(X, -X.transpose(p, q), atol=1e-15)
    ev = T.Evaluator(d)
    Ws, Vs = ev.same_spin_wv(0, 0, 1, 2)
    for X in (Ws, Vs):
        assert torch.allclose(X, -X.permute(1, 0, 2), atol=1e-15)
        assert torch.allclose(X, -X.permute(0, 2, 1), atol=1e-15)
    Wm, Vm = ev.mixed_wv(0, 0, 2, 1)
    assert torch.allclose(Wm, -Wm.permute(1, 0, 2), atol=1e-15)
    assert torch.allclose(Vm, -Vm.permute(1, 0, 2), atol=1e-15)
    # the triplet's W is antisymmetric in its occupied labels as well
    Wji, _ = ev.same_spin_wv(0, 1, 0, 2)
    assert torch.allclose(Wji, -Ws, atol=1e-15)


def flip_spins(d):
    f = copy.deepcopy(d)
    f["B"] = [d["B"][1], d["B"][0]]
    f["eps"] = [d["eps"][1], d["eps"][0]]
    f["t1"] = [d["t1"][1], d["t1"][0]]
    f["t2aa"], f["t2bb"] = d["t2bb"], d["t2aa"]
    f["t2ab"] = np.ascontiguousarray(d["t2ab"].transpose(1, 0, 3, 2))
    f["nocc"] = (d["nocc"][1], d["nocc"][0])
    return f


def test_p4_spin_flip_swaps_cases():
    d = tiny(10, 3, 3, 41)
    e, f = T.energy(d), T.energy(flip_spins(d))
    assert close(e["aaa"], f["bbb"]) and close(e["bbb"], f["aaa"])
    assert close(e["aab"], f["abb"]) and close(e["abb"], f["aab"])
    assert not close(e["aab"], e["abb"], rel=1e-6)


def test_p5_uniform_orbital_energy_shift_leaves_energy():
    d = tiny(9, 3, 2, 51)
    s = copy.deepcopy(d)
    s["eps"] = [d["eps"][0] + 0.37, d["eps"][1] + 0.37]
    e, es = T.energy(d), T.energy(s)
    for k in CASES:
        assert close(e[k], es[k], rel=1e-12)
    # shifting only the spin-up occupied energies does change it
    e0 = d["eps"][0].copy()
    e0[:d["nocc"][0]] += 0.37
    s["eps"] = [e0, d["eps"][1]]
    assert not close(T.energy(s)["aab"], e["aab"], rel=1e-6)


def test_p6_homogeneity_in_b_and_t2():
    d = tiny(9, 3, 2, 61)
    e = T.energy(d)
    s = 1.7
    b = copy.deepcopy(d)
    b["B"] = [d["B"][0] * s, d["B"][1] * s]
    eb = T.energy(b)
    for k in CASES:
        assert close(eb[k], s ** 4 * e[k], rel=1e-12)
    z = copy.deepcopy(d)
    z["t1"] = [0 * d["t1"][0], 0 * d["t1"][1]]
    ez = T.energy(z)
    for key in ("t2aa", "t2bb", "t2ab"):
        z[key] = d[key] * s
    ez2 = T.energy(z)
    for k in CASES:
        assert close(ez2[k], s ** 2 * ez[k], rel=1e-12)


def relabel(d, perm_a, perm_va):
    """Permute spin-up occupied and virtual orbital labels in every input."""
    r = copy.deepcopy(d)
    na = d["nocc"][0]
    full = np.concatenate([perm_a, na + perm_va])
    r["B"][0] = d["B"][0][:, full][:, :, full]
    r["eps"][0] = d["eps"][0][full]
    r["t1"][0] = d["t1"][0][perm_a][:, perm_va]
    r["t2aa"] = d["t2aa"][perm_a][:, perm_a][:, :, perm_va][:, :, :, perm_va]
    r["t2ab"] = d["t2ab"][perm_a][:, :, perm_va]
    return r


def test_p7_relabelling_invariance():
    d = tiny(10, 4, 2, 71)
    rng = np.random.default_rng(5)
    r = relabel(d, rng.permutation(4), rng.permutation(6))
    e, er = T.energy(d), T.energy(r)
    for k in CASES:
        assert close(e[k], er[k], rel=1e-12)


def test_triplet_counts_and_order():
    for na, nb in ((6, 4), (3, 3), (4, 1), (2, 0)):
        for c in CASES:
            tr = T.triplets(c, na, nb)
            assert len(tr) == T.n_triplets(c, na, nb)
            assert tr == sorted(tr) and len(set(tr)) == len(tr)


def test_oracle_gradient_matches_central_differences():
    d = tiny(8, 3, 2, 81)
    dt = T.as_tensors(d, requires_grad=True)
    E = T.energy_graph(dt)
    E.backward()
    rng = np.random.default_rng(3)
    h = 1e-5
    # directional derivative along symmetry-respecting random directions
    for name in ("B0", "eps1", "t1_0", "t2aa", "t2ab"):
        dp, dm = T.as_tensors(d), T.as_tensors(d)
        if name == "B0":
            x = rng.standard_normal(d["B"][0].shape)
            x = x + x.transpose(0, 2, 1)
            g = float((dt["B"][0].grad * torch.as_tensor(x)).sum())
            dp["B"][0] += h * torch.as_tensor(x)
            dm["B"][0] -= h * torch.as_tensor(x)
        elif name == "eps1":
            x = rng.standard_normal(d["eps"][1].shape)
            g = float((dt["eps"][1].grad * torch.as_tensor(x)).sum())
            dp["eps"][1] += h * torch.as_tensor(x)
            dm["eps"][1] -= h * torch.as_tensor(x)
        elif name == "t1_0":
            x = rng.standard_normal(d["t1"][0].shape)
            g = float((dt["t1"][0].grad * torch.as_tensor(x)).sum())
            dp["t1"][0] += h * torch.as_tensor(x)
            dm["t1"][0] -= h * torch.as_tensor(x)
        elif name == "t2aa":
            x = rng.standard_normal(d["t2aa"].shape)
            x = x - x.transpose(1, 0, 2, 3)
            x = x - x.transpose(0, 1, 3, 2)
            g = float((dt["t2aa"].grad * torch.as_tensor(x)).sum())
            dp["t2aa"] += h * torch.as_tensor(x)
            dm["t2aa"] -= h * torch.as_tensor(x)
        else:
            x = rng.standard_normal(d["t2ab"].shape)
            g = float((dt["t2ab"].grad * torch.as_tensor(x)).sum())
            dp["t2ab"] += h * torch.as_tensor(x)
            dm["t2ab"] -= h * torch.as_tensor(x)
        fd = (T.energy(dp)["total"] - T.energy(dm)["total"]) / (2 * h)
        assert abs(fd - g) <= 1e-7 * max(1.0, abs(g)), (name, fd, g)


def test_generator_recipe_properties():
    d = make_domain(30, (5, 3), naux=50, L=12.5, seed=9)
    for s in (0, 1):
        B = d["B"][s]
        assert np.array_equal(B, B.transpose(0, 2, 1))
        no = d["nocc"][s]
        e = d["eps"][s]
        assert np.all(np.diff(e[:no]) >= 0) and np.all(np.diff(e[no:]) >= 0)
        assert e[:no].max() < -0.3 + 1e-12 and e[no:].min() > 0.1 - 1e-12
    t2 = d["t2aa"]
    assert np.allclose(t2, -t2.transpose(1, 0, 2, 3))
    assert np.allclose(t2, -t2.transpose(0, 1, 3, 2))
    d2 = make_domain(30, (5, 3), naux=50, L=12.5, seed=9)
    assert all(np.array_equal(d[k], d2[k]) for k in ("t2aa", "t2bb", "t2ab"))


def test_stored_c0_golden_matches_oracle():
    path = os.path.join(os.path.dirname(__file__), "golden", "c0_energy.json")
    g = json.load(open(path))
    e = T.energy(config_domain("c0"))
    for c in CASES:
        assert close(g["cases"][c]["sum"], e[c], rel=1e-12)
    assert close(g["total"], e["total"], rel=1e-12)


class _Planted:
    """Context manager that plants a mistake in the oracle (CPU only)."""

    def __init__(self, attr, fn):
        self.attr, self.fn = attr, fn

    def __enter__(self):
        self.old = getattr(T.Evaluator, self.attr)
        setattr(T.Evaluator, self.attr, self.fn(self.old))

    def __exit__(self, *a):
        setattr(T.Evaluator, self.attr, self.old)


@pytest.mark.parametrize("mistake", ["hole_sign", "drop_v", "swap_h"])
def test_planted_oracle_mistakes_are_caught_by_brute_force(mistake):
    d = tiny(9, 3, 2, 91)
    ref = brute_force(d)
    if mistake == "hole_sign":
        def mk(old):
            def z(self, s, i, j, k):
                t2 = self.t2ss[s]
                part = torch.einsum("ae,ebc->abc", t2[j, k], self._abar(s, i))
                hole = torch.einsum("mbc,ma->abc", t2[i], self._hbar(s, j, k))
                return part + hole
            return z
        attr = "_z_same"
    elif mistake == "drop_v":
        def mk(old):
            def wv(self, s, i, j, k):
                W, V = old(self, s, i, j, k)
                return W, 0 * V
            return wv
        attr = "same_spin_wv"
    else:
        def mk(old):
            def h(self, s, j, k):
                return old(self, s, k, j)
            return h
        attr = "_hbar"
    with _Planted(attr, mk):
        bad = T.energy(d)
    assert not close(bad["aaa"], ref["aaa"], rel=1e-9)


# ---- restricted open-shell f_ov term and orbital contributions --------------
from oracle.spinorbital import orbital_partition
from paper_2311_10048_gb300.synth import add_fov

FOV_SHAPES = [(9, 3, 2, 1), (10, 4, 4, 2), (8, 3, 1, 4), (9, 4, 2, 6), (7, 2, 2, 7)]


@pytest.mark.parametrize("shape", FOV_SHAPES)
def test_fov_spin_cases_equal_spin_orbital_brute_force(shape):
    d = add_fov(tiny(*shape), sd=0.05, seed=shape[-1])
    e, b = T.energy(d), brute_force(d)
    for k in CASES + ("total",):
        assert close(e[k], b[k]), (k, e[k], b[k])
    # the term is not a no-op on these inputs
    assert not close(e["total"], T.energy(tiny(*shape))["total"], rel=1e-9)


def test_fov_enters_affinely_with_t1():
    # V is linear in (t1, f) and E is affine in V:
    # E(t1, f) - E(0, 0) = [E(t1, 0) - E(0, 0)] + [E(0, f) - E(0, 0)]
    base = tiny(9, 3, 2, 41)
    f = add_fov(base, sd=0.05, seed=41)["fov"]
    z1 = [np.zeros_like(x) for x in base["t1"]]
    e = lambda t1, fov: T.energy(dict(base, t1=t1, fov=fov))["total"]
    e00, e10, e01, e11 = e(z1, None), e(base["t1"], None), e(z1, f), e(base["t1"], f)
    assert close(e11 - e00, (e10 - e00) + (e01 - e00), rel=1e-10)
    # zero block == no block
    assert e(base["t1"], [np.zeros_like(x) for x in f]) == e10
    # and the f part scales linearly
    e02 = e(z1, [2 * x for x in f])
    assert close(e02 - e00, 2 * (e01 - e00), rel=1e-10)


@pytest.mark.parametrize("shape", FOV_SHAPES[:3])
@pytest.mark.parametrize("with_fov", [False, True])
def test_orbital_energies_equal_eq_prefactor_sums(shape, with_fov):
    d = tiny(*shape)
    if with_fov:
        d = add_fov(d, sd=0.05, seed=shape[-1])
    o, ob = T.orbital_energies(d), orbital_partition(d)
    for s in ("alpha", "beta"):
        assert len(o[s]) == len(ob[s])
        for x, y in zip(o[s], ob[s]):
            assert close(x, y, rel=1e-11, abs_=1e-14), (s, x, y)
    assert close(math.fsum(o["alpha"] + o["beta"]), T.energy(d)["total"], rel=1e-12)


def test_orbital_energies_follow_relabelling():
    d = tiny(9, 4, 2, 51)
    perm = np.array([2, 0, 3, 1])                # spin-up occupied relabelling
    p = dict(d)
    na = d["nocc"][0]
    full = np.concatenate([perm, np.arange(na, d["nbas"])])
    p["B"] = [d["B"][0][:, full][:, :, full], d["B"][1]]
    p["eps"] = [d["eps"][0][full], d["eps"][1]]
    p["t1"] = [d["t1"][0][perm], d["t1"][1]]
    p["t2aa"] = d["t2aa"][perm][:, perm]
    p["t2ab"] = d["t2ab"][perm]
    o, op = T.orbital_energies(d), T.orbital_energies(p)
    for q in range(na):
        assert close(op["alpha"][q], o["alpha"][perm[q]], rel=1e-11)
    for q in range(d["nocc"][1]):
        assert close(op["beta"][q], o["beta"][q], rel=1e-11)


@pytest.mark.parametrize("mistake", ["fov_mixed_sign", "fov_same_swap"])
def test_planted_fov_mistakes_are_caught_by_brute_force(mistake):
    d = add_fov(tiny(9, 3, 2, 93), sd=0.05, seed=93)
    ref = brute_force(d)
    if mistake == "fov_mixed_sign":
        def mk(old):
            def wv(self, s, i, j, K):
                W, V = old(self, s, i, j, K)
                # undo the f_KC term and add it with the wrong sign
                ft, tss = self.fov[1 - s], self.t2ss[s]
                return W, V - 2 * ft[K][None, None, :] * tss[i, j][:, :, None]
            return wv
        attr, case = "mixed_wv", "aab"
    else:
        def mk(old):
            def wv(self, s, i, j, k):
                W, V = old(self, s, i, j, k)
                fv, t2 = self.fov[s], self.t2ss[s]
                # replace f_pa t^{bc}_{qr} by f_pa t^{cb}_{qr} for p = i
                delta = fv[i][:, None, None] * (t2[j, k] - t2[j, k].T)[None]
                Y = -delta
                return W, V + Y - Y.permute(1, 0, 2) - Y.permute(2, 1, 0)
            return wv
        attr, case = "same_spin_wv", "aaa"
    with _Planted(attr, mk):
        bad = T.energy(d)
    assert not close(bad[case], ref[case], rel=1e-9)


def test_planted_partition_mistake_is_caught():
    # an equal 1/3 split of mixed triplets is a valid-looking partition that
    # sums to the total, but not the one eq cim_pt_energy defines
    d = tiny(9, 3, 2, 95)
    ob = orbital_partition(d)
    ev = T.Evaluator(d)
    na, nb = d["nocc"]
    eq = {"alpha": [0.0] * na, "beta": [0.0] * nb}
    with torch.no_grad():
        for c in CASES:
            s = 0 if c in ("aaa", "aab") else 1
            for (i, j, k) in T.triplets(c, na, nb):
                e = float(ev.triplet_energy(c, (i, j, k)))
                key = "alpha" if s == 0 else "beta"
                other = "beta" if s == 0 else "alpha"
                eq[key][i] += e / 3
                eq[key][j] += e / 3
                eq[key if c in ("aaa", "bbb") else other][k] += e / 3
    worst = max(abs(x - y) for s in ("alpha", "beta") for x, y in zip(eq[s], ob[s]))
    assert worst > 1e-6 * max(abs(x) for x in ob["alpha"] + ob["beta"])
