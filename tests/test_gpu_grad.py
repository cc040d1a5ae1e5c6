"""Adjoint (lno_ot_backward / torch.autograd) vs the oracle gradient and
central finite differences.

The oracle gradient is PyTorch autograd through the CPU float64 oracle,
projected onto the inputs' symmetries exactly as the C ABI documents
(dB symmetric in (p,q); dT2aa/bb antisymmetric in (i,j) and (a,b)).
Tolerance: 1e-6 relative (element-wise against the largest entry of each
gradient; directional derivatives against central differences at h = 1e-5 and
h/2, Richardson-extrapolated).  The float64 context runs the adjoint's
contractions in float64; a BF16X10 context runs them on the tensor cores
(tc_matmul: exact 4-slice BF16 operands, float64 output) and is held to the
same tolerance.
"""
import numpy as np
import pytest
import torch

from oracle import triples as T
from paper_2311_10048_gb300 import lno_ot
from paper_2311_10048_gb300.synth import config_domain, make_domain

pytestmark = pytest.mark.gpu
CASES = ("aaa", "aab", "abb", "bbb")
KEYS = ["B0", "B1", "e0", "e1", "t10", "t11", "t2aa", "t2bb", "t2ab"]


@pytest.fixture(scope="module")
def ctx64(lib):
    c = lno_ot.Context(0, "fp64")
    yield c
    c.close()


@pytest.fixture(scope="module")
def ctx10(lib):
    c = lno_ot.Context(0, "bf16x10")
    yield c
    c.close()


def oracle_grad(d, sel=None):
    dt = T.as_tensors(d, requires_grad=True)
    ev = T.Evaluator(dt)
    na, nb = dt["nocc"]
    E = torch.zeros((), dtype=torch.float64)
    for ci, c in enumerate(CASES):
        trs = T.triplets(c, na, nb)
        idx = range(len(trs)) if sel is None else [int(q) for q in sel[ci]]
        for q in idx:
            E = E + ev.triplet_energy(c, trs[q])
    E.backward()
    for key in ("B", "eps", "t1"):
        for x in dt[key]:
            if x.grad is None:
                x.grad = torch.zeros_like(x)
    for key in ("t2aa", "t2bb", "t2ab"):
        if dt[key].grad is None:
            dt[key].grad = torch.zeros_like(dt[key])
    sym = lambda g: 0.5 * (g + g.transpose(1, 2))
    asym = lambda g: 0.25 * (g - g.transpose(0, 1) - g.transpose(2, 3) + g.transpose(0, 1).transpose(2, 3))
    return [sym(dt["B"][0].grad), sym(dt["B"][1].grad), dt["eps"][0].grad, dt["eps"][1].grad,
            dt["t1"][0].grad, dt["t1"][1].grad, asym(dt["t2aa"].grad), asym(dt["t2bb"].grad),
            dt["t2ab"].grad], float(E.detach())


def gpu_grad(ctx, d, sel=None, gE=1.0):
    dd = lno_ot.to_device(d)
    ins = [dd["B"][0], dd["B"][1], dd["eps"][0], dd["eps"][1], dd["t1"][0], dd["t1"][1],
           dd["t2aa"], dd["t2bb"], dd["t2ab"]]
    for x in ins:
        x.requires_grad_(True)
    dom = dict(dd, B=ins[0:2], eps=ins[2:4], t1=ins[4:6], t2aa=ins[6], t2bb=ins[7], t2ab=ins[8])
    E = lno_ot.triples_energy(ctx, dom, trip_sel=sel)
    grads = torch.autograd.grad(E * gE, ins)
    return [g.detach().cpu() for g in grads], float(E.detach())


def compare(g_gpu, g_ref, rel=1e-6):
    for k, a, b in zip(KEYS, g_gpu, g_ref):
        scale = float(b.abs().max()) if b.numel() else 0.0
        if scale == 0.0:
            assert float(a.abs().max()) <= 1e-14, k
            continue
        err = float((a - b).abs().max())
        assert err <= rel * scale, (k, err, scale)


@pytest.mark.parametrize("shape", [(9, 3, 2, 1), (12, 4, 4, 2), (10, 4, 1, 3), (20, 5, 3, 4)])
def test_gradient_matches_oracle_small(ctx64, shape):
    nbas, na, nb, seed = shape
    d = make_domain(nbas, (na, nb), naux=2 * nbas, L=nbas / 2, seed=seed, t1_sd=0.05)
    g_ref, e_ref = oracle_grad(d)
    g, e = gpu_grad(ctx64, d, gE=1.0)
    assert abs(e - e_ref) <= 1e-12 * max(1.0, abs(e_ref))
    compare(g, g_ref)


@pytest.mark.parametrize("shape", [(9, 3, 2, 1), (20, 5, 3, 4), (40, 6, 5, 5)])
def test_tensor_core_adjoint_matches_oracle_small(ctx10, shape):
    nbas, na, nb, seed = shape
    d = make_domain(nbas, (na, nb), naux=2 * nbas, L=nbas / 2, seed=seed, t1_sd=0.05)
    g_ref, e_ref = oracle_grad(d)
    g, e = gpu_grad(ctx10, d, gE=1.0)
    assert abs(e - e_ref) <= 1e-9 * max(1.0, abs(e_ref))
    compare(g, g_ref)


def test_gradient_scales_with_gE(ctx64):
    d = make_domain(11, (3, 2), naux=22, L=6.0, seed=9, t1_sd=0.05)
    g1, _ = gpu_grad(ctx64, d, gE=1.0)
    g2, _ = gpu_grad(ctx64, d, gE=-2.5)
    for a, b in zip(g1, g2):
        # atomics make the summation order differ from run to run
        assert float((-2.5 * a - b).abs().max()) <= 1e-12 * max(float(b.abs().max()), 1e-300)


def test_c0_gradient_vs_oracle_and_central_differences(ctx64):
    d = config_domain("c0")
    g_ref, _ = oracle_grad(d)
    g, _ = gpu_grad(ctx64, d)
    compare(g, g_ref)
    # directional derivatives along symmetry-respecting random directions
    rng = np.random.default_rng(17)
    h = 1e-5
    dd = lno_ot.to_device(d)

    def E(dm):
        return ctx64.energy(dm)["total"]

    def perturbed(key, x, sign, h):
        dm = dict(dd, B=list(dd["B"]), eps=list(dd["eps"]), t1=list(dd["t1"]))
        xt = torch.as_tensor(x, device="cuda")
        if key in ("B0", "B1"):
            s = int(key[1]); dm["B"][s] = dd["B"][s] + sign * h * xt
        elif key in ("e0", "e1"):
            s = int(key[1]); dm["eps"][s] = dd["eps"][s] + sign * h * xt
        elif key in ("t10", "t11"):
            s = int(key[2]); dm["t1"][s] = dd["t1"][s] + sign * h * xt
        else:
            dm[key] = dd[key] + sign * h * xt
        return dm

    shapes = {"B0": d["B"][0].shape, "B1": d["B"][1].shape, "e0": d["eps"][0].shape,
              "e1": d["eps"][1].shape, "t10": d["t1"][0].shape, "t11": d["t1"][1].shape,
              "t2aa": d["t2aa"].shape, "t2bb": d["t2bb"].shape, "t2ab": d["t2ab"].shape}
    for ki, key in enumerate(KEYS):
        x = rng.standard_normal(shapes[key])
        if key in ("B0", "B1"):
            x = x + x.transpose(0, 2, 1)
        if key in ("t2aa", "t2bb"):
            x = x - x.transpose(1, 0, 2, 3)
            x = x - x.transpose(0, 1, 3, 2)
        fd1 = (E(perturbed(key, x, +1, h)) - E(perturbed(key, x, -1, h))) / (2 * h)
        fd2 = (E(perturbed(key, x, +1, h / 2)) - E(perturbed(key, x, -1, h / 2))) / h
        fd = (4 * fd2 - fd1) / 3
        an = float((g[ki] * torch.as_tensor(x)).sum())
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3), (key, fd, an, fd1, fd2)


def test_c4_subset_central_differences_all_nine_inputs(ctx64):
    # at the differentiation domain's size (nbas 200, 20/18 occupied): the
    # adjoint on a seeded triplet subset against central differences of the
    # float64 forward on the same subset, along one random symmetry-respecting
    # direction per input; central differences at h = 1e-5 and h/2 combined by
    # Richardson extrapolation (the O(h^2) term cancels; a direction that moves
    # every entry of an input at once has a large third derivative)
    d = config_domain("c4")
    rng = np.random.default_rng(2024)
    na, nb = d["nocc"]
    sel = [np.sort(rng.choice(T.n_triplets(c, na, nb), size=2, replace=False)).astype(np.int64)
           for c in CASES]
    g, _ = gpu_grad(ctx64, d, sel)
    dd = lno_ot.to_device(d)
    h = 1e-5

    def E(dm):
        return ctx64.energy(dm, trip_sel=sel)["total"]

    def perturbed(key, x, sign, h):
        dm = dict(dd, B=list(dd["B"]), eps=list(dd["eps"]), t1=list(dd["t1"]))
        xt = torch.as_tensor(x, device="cuda")
        if key in ("B0", "B1"):
            s = int(key[1]); dm["B"][s] = dd["B"][s] + sign * h * xt
        elif key in ("e0", "e1"):
            s = int(key[1]); dm["eps"][s] = dd["eps"][s] + sign * h * xt
        elif key in ("t10", "t11"):
            s = int(key[2]); dm["t1"][s] = dd["t1"][s] + sign * h * xt
        else:
            dm[key] = dd[key] + sign * h * xt
        return dm

    shapes = {"B0": d["B"][0].shape, "B1": d["B"][1].shape, "e0": d["eps"][0].shape,
              "e1": d["eps"][1].shape, "t10": d["t1"][0].shape, "t11": d["t1"][1].shape,
              "t2aa": d["t2aa"].shape, "t2bb": d["t2bb"].shape, "t2ab": d["t2ab"].shape}
    for ki, key in enumerate(KEYS):
        x = rng.standard_normal(shapes[key])
        if key in ("B0", "B1"):
            x = x + x.transpose(0, 2, 1)
        if key in ("t2aa", "t2bb"):
            x = x - x.transpose(1, 0, 2, 3)
            x = x - x.transpose(0, 1, 3, 2)
        fd1 = (E(perturbed(key, x, +1, h)) - E(perturbed(key, x, -1, h))) / (2 * h)
        fd2 = (E(perturbed(key, x, +1, h / 2)) - E(perturbed(key, x, -1, h / 2))) / h
        fd = (4 * fd2 - fd1) / 3
        an = float((g[ki] * torch.as_tensor(x)).sum())
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3), (key, fd, an, fd1, fd2)


@pytest.fixture(scope="module")
def c4_subset_oracle():
    d = config_domain("c4")
    sel = [np.array([0, 500]), np.array([7]), np.array([1000]), np.array([3, 815])]
    g_ref, e_ref = oracle_grad(d, sel)
    return d, sel, g_ref, e_ref


def test_c4_subset_gradient_vs_oracle(ctx64, c4_subset_oracle):
    d, sel, g_ref, e_ref = c4_subset_oracle
    g, e = gpu_grad(ctx64, d, sel)
    assert abs(e - e_ref) <= 1e-10 * abs(e_ref)
    compare(g, g_ref)


def test_c4_subset_tensor_core_adjoint_vs_oracle(ctx10, c4_subset_oracle):
    d, sel, g_ref, e_ref = c4_subset_oracle
    g, e = gpu_grad(ctx10, d, sel)
    # the forward is the BF16X10 energy (float32 element arithmetic, ~1e-10 Eh per triplet)
    assert abs(e - e_ref) <= 1e-8
    compare(g, g_ref)


# ---- with the restricted open-shell f_ov block -------------------------------
from paper_2311_10048_gb300.synth import add_fov  # noqa: E402

KEYS_F = KEYS + ["f0", "f1"]


def oracle_grad_fov(d):
    dt = T.as_tensors(d, requires_grad=True)
    E = T.energy_graph(dt)
    E.backward()
    grads, _ = [], None
    ins = [dt["B"][0], dt["B"][1], dt["eps"][0], dt["eps"][1], dt["t1"][0], dt["t1"][1],
           dt["t2aa"], dt["t2bb"], dt["t2ab"], dt["fov"][0], dt["fov"][1]]
    for x in ins:
        grads.append(torch.zeros_like(x) if x.grad is None else x.grad)
    sym = lambda g: 0.5 * (g + g.transpose(1, 2))
    asym = lambda g: 0.25 * (g - g.transpose(0, 1) - g.transpose(2, 3) + g.transpose(0, 1).transpose(2, 3))
    grads[0], grads[1] = sym(grads[0]), sym(grads[1])
    grads[6], grads[7] = asym(grads[6]), asym(grads[7])
    return grads, float(E.detach())


def gpu_grad_fov(ctx, d, fov_given=True):
    dd = lno_ot.to_device(d)
    if not fov_given:
        dd["fov"] = [torch.zeros_like(dd["t1"][0]), torch.zeros_like(dd["t1"][1])]
    ins = [dd["B"][0], dd["B"][1], dd["eps"][0], dd["eps"][1], dd["t1"][0], dd["t1"][1],
           dd["t2aa"], dd["t2bb"], dd["t2ab"], dd["fov"][0], dd["fov"][1]]
    for x in ins:
        x.requires_grad_(True)
    dom = dict(dd, B=ins[0:2], eps=ins[2:4], t1=ins[4:6], t2aa=ins[6], t2bb=ins[7],
               t2ab=ins[8], fov=ins[9:11])
    E = lno_ot.triples_energy(ctx, dom)
    return [g.detach().cpu() for g in torch.autograd.grad(E, ins)], float(E.detach())


@pytest.mark.parametrize("shape", [(9, 3, 2, 1), (12, 4, 4, 2), (10, 4, 1, 3), (20, 5, 3, 4)])
def test_gradient_with_fov_matches_oracle(ctx64, shape):
    nbas, na, nb, seed = shape
    d = add_fov(make_domain(nbas, (na, nb), naux=2 * nbas, L=nbas / 2, seed=seed, t1_sd=0.05),
                sd=0.05, seed=seed)
    g_ref, e_ref = oracle_grad_fov(d)
    g, e = gpu_grad_fov(ctx64, d)
    assert abs(e - e_ref) <= 1e-12 * max(1.0, abs(e_ref))
    for k, a, b in zip(KEYS_F, g, g_ref):
        scale = float(b.abs().max()) if b.numel() else 0.0
        if scale == 0.0:
            assert float(a.abs().max()) <= 1e-14, k
            continue
        assert float((a - b).abs().max()) <= 1e-6 * scale, (k, float((a - b).abs().max()), scale)


def test_fov_gradient_at_zero_block(ctx64, lib):
    # dE/df_ov at f_ov = 0, requested from a domain without an f_ov block,
    # equals the gradient of a domain whose block is explicitly zero
    d = make_domain(12, (4, 3), naux=24, L=6.0, seed=5, t1_sd=0.05)
    dd = lno_ot.to_device(d)
    gA = dict(dfov=[torch.empty_like(dd["t1"][0]), torch.empty_like(dd["t1"][1])])
    ctx64.backward(dd, 1.0, gA)
    gz, _ = gpu_grad_fov(ctx64, d, fov_given=False)
    for s in (0, 1):
        ref = gz[9 + s]
        assert float(ref.abs().max()) > 0
        assert float((gA["dfov"][s].cpu() - ref).abs().max()) <= 1e-12 * float(ref.abs().max())
    # and central differences along a random f_ov direction
    rng = np.random.default_rng(3)
    x = [rng.standard_normal(dd["t1"][s].shape) for s in (0, 1)]
    h = 1e-5
    E = lambda sg: ctx64.energy(dict(dd, fov=[sg * h * torch.as_tensor(x[s], device="cuda")
                                              for s in (0, 1)]))["total"]
    fd = (E(+1) - E(-1)) / (2 * h)
    an = sum(float((gA["dfov"][s].cpu() * torch.as_tensor(x[s])).sum()) for s in (0, 1))
    assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3), (fd, an)
