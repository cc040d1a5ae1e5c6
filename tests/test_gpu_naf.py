"""NAF compression on the GPU (lno_ot_naf, Sec. 3.6, eq naf_w) against the
oracle: the eigenvalues of W, the number of kept NAFs, the compressed factors
up to the sign of each NAF, and E(T) of the compressed domain (float64 path),
for thresholds that keep everything, about half, and few NAFs."""
import numpy as np
import pytest
import torch

from oracle import naf as N
from oracle import triples as T
from paper_2311_10048_gb300 import lno_ot
from paper_2311_10048_gb300.synth import config_domain, make_domain

pytestmark = pytest.mark.gpu


def sign_fixed(B):
    """Each NAF block times the sign of its largest-magnitude element."""
    B = np.array(B)
    flat = B.reshape(B.shape[0], -1)
    idx = np.abs(flat).argmax(axis=1)
    return B * np.sign(flat[np.arange(len(idx)), idx])[:, None, None]


CASES = [("small", dict(nbas=14, nocc=(4, 2), naux=40, L=6.0, seed=3), (0.0, 1e-3, 1e-1)),
         ("c0", None, (1e-2, 1.0))]


@pytest.mark.parametrize("name,kw,epss", CASES)
def test_naf_matches_oracle(lib, name, kw, epss):
    d = config_domain("c0") if kw is None else make_domain(t1_sd=0.02, **kw)
    dd = lno_ot.to_device(d)
    ctx = lno_ot.Context(0, "fp64")
    for eps in epss:
        lam_ref, V, Bu, Bd = N.naf(d["B"][0], d["B"][1], eps)
        comp, lam = ctx.naf(dd, eps)
        np.testing.assert_allclose(lam, lam_ref, rtol=0, atol=1e-12 * lam_ref[0])
        assert comp["naux"] == V.shape[1]
        for s, ref in ((0, Bu), (1, Bd)):
            got = comp["B"][s].cpu().numpy()
            np.testing.assert_allclose(sign_fixed(got), sign_fixed(ref), rtol=0,
                                       atol=1e-11 * np.abs(ref).max())
        e_gpu = ctx.energy(comp)["total"]
        oc, _ = N.compressed_domain(d, eps)
        e_ref = T.energy(oc)["total"]
        assert abs(e_gpu - e_ref) <= 1e-10 * abs(e_ref), (eps, e_gpu, e_ref)
    ctx.close()
