"""Write the stored oracle values under tests/golden/.

Calls only ``oracle`` (and the seeded input generator).  Usage:

    python tests/golden/make_golden.py c0        # all triplets, seconds
    python tests/golden/make_golden.py c4        # all triplets, ~1-2 h CPU
    python tests/golden/make_golden.py c1s       # seeded triplet sample of c1
    python tests/golden/make_golden.py c2s       # seeded triplet sample of c2 (~80 GB host)
    python tests/golden/make_golden.py c0f       # c0 plus an f_ov block (add_fov)

``--out DIR`` writes the files to DIR instead of this folder.

Each output file holds the configuration, the per-triplet contributions e_t
(in the oracle's triplet order, or with explicit indices for samples) and the
per-case sums (math.fsum); full runs also hold the orbital contributions
of eq cim_pt_energy (``orbital``: alpha and beta lists).
"""
from __future__ import annotations

import json
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.triples import CASES, Evaluator, orbital_energies, triplets  # noqa: E402
from paper_2311_10048_gb300.synth import CONFIGS, add_fov, config_domain  # noqa: E402

FOV_SD, FOV_SEED = 0.02, 0

SAMPLE_SEED = 20231110
SAMPLE_PER_CASE = 6
# c2: each triplet costs the oracle ~1e12 flops plus ~2 GB of cached integrals
SAMPLE_PER_CASE_CFG = {"c2": 2}


def sample_indices(case, na, nb, k=SAMPLE_PER_CASE, seed=SAMPLE_SEED, ends=True):
    """Seeded sample of triplet indices of one case (first and last included
    when ``ends``)."""
    n = len(triplets(case, na, nb))
    if n == 0:
        return []
    rng = np.random.default_rng(seed + CASES.index(case))
    pick = set(rng.choice(n, size=min(k, n), replace=False).tolist())
    if ends:
        pick.update({0, n - 1})
    return sorted(pick)


def run(name, outdir=HERE):
    import torch
    torch.set_num_threads(int(os.environ.get("ORACLE_THREADS", os.cpu_count())))
    cfg = name[:-1] if name.endswith(("s", "f")) else name
    d = config_domain(cfg)
    if name.endswith("f"):
        d = add_fov(d, sd=FOV_SD, seed=FOV_SEED)
    na, nb = d["nocc"]
    # share the numpy buffers with the oracle (no second copy of a large domain)
    dt = dict(nbas=d["nbas"], naux=d["naux"], nocc=d["nocc"],
              B=[torch.from_numpy(x) for x in d["B"]],
              eps=[torch.from_numpy(x) for x in d["eps"]],
              t1=[torch.from_numpy(x) for x in d["t1"]],
              **{k: torch.from_numpy(d[k]) for k in ("t2aa", "t2bb", "t2ab")})
    if d.get("fov") is not None:
        dt["fov"] = [torch.from_numpy(x) for x in d["fov"]]
    ev = Evaluator(dt)
    out = dict(config=cfg, params=CONFIGS[cfg], cases={})
    if name.endswith("f"):
        out["fov"] = dict(sd=FOV_SD, seed=FOV_SEED)
    t0 = time.time()
    with torch.no_grad():
        for case in CASES:
            trips = triplets(case, na, nb)
            if name.endswith("s"):
                k = SAMPLE_PER_CASE_CFG.get(cfg, SAMPLE_PER_CASE)
                idx = sample_indices(case, na, nb, k=k, ends=cfg not in SAMPLE_PER_CASE_CFG)
                ev._cache.clear()
                e = [float(ev.triplet_energy(case, trips[q])) for q in idx]
                out["cases"][case] = dict(index=idx, e=e)
            else:
                e = [float(ev.triplet_energy(case, t)) for t in trips]
                out["cases"][case] = dict(e=e, sum=math.fsum(e))
            print(name, case, len(e), time.time() - t0, flush=True)
    if not name.endswith("s"):
        out["total"] = math.fsum(out["cases"][c]["sum"] for c in CASES)
        out["orbital"] = orbital_energies(d)
    out["oracle_seconds"] = time.time() - t0
    path = os.path.join(outdir, f"{name}_energy.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=0)
    print("wrote", path)


if __name__ == "__main__":
    args = sys.argv[1:]
    out = HERE
    if "--out" in args:
        i = args.index("--out")
        out = args[i + 1]
        del args[i:i + 2]
        os.makedirs(out, exist_ok=True)
    for n in args:
        run(n, out)
