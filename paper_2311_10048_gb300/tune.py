"""Autotuner of the contraction schedule per virtual-space size bucket.

For each bucket it builds one synthetic domain of that virtual size (few
occupied orbitals, so a trial takes milliseconds), times lno_ot_energy with
every candidate row (contraction tile width x triplet-group cap) written to a
one-row table, and keeps the fastest.  The result is the text table the
library reads through lno_ot_options.tune_cache ("vmax bn group_cap").

    python -m paper_2311_10048_gb300.tune out.txt [--precision bf16x6]
"""
from __future__ import annotations

import argparse
import os
import tempfile
import time

BUCKETS = (96, 160, 224, 320, 448)          # vmax of each bucket
# contraction tile widths the library has per precision (S * BN <= 512 TMEM columns)
TILE_WIDTHS = {"bf16x3": (256, 128), "bf16x6": (128, 64), "bf16x10": (128, 96, 64),
               "bf16x15": (64,)}
GROUP_CAPS = (16, 64)


def candidates(precision):
    return [(bn, g) for bn in TILE_WIDTHS.get(precision, (0,)) for g in GROUP_CAPS]


def _time_row(lno_ot, dd, precision, row, reps=2):
    fd, path = tempfile.mkstemp(suffix=".tune")
    with os.fdopen(fd, "w") as f:
        f.write(f"{100000} {row[0]} {row[1]}\n")
    try:
        ctx = lno_ot.Context(0, precision, tune_cache=path)
        ctx.energy(dd)                                   # warm-up
        best = float("inf")
        for _ in range(reps):
            ctx.energy(dd)
            st = ctx.stats()
            best = min(best, st["ms_contract"] + st["ms_energy"])
        ctx.close()
    finally:
        os.unlink(path)
    return best


def autotune(path, precision="bf16x6", buckets=BUCKETS, nocc=(10, 8), log=print):
    """Write the tuning table to ``path``; returns the rows."""
    from . import lno_ot
    from .synth import make_domain
    rows = []
    for vmax in buckets:
        v = vmax - 16
        d = make_domain(v + nocc[0], nocc, naux=3 * (v + nocc[0]), L=0.75 * (v + nocc[0]),
                        seed=vmax)
        dd = lno_ot.to_device(d)
        times = {row: _time_row(lno_ot, dd, precision, row) for row in candidates(precision)}
        best = min(times, key=times.get)
        rows.append((vmax,) + best)
        log(f"bucket v<={vmax}: " + ", ".join(f"bn={c} cap={g}: {t:.2f} ms"
                                            for (c, g), t in times.items()) + f" -> {best}")
        del dd
    with open(path, "w") as f:
        f.write(f"# lno_ot tuning table ({precision}); vmax bn group_cap\n")
        for r in rows:
            f.write(f"{r[0]} {r[1]} {r[2]}\n")
    return rows


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("out")
    ap.add_argument("--precision", default="bf16x6")
    a = ap.parse_args()
    t = time.time()
    autotune(a.out, a.precision)
    print(f"tuned in {time.time() - t:.1f} s -> {a.out}")
