"""Benchmark: open-shell domain E(T) on GB300 through the lno_ot C ABI.

Workload: the medium single domain (nbas 400, 40/38 occupied, naux 1200).
The K timed steps together compute the whole domain exactly once: step s is
one lno_ot_energy call over block s of K of every spin case's restricted
triplets (contiguous in the lexicographic triplet order), and runs every
stage of the hot path for that block (staging, DF assembly, operand layout,
W/V contractions, energy reduction) with the inputs resident in HBM.  The
warm-up steps repeat the first blocks.  After the timed region:
  * e2e: a few steps through the same call with the inputs copied from pinned
    host memory inside the timed region;
  * the float64 GPU path on a seeded triplet sample (the comparator), whose
    per-triplet differences give the domain-total error estimate (bias and
    rounding spread, per spin case);
  * optionally (--ref-precision bf16x15) the whole domain once more in
    BF16X15, reported as a difference;
  * the CPU oracle on a bounded triplet sample (cpu_baseline and parity).

Prints ONE JSON line (rank 0).  Under torchrun each rank computes its own
domain of the same shape (seed + rank): weak scaling, no data-path
collective; the wall time is the max over ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2311_10048_gb300.synth import (CONFIGS, add_fov, c3_shapes,  # noqa: E402
                                          domain_bytes, make_domain)

METRIC = "open-shell E(T) TFLOP/s & domains/s at |dE(T)|<=1e-7 Eh vs plain FP64 GPU path"
UNIT = "TFLOP/s"
CASES = ("aaa", "aab", "abb", "bbb")
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        d["source"] = "measured"
        return d
    d = dict(PEAKS_FALLBACK)
    d["source"] = "fallback"
    return d


# DRAM bytes (read + write) per tensor-core flop of the contraction kernel as
# it is now, from one ncu capture per precision on a c1-sized group; the
# per-launch traffic scales with the launch's tensor flops at a fixed virtual
# space.  None is listed while the kernel has changed since its last capture
# (profiles/tc_gemm_sliced_bf16x10_c1shape.md holds the last one, 1.3239e-3
# B/flop, before the register-staged epilogue and the tiled Y/Z' stores), and
# the bench line then reports traffic as null.
DRAM_BYTES_PER_TENSOR_FLOP = {}

# FP32 operations per restricted (abc) element in the float32 energy kernel
# (an FMA counts 2): W 2, V 17 (same spin) / 9 (mixed), W (W + V) 2,
# double-float denominator 9, reciprocal + Newton step + product 6, sum 1.
ENERGY_FLOPS_PER_ELEMENT = {"same": 37, "mixed": 29}


def energy_elements(nocc, nbas):
    """Restricted (abc) elements of the same-spin and mixed cases."""
    na, nb = nocc
    va, vb = nbas - na, nbas - nb
    c2 = lambda n: n * (n - 1) // 2
    c3 = lambda n: n * (n - 1) * (n - 2) // 6
    same = c3(na) * c3(va) + c3(nb) * c3(vb)
    mixed = c2(na) * nb * c2(va) * vb + c2(nb) * na * c2(vb) * va
    return same, mixed


def alg_flops_triplet(case, nocc, nbas):
    """W-contraction flops of one triplet, every (b,c) output counted."""
    na, nb = nocc
    va, vb = nbas - na, nbas - nb
    if case in ("aaa", "bbb"):
        v, o = (va, na) if case == "aaa" else (vb, nb)
        return 3.0 * (2 * v ** 4 + 2 * v ** 3 * o)
    s, t = ((va, na), (vb, nb)) if case == "aab" else ((vb, nb), (va, na))
    vs, os_ = s
    vt, ot = t
    return (4 * vs ** 2 * vt ** 2 + 6 * vs ** 3 * vt + 4 * vs ** 2 * vt * ot
            + 6 * os_ * vs ** 2 * vt)


def ntrip(case, nocc):
    na, nb = nocc
    c2 = lambda n: n * (n - 1) // 2
    c3 = lambda n: n * (n - 1) * (n - 2) // 6
    return {"aaa": c3(na), "bbb": c3(nb), "aab": c2(na) * nb, "abb": c2(nb) * na}[case]


def total_alg_flops(nocc, nbas):
    return sum(alg_flops_triplet(c, nocc, nbas) * ntrip(c, nocc) for c in CASES)


def sample_triplets(nocc, per_case, seed=7):
    """Seeded sample of triplet indices per case (first and last included)."""
    out = []
    for ci, c in enumerate(CASES):
        n = ntrip(c, nocc)
        if n == 0 or per_case == 0:
            out.append(np.zeros(0, dtype=np.int64))
            continue
        rng = np.random.default_rng(seed + ci)
        pick = set(rng.choice(n, size=min(per_case, n), replace=False).tolist())
        out.append(np.array(sorted(pick), dtype=np.int64))
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = tempfile.mktemp(suffix=".csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            try:
                pw.append(float(p[3]))
            except ValueError:
                pass
            for n, v in zip(names, p[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_median": statistics.median(pw) if pw else None,
                "power_w_max": max(pw) if pw else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def cpu_oracle_sample(dom, sel, max_seconds=30.0):
    """Time the CPU oracle on the sampled triplets (host cores).

    Returns (values {case: [e_t]}, seconds, algorithmic flops, threads).
    """
    import torch
    from oracle.triples import Evaluator, triplets
    torch.set_num_threads(os.cpu_count() or 1)
    ev = Evaluator(dom)
    na, nb = dom["nocc"]
    vals, flops = {}, 0.0
    t0 = time.time()
    with torch.no_grad():
        for ci, c in enumerate(CASES):
            trs = triplets(c, na, nb)
            vals[c] = []
            for q in sel[ci]:
                vals[c].append(float(ev.triplet_energy(c, trs[int(q)])))
                flops += alg_flops_triplet(c, dom["nocc"], dom["nbas"])
                if time.time() - t0 > max_seconds:
                    break
    return vals, time.time() - t0, flops, torch.get_num_threads()


def run_reference(args):
    """Reference arm: the CPU oracle, as it stands, one triplet per step.

    Step s evaluates one seeded triplet of the workload (the cases in turn);
    W untimed warm-up steps, then K timed steps.  The oracle's lazily built
    integral cache is emptied before every step so that each step pays for
    the whole triplet and the host memory stays bounded."""
    import torch
    from oracle.triples import Evaluator, triplets
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cfg = dict(CONFIGS[args.config])
    dom = make_domain(**cfg)
    torch.set_num_threads(os.cpu_count() or 1)
    na, nb = dom["nocc"]
    nsteps = max(1, args.steps)
    sel = sample_triplets(dom["nocc"], (nsteps + args.warmup + 3) // 4 + 1, seed=29)
    order = [(ci, int(q)) for k in range(max(len(x) for x in sel))
             for ci in range(4) if k < len(sel[ci]) for q in [sel[ci][k]]]
    ev = Evaluator(dom)
    trs = {c: triplets(c, na, nb) for c in CASES}
    times, flops, counts = [], 0.0, {c: 0 for c in CASES}
    with torch.no_grad():
        for st in range(args.warmup + nsteps):
            ci, q = order[st % len(order)]
            c = CASES[ci]
            ev._cache.clear()
            t0 = time.perf_counter()
            ev.triplet_energy(c, trs[c][q])
            dt = time.perf_counter() - t0
            if st >= args.warmup:
                times.append(dt)
                flops += alg_flops_triplet(c, dom["nocc"], dom["nbas"])
                counts[c] += 1
    sec = sum(times)
    value = flops / sec / 1e12
    cores = torch.get_num_threads()
    sample = (f"{nsteps} seeded triplets of {args.config}, one per step "
              f"({', '.join(f'{c}:{counts[c]}' for c in CASES)}), after {args.warmup} warm-up "
              f"triplets")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": nsteps, "warmup": args.warmup,
        "ms_per_step": sec * 1e3 / nsteps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args.config), **cfg_public(cfg)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def workload_name(cfg):
    c = CONFIGS[cfg]
    return (f"single LNO domain E(T): nbas={c['nbas']} nocc={c['nocc'][0]}/{c['nocc'][1]} "
            f"naux={c['naux']} (all four spin cases)")


def cfg_public(cfg):
    return {"nbas": cfg["nbas"], "nocc": list(cfg["nocc"]), "naux": cfg["naux"],
            "B_decay_length": cfg["L"], "seed": cfg["seed"]}


def c3_sample(n, upto=0.75):
    """Stratified sample of the 2000-domain batch: n domains evenly spaced in
    the cost ranking up to the `upto` quantile (the top quarter of the
    domains alone takes hours; the sample keeps a bench run within minutes).  Returns (indices, shapes,
    total algorithmic flops of all 2000 domains)."""
    shapes = c3_shapes()
    cost = [total_alg_flops(s["nocc"], s["nbas"]) for s in shapes]
    order = sorted(range(len(shapes)), key=lambda d: cost[d])
    top = int(upto * (len(order) - 1))
    pick = sorted({order[round(k * top / max(1, n - 1))] for k in range(n)})
    return pick, shapes, float(sum(cost))


def run_c3(args):
    """Batched mode: lno_ot_energy_batched over a stratified c3 sample.

    Under torchrun the sampled domains are split across ranks by LPT on the
    flop model (strong scaling over the sample, no data-path collective)."""
    import torch
    import torch.distributed as dist
    from paper_2311_10048_gb300 import lno_ot, shard, tune
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pick, shapes, total_flops = c3_sample(args.c3_sample)
    costs = [total_alg_flops(shapes[d]["nocc"], shapes[d]["nbas"]) for d in pick]
    parts, _ = shard.lpt_shards(costs, world)
    mine = [pick[q] for q in parts[rank]]
    t0 = time.time()
    doms = [make_domain(**shapes[d]) for d in mine]
    t_gen = time.time() - t0
    tune_path = os.path.join(tempfile.gettempdir(), f"lno_ot_tune_{args.precision}_{local}.txt")
    t0 = time.time()
    rows = tune.autotune(tune_path, args.precision, log=lambda *a: None)
    t_tune = time.time() - t0
    dds = [lno_ot.to_device(d, dev) for d in doms]
    ctx = lno_ot.Context(local, args.precision, tune_cache=tune_path)
    for _ in range(args.warmup):
        if dds:
            rc, res = ctx.energy_batched(dds)
            assert rc == 0, rc
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = []
    with ClockSampler(local) as clk:
        e0.record(st)
        for _ in range(args.steps):
            if dds:
                rc, res = ctx.energy_batched(dds)
        e1.record(st)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = shard.max_over_ranks(e0.elapsed_time(e1) / args.steps)
    stats = ctx.stats()
    ctx.close()
    energies = shard.gather_results({d: r["total"] for d, r in zip(mine, res)}, world)
    flops = float(sum(costs))
    value = flops / (ms / 1e3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "strong" if world > 1 else "weak", "vs_baseline": None,
        "dtype": "bf16", "data": "synthetic",
        "config": {"workload": (f"batched LNO domains: stratified sample of {len(pick)} of the "
                                f"2000-domain batch (lognormal occupied counts, see synth.c3_shapes)"),
                   "domains": [dict(shapes[d], index=d) for d in pick],
                   "l2": "inputs larger than L2",
                   "parallelism": f"LPT shards of whole domains over {world} GPU(s)"},
        "domains_per_s": len(pick) / (ms / 1e3),
        "full_batch_flops": total_flops,
        "full_batch_estimate_h": total_flops / (value * 1e12) / 3600,
        "tuning_table": rows, "tune_seconds": t_tune, "gen_seconds": t_gen,
        "energies_Eh": {int(k): v for k, v in sorted(energies.items())},
        "breakdown_ms_rank0": {k: stats[k] for k in ("ms_total", "ms_stage", "ms_contract",
                                                     "ms_energy")},
        "contraction_tflops_per_launch_rank0": (stats["tensor_flops"] / stats["ms_contract"] / 1e9
                                                if stats["ms_contract"] > 0 else None),
        "energy_elements_per_s_rank0": (stats["elements"] / stats["ms_energy"] * 1e3
                                        if stats["ms_energy"] > 0 else None),
        "gpu_launches": int(stats["contract_launches"] + stats["energy_launches"]
                            + stats["other_launches"]),
        "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_backward(args):
    """Adjoint timing: lno_ot_backward (W recomputed per triplet) on a seeded
    triplet sample of the domain, against its forward on the same sample, both
    in --precision (a tensor-core precision runs the adjoint's contractions on
    the tensor cores, float64 runs them in float64)."""
    import torch
    from paper_2311_10048_gb300 import lno_ot
    cfg = dict(CONFIGS[args.config])
    dom = make_domain(**cfg)
    nbas, nocc = dom["nbas"], dom["nocc"]
    sel = sample_triplets(nocc, args.bwd_sample, seed=13)
    dev = torch.device("cuda", 0)
    dd = lno_ot.to_device(dom, dev)
    ctx = lno_ot.Context(0, args.precision)
    g = dict(dB=[torch.empty_like(dd["B"][0]), torch.empty_like(dd["B"][1])],
             deps=[torch.empty_like(dd["eps"][0]), torch.empty_like(dd["eps"][1])],
             dt1=[torch.empty_like(dd["t1"][0]), torch.empty_like(dd["t1"][1])],
             dt2aa=torch.empty_like(dd["t2aa"]), dt2bb=torch.empty_like(dd["t2bb"]),
             dt2ab=torch.empty_like(dd["t2ab"]))
    ctx.backward(dd, 1.0, g, trip_sel=sel)        # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.backward(dd, 1.0, g, trip_sel=sel)
    torch.cuda.synchronize()
    t_bwd = time.perf_counter() - t0
    bst = ctx.stats()
    t0 = time.perf_counter()
    ctx.energy(dd, trip_sel=sel)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    fst = ctx.stats()
    ctx.close()
    ntr = sum(len(x) for x in sel)
    flops = sum(alg_flops_triplet(c, nocc, nbas) * len(sel[ci]) for ci, c in enumerate(CASES))
    line = {"metric": "E(T) adjoint (dE/dB, deps, dT1, dT2) wall time on a triplet sample",
            "value": t_bwd, "unit": "s", "higher_is_better": False,
            "dtype": "f64" if args.precision == "fp64" else "bf16",
            "precision": args.precision,
            "adjoint_contractions": ("float64 CUDA cores" if args.precision == "fp64" else
                                     "tensor cores, 4 exact BF16 slices, float64 output"),
            "data": "synthetic", "steps": 1, "warmup": 1,
            "config": {"workload": workload_name(args.config) + " (adjoint)", **cfg_public(cfg),
                       "sample": f"{ntr} seeded triplets ({', '.join(f'{c}:{len(sel[i])}' for i, c in enumerate(CASES))})"},
            "forward_same_sample_s": t_fwd,
            "backward_over_forward": t_bwd / t_fwd,
            "sample_algorithmic_flops": flops,
            "forward_breakdown_ms": {k: fst[k] for k in ("ms_stage", "ms_contract", "ms_energy")},
            "backward_breakdown_ms": {
                "ms_total": bst["ms_total"],
                "ms_stage_and_operand_build": bst["ms_stage"],
                "ms_contractions": bst["ms_contract"],
                "ms_energy_adjoint": bst["ms_energy"]},
            "w_recomputed_per_triplet": True}
    print(json.dumps(line), flush=True)
    return 0


def run_central(args):
    """Central-LMO share in the Laplace form (Sec. 3.7): one seeded random
    central orbital of each spin of the domain, the laptol = 1e-2 quadrature
    from the library; times lno_ot_energy_central (all stages, per call)."""
    import torch
    from paper_2311_10048_gb300 import lno_ot
    cfg = dict(CONFIGS[args.config])
    dom = make_domain(**cfg)
    nbas, nocc = dom["nbas"], dom["nocc"]
    dev = torch.device("cuda", 0)
    dd = lno_ot.to_device(dom, dev)
    eo = np.sort(np.concatenate([dom["eps"][0][:nocc[0]], dom["eps"][1][:nocc[1]]]))
    ev = np.sort(np.concatenate([dom["eps"][0][nocc[0]:], dom["eps"][1][nocc[1]:]]))
    lo, hi = ev[:3].sum() - eo[-3:].sum(), ev[-3:].sum() - eo[:3].sum()
    s, w = lno_ot.laplace_quadrature(lo, hi, 1e-2)
    rng = np.random.default_rng(17)
    U = []
    for x in (0, 1):
        u = rng.standard_normal((1, nocc[x]))
        U.append(torch.as_tensor(u / np.linalg.norm(u), dtype=torch.float64, device=dev))
    ctx = lno_ot.Context(0, args.precision)
    for _ in range(args.warmup if args.warmup < 3 else 1):
        ctx.energy_central(dd, 0, U[0], s, w)
    torch.cuda.synchronize()
    res, secs, stats = [], [], []
    for x in (0, 1):
        t0 = time.perf_counter()
        res.append(float(ctx.energy_central(dd, x, U[x], s, w)[0]))
        secs.append(time.perf_counter() - t0)
        stats.append(ctx.stats())
    ctx.close()
    na, nb = nocc
    c2 = lambda n: n * (n - 1) // 2
    # triplets per central orbital and quadrature point: same-spin pairs,
    # same-spin x other-spin, other-spin pairs
    fl = 0.0
    for x, (o, ot) in enumerate(((na, nb), (nb, na))):
        cs = ("aaa", "aab", "abb") if x == 0 else ("bbb", "abb", "aab")
        fl += len(s) * (c2(o) * alg_flops_triplet(cs[0], nocc, nbas)
                        + o * ot * alg_flops_triplet(cs[1], nocc, nbas)
                        + c2(ot) * alg_flops_triplet(cs[2], nocc, nbas))
    line = {"metric": "central-LMO (T) share, Laplace form (eq local_pt): TFLOP/s",
            "value": fl / sum(secs) / 1e12, "unit": UNIT, "higher_is_better": True,
            "dtype": "bf16" if args.precision != "fp64" else "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.config) + "; one random central orbital "
                                                               "per spin", **cfg_public(cfg)},
            "quadrature": {"points": len(s), "laptol": 1e-2, "range_Eh": [lo, hi],
                           "s": s.tolist(), "w": w.tolist()},
            "dE_Eh": {"spin_up": res[0], "spin_down": res[1]},
            "seconds": {"spin_up": secs[0], "spin_down": secs[1]},
            "breakdown_ms": [{k: st[k] for k in ("ms_total", "ms_stage", "ms_contract",
                                                 "ms_energy")} for st in stats],
            "precision": args.precision}
    print(json.dumps(line), flush=True)
    return 0


def run_naf(args):
    """NAF compression (Sec. 3.6): time lno_ot_naf at eps_naf = 1e-2 and at a
    threshold that keeps about half of the auxiliary functions, and the E(T)
    change of the compressed domain (timed precision)."""
    import torch
    from paper_2311_10048_gb300 import lno_ot
    cfg = dict(CONFIGS[args.config])
    dom = make_domain(**cfg)
    dd = lno_ot.to_device(dom, torch.device("cuda", 0))
    c64 = lno_ot.Context(0, "fp64")
    c64.naf(dd, 1e-2)      # warm-up
    torch.cuda.synchronize()
    out = {}
    t0 = time.perf_counter()
    comp, lam = c64.naf(dd, 1e-2)
    out["1e-2"] = {"seconds": time.perf_counter() - t0, "naux_kept": comp["naux"]}
    eps_half = float(lam[len(lam) // 2])
    t0 = time.perf_counter()
    comp_h, _ = c64.naf(dd, eps_half)
    out["half"] = {"eps_naf": eps_half, "seconds": time.perf_counter() - t0,
                   "naux_kept": comp_h["naux"]}
    c64.close()
    del comp
    e_full = e_half = None
    if dom["nbas"] <= 200:   # E(T) of the full and the compressed domain (small domains)
        ctx = lno_ot.Context(0, args.precision)
        e_full = ctx.energy(dd)["total"]
        e_half = ctx.energy(comp_h)["total"]
        ctx.close()
    line = {"metric": "NAF compression (eq naf_w) seconds and E(T) change", "unit": "s",
            "value": out["1e-2"]["seconds"], "higher_is_better": False, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(args.config), **cfg_public(cfg)},
            "naux": dom["naux"], "eigenvalues": {"max": float(lam[0]), "min": float(lam[-1])},
            "runs": out, "E_full_Eh": e_full, "E_half_naf_Eh": e_half,
            "dE_half_Eh": None if e_full is None else e_half - e_full,
            "energy_precision": args.precision}
    print(json.dumps(line), flush=True)
    return 0


def step_blocks(nocc, K):
    """trip_sel of each of K steps: block s of every case's triplets."""
    out = []
    for st in range(K):
        sel = []
        for c in CASES:
            n = ntrip(c, nocc)
            sel.append(np.arange(n * st // K, n * (st + 1) // K, dtype=np.int64))
        out.append(sel)
    return out


def sel_flops(sel, nocc, nbas):
    return sum(alg_flops_triplet(c, nocc, nbas) * len(sel[ci]) for ci, c in enumerate(CASES))


def err_stats(d):
    d = np.asarray(d, dtype=np.float64)
    if d.size == 0:
        return None
    return {"n": int(d.size), "max_abs_Eh": float(np.abs(d).max()), "mean_Eh": float(d.mean()),
            "sd_Eh": float(d.std(ddof=1)) if d.size > 1 else 0.0}


def run_domain(args):
    import torch
    import torch.distributed as dist
    from paper_2311_10048_gb300 import lno_ot

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    cfg = dict(CONFIGS[args.config])
    cfg["seed"] = cfg["seed"] + 1000 * rank
    if args.closed_shell:
        cfg["nocc"] = (cfg["nocc"][0], cfg["nocc"][0])
        cfg["closed_shell"] = True
    t_gen = time.time()
    dom = make_domain(**cfg)
    if args.fov:
        dom = add_fov(dom, sd=0.02, seed=cfg["seed"])
    t_gen = time.time() - t_gen
    nbas, nocc = dom["nbas"], dom["nocc"]
    K = max(1, args.steps)
    ntr = [ntrip(c, nocc) for c in CASES]
    N_all = sum(ntr)
    # the triplets the steps compute: the whole domain, or a seeded sample of
    # --triplet-sample per case (domains too large to time whole)
    sampled = args.triplet_sample > 0
    universe = (sample_triplets(nocc, args.triplet_sample, seed=23) if sampled
                else [np.arange(n, dtype=np.int64) for n in ntr])
    nun = [len(u) for u in universe]
    blocks = [[universe[ci][nun[ci] * st // K:nun[ci] * (st + 1) // K] for ci in range(4)]
              for st in range(K)]
    bpos = [[(nun[ci] * st // K, nun[ci] * (st + 1) // K) for ci in range(4)] for st in range(K)]

    def positions(per_case, seed):
        # seeded positions within the universe, per case
        out = []
        for ci in range(4):
            n = nun[ci]
            if n == 0 or per_case == 0:
                out.append(np.zeros(0, dtype=np.int64))
                continue
            rng = np.random.default_rng(seed + ci)
            out.append(np.sort(rng.choice(n, size=min(per_case, n), replace=False)))
        return out

    # CPU baseline (rank 0, single GPU only): the oracle on a bounded sample
    cpu = None
    oracle_vals = None
    pos_cpu = positions(args.cpu_sample, 7)
    sel_cpu = [universe[ci][pos_cpu[ci]] for ci in range(4)]
    if rank == 0 and world == 1 and args.cpu_sample > 0:
        oracle_vals, sec, flops, cores = cpu_oracle_sample(dom, sel_cpu, args.cpu_seconds)
        nor = sum(len(v) for v in oracle_vals.values())
        cpu = {"value": flops / sec / 1e12, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{nor} seeded triplets of the same domain "
                         f"({', '.join(f'{c}:{len(oracle_vals[c])}' for c in CASES)}), "
                         f"{sec:.1f} s"}

    dd = lno_ot.to_device(dom, dev)
    if args.closed_shell:  # the closed-shell calling form: one set of arrays for both spins
        dd = dict(dd, B=[dd["B"][0]] * 2, eps=[dd["eps"][0]] * 2, t1=[dd["t1"][0]] * 2,
                  t2bb=dd["t2aa"])
    # the context keeps the domain's DF blocks and contraction operands
    # between the steps (built once, for all triplets, by the first step)
    ctx = lno_ot.Context(local, args.precision, keep_operands=not (args.no_keep or sampled),
                         tune_cache=args.tune)
    alg = sum(alg_flops_triplet(c, nocc, nbas) * nun[ci] for ci, c in enumerate(CASES))
    # per-triplet contributions of the computed triplets, written block by block
    et = [torch.zeros(max(n, 1), dtype=torch.float64, device=dev) for n in nun]
    eorb = ([torch.zeros(max(n, 1), dtype=torch.float64, device=dev) for n in nocc]
            if args.fov else None)

    def views(st):
        return [et[ci][bpos[st][ci][0]:bpos[st][ci][1]] if bpos[st][ci][1] > bpos[st][ci][0]
                else None for ci in range(4)]

    def step(st, **kw):
        sel = blocks[st % K]
        if args.closed_shell and K == 1 and not sampled:   # whole domain: spin-flip shortcut
            return ctx.energy(dd, e_trip=views(st % K), e_orb=eorb, **kw)
        return ctx.energy(dd, e_trip=views(st % K), trip_sel=sel, e_orb=eorb, **kw)

    for w in range(args.warmup):
        step(w)
    # the timed region builds the operands again: nothing prepared by the
    # warm-up is reused
    ctx.release()
    torch.cuda.synchronize()

    # timed region: K steps = the whole domain once, device-resident inputs
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    st_ = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats, outs = [], []
    with ClockSampler(local) as clk:
        e0.record(st_)
        for s_ in range(K):
            outs.append(step(s_))
            stats.append(ctx.stats())
        e1.record(st_)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    t_local = torch.tensor([ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t_local, op=dist.ReduceOp.MAX)
    ms_max = float(t_local.item())
    ms_step = ms_max / K
    value = alg * world / (ms_max / 1e3) / 1e12
    clocks = clk.summary()
    e_case = {c: math.fsum(o[c] for o in outs) for c in CASES}
    e_case["total"] = math.fsum(e_case[c] for c in CASES)
    et_host = [x[:n].cpu().numpy() for x, n in zip(et, nun)]   # in universe order

    parity = None
    if oracle_vals is not None:
        errs = []
        for ci, c in enumerate(CASES):
            for q, ref in zip(pos_cpu[ci], oracle_vals[c]):
                errs.append(abs(float(et_host[ci][int(q)]) - ref))
        parity = {"sampled_triplets": len(errs), "max_abs_dE_per_triplet_Eh": max(errs),
                  "tolerance_Eh": 1e-8, "vs": "CPU oracle"}

    # end to end: host (pinned) inputs -> device -> E(T) of the step's block -> host
    e2e = None
    if args.e2e_steps > 0:
        host = {k: dom[k] for k in ("B", "eps", "t1", "t2aa", "t2bb", "t2ab")
                + (("fov",) if args.fov else ())}
        pinned, h2d = {}, 0
        for k, v in host.items():
            if isinstance(v, list):
                pinned[k] = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory() for x in v]
                h2d += sum(int(x.size) * 8 for x in v)
            else:
                pinned[k] = torch.from_numpy(np.ascontiguousarray(v)).pin_memory()
                h2d += int(v.size) * 8
        torch.cuda.synchronize()
        fl = 0.0
        t0 = time.perf_counter()
        for s_ in range(args.e2e_steps):
            dn = dict(nbas=nbas, naux=dom["naux"], nocc=nocc)
            for k, v in pinned.items():
                dn[k] = ([x.to(dev, non_blocking=True) for x in v] if isinstance(v, list)
                         else v.to(dev, non_blocking=True))
            sel = blocks[s_ % K]
            ctx.energy(dn, trip_sel=sel)        # returns after the result is on the host
            fl += sel_flops(sel, nocc, nbas)
            del dn
        e2e_s = (time.perf_counter() - t0) / args.e2e_steps
        e2e = {"value": fl / args.e2e_steps / e2e_s / 1e12, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": 40,
               "steps": args.e2e_steps, "seconds_per_step": e2e_s,
               "what": "lno_ot_energy on one step's triplet block; every step copies the whole "
                       "domain's inputs from pinned host memory (new device arrays, so the "
                       "step also stages them and builds all operands) and reads the 5 "
                       "energies back"}
    ctx.close()

    # plain FP64 GPU path on a seeded triplet sample (same domain, same GPU)
    fp64, e64, accuracy_fp64 = None, None, None
    pos64 = positions(args.fp64_sample, 11)
    fsel = [universe[ci][pos64[ci]] for ci in range(4)]
    if args.fp64_sample > 0:
        c64 = lno_ot.Context(local, "fp64")
        et64 = [torch.zeros(max(len(x), 1), dtype=torch.float64, device=dev) for x in fsel]
        c64.energy(dd, trip_sel=fsel, e_trip=et64)
        s64 = c64.stats()
        c64.close()
        e64 = [x[:len(q)].cpu().numpy() for x, q in zip(et64, fsel)]
        fl = sel_flops(fsel, nocc, nbas)
        kern_ms = s64["ms_contract"] + s64["ms_energy"]
        v64 = fl / (kern_ms / 1e3) / 1e12
        fp64 = {"value": v64, "unit": UNIT,
                "value_whole_call": fl / (s64["ms_total"] / 1e3) / 1e12,
                "sample": f"{sum(len(x) for x in fsel)} seeded triplets ({args.fp64_sample} per "
                          f"case); value = contraction + energy kernels, value_whole_call adds "
                          f"its float64 DF assembly of the orbitals the sample uses",
                "speedup_of_timed_precision": value / world / v64}
        d = [et_host[ci][pos64[ci]] - e64[ci] for ci in range(4)]
        fp64["timed_precision_minus_fp64_per_triplet"] = err_stats(np.concatenate(d))
        # domain-total error of the timed precision from the sample, per case:
        # bias N_c mean_c (its 1-sigma uncertainty N_c sd_c / sqrt(n_c)) and the
        # unbiased rounding part sqrt(N_c) sd_c
        bias, bias_u, rnd = 0.0, 0.0, 0.0
        per_case = {}
        for ci, c in enumerate(CASES):
            if len(d[ci]) < 2:
                continue
            m, sd, nn = float(np.mean(d[ci])), float(np.std(d[ci], ddof=1)), len(d[ci])
            per_case[c] = {"n": nn, "mean_Eh": m, "sd_Eh": sd, "N": ntr[ci]}
            bias += ntr[ci] * m
            bias_u += (ntr[ci] * sd / math.sqrt(nn)) ** 2
            rnd += ntr[ci] * sd * sd
        bias_u, rnd = math.sqrt(bias_u), math.sqrt(rnd)
        sig = math.sqrt(bias_u ** 2 + rnd ** 2)
        verdict = ("yes" if abs(bias) + 3 * sig <= 1e-7
                   else "no" if abs(bias) - 3 * sig > 1e-7 else "undetermined at 3 sigma")
        accuracy_fp64 = {
            "method": "per-triplet timed-precision minus float64-path values on the seeded "
                      "sample, per spin case; domain total = sum_c N_c x (mean_c, and the "
                      "rounding spread sqrt(N_c) sd_c)",
            "per_case": per_case, "bias_estimate_Eh": bias, "bias_estimate_1sigma_Eh": bias_u,
            "rounding_1sigma_Eh": rnd, "domain_total_estimate_Eh": [bias, sig],
            "meets_1e-7_Eh": verdict}

    # domain-total error: the whole domain again in BF16X15
    accuracy = None if fp64 is None else {"vs_fp64_sample": accuracy_fp64}
    if args.ref_precision != "none" and args.precision != args.ref_precision:
        cref = lno_ot.Context(local, args.ref_precision)
        etr = [torch.zeros(max(n, 1), dtype=torch.float64, device=dev) for n in nun]
        t0 = time.perf_counter()
        outr = cref.energy(dd, e_trip=etr, trip_sel=universe if sampled else None)
        t_ref = time.perf_counter() - t0
        cref.close()
        etr_h = [x[:n].cpu().numpy() for x, n in zip(etr, nun)]
        diff = {c: math.fsum((et_host[ci] - etr_h[ci]).tolist()) for ci, c in enumerate(CASES)}
        dtot = math.fsum(diff.values())
        accuracy = dict(accuracy or {})
        accuracy.update({"reference": args.ref_precision.upper(), "reference_seconds": t_ref,
                    "reference_energy_Eh": outr["total"],
                    "timed_minus_reference_Eh": {**diff, "total": dtot},
                    "max_abs_per_triplet_Eh": float(max(np.abs(et_host[ci] - etr_h[ci]).max()
                                                        for ci in range(4) if nun[ci]))})
        if e64 is not None:
            dr = np.concatenate([etr_h[ci][pos64[ci]] - e64[ci] for ci in range(4)])
            stt = err_stats(dr)
            # the reference's own domain-total error, from the float64 sample:
            # N (|mean| + 3 sd / sqrt(n)) over all N triplets of the domain
            ref_bound = N_all * (abs(stt["mean_Eh"]) + 3 * stt["sd_Eh"] / math.sqrt(stt["n"]))
            accuracy["reference_minus_fp64_per_triplet"] = stt
            accuracy["reference_total_error_bound_Eh"] = ref_bound
            accuracy["domain_total_abs_dE_bound_Eh"] = abs(dtot) + ref_bound
            accuracy["meets_1e-7_Eh"] = abs(dtot) + ref_bound <= 1e-7

    pk = peaks()
    tot = {k: sum(s[k] for s in stats) for k in ("ms_contract", "ms_energy", "ms_stage",
                                                  "ms_total", "tensor_flops")}
    nlaunch = sum(s["contract_launches"] for s in stats)
    tc_launch_ms = tot["ms_contract"] / max(1, nlaunch)
    tc_flops_launch = tot["tensor_flops"] / max(1, nlaunch)
    achieved = tc_flops_launch / (tc_launch_ms / 1e3) / 1e12
    peak = pk.get("bf16_tflops_sustained", PEAKS_FALLBACK["bf16_tflops_sustained"])
    launches = sum(s["contract_launches"] + s["energy_launches"] + s["other_launches"]
                   for s in stats)
    bpf = DRAM_BYTES_PER_TENSOR_FLOP.get(args.precision)
    traffic = bpf * tc_flops_launch / 1e9 if bpf else None
    # the float32 energy kernel is bound by the FP32 ALUs: peak = 152 SMs x 128
    # FP32 lanes x 2 flop (FMA) x the SM clock seen under load
    n_same, n_mixed = energy_elements(nocc, nbas)
    passes = 2 if args.fov else 1
    en_flops = passes * (n_same * ENERGY_FLOPS_PER_ELEMENT["same"]
                         + n_mixed * ENERGY_FLOPS_PER_ELEMENT["mixed"])
    mhz = clocks.get("sm_mhz") or 2070.0
    en_peak = 152 * 128 * 2 * mhz * 1e6 / 1e12
    en_achieved = en_flops / (tot["ms_energy"] / 1e3) / 1e12
    # its HBM floor: every restricted element reads three float32 intermediates
    # once (X[a,(bc)], X[b,(ac)], X[c,(ab)]; mixed: Y twice and Z' once)
    en_bytes = passes * 12.0 * (n_same + n_mixed)
    en_gbs = en_bytes / (tot["ms_energy"] / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": K, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16", "data": "synthetic",
        "precision": (f"{args.precision.upper()}: exact BF16 slices of float64 operands on "
                      f"tcgen05 (FP32 TMEM accumulators per weight class), float64 "
                      f"denominators and compensated sums"),
        "config": {"workload": (f"single LNO domain E(T): nbas={nbas} nocc={nocc[0]}/{nocc[1]} "
                                f"naux={dom['naux']}, closed shell" if args.closed_shell
                                else workload_name(args.config))
                   + (" + f_ov (RO reference)" if args.fov else "")
                   + (f"; the {K} timed steps compute a seeded sample of {args.triplet_sample} "
                      f"triplets per spin case once (block s of {K} of each case's sample)"
                      if sampled else
                      f"; the {K} timed steps compute the whole domain once (step s: block s "
                      f"of {K} of every spin case's restricted triplets; the first step also "
                      f"stages the domain and builds its DF blocks and contraction operands, "
                      f"which the context keeps for the later steps)"),
                   **cfg_public(cfg), **({"fov_sd": 0.02} if args.fov else {}),
                   "triplets": dict(zip(CASES, ntr)),
                   **({"timed_triplet_sample": dict(zip(CASES, nun)),
                       "sample_flop_fraction": alg / total_alg_flops(nocc, nbas)}
                      if sampled else {}),
                   "l2": f"inputs larger than L2 ({domain_bytes(nbas, nocc, dom['naux']) / 1e9:.1f} GB)",
                   "parallelism": f"replicas x{world} (one domain per GPU)"},
        "domains_per_s": None if sampled else world / (ms_max / 1e3),
        "energy_Eh": e_case,
        "accuracy": accuracy,
        "parity": parity,
        "roofline": {"kernel": "tc_gemm_sliced (W contraction)", "bound": "tensor",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "traffic_unit": "GB per launch (ncu DRAM bytes per tensor flop, scaled)",
                     "peak_source": f"{pk['source']} bf16 sustained",
                     "per_launch": {"ms": tc_launch_ms, "tensor_flops": tc_flops_launch,
                                    "launches": nlaunch}},
        "roofline_energy": {"kernel": "energy_f32 (W/V assembly, W(W+V)/D, sums)",
                            "bound": "hbm", "achieved": en_gbs, "peak": pk["hbm_gbs"],
                            "unit": "GB/s", "frac": en_gbs / pk["hbm_gbs"],
                            "algorithmic_bytes": en_bytes,
                            "bytes_per_element": 12, "elements": n_same + n_mixed,
                            "passes": passes, "peak_source": f"{pk['source']} copy bandwidth",
                            "alu": {"achieved": en_achieved, "peak": en_peak,
                                    "unit": "TFLOP/s (FP32)", "frac": en_achieved / en_peak,
                                    "peak_source": "152 SMs x 128 FP32 lanes x 2 x median SM "
                                                   "clock"}},
        "breakdown_ms": {"ms_total": tot["ms_total"], "ms_stage": tot["ms_stage"],
                         "ms_contract": tot["ms_contract"], "ms_energy": tot["ms_energy"]},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "cpu_baseline": cpu,
        "fp64_gpu_path": fp64,
        "e2e": e2e,
        "gen_seconds": t_gen,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20,
                    help="timed steps; together they compute the whole domain once")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c1", choices=sorted(CONFIGS) + ["custom", "c3"])
    ap.add_argument("--c3-sample", type=int, default=8, help="domains of the c3 batch")
    ap.add_argument("--backward", action="store_true", help="time the adjoint on a sample")
    ap.add_argument("--bwd-sample", type=int, default=1, help="adjoint triplets per case")
    ap.add_argument("--precision", default="bf16x10",
                    choices=["bf16x15", "bf16x10", "bf16x6", "bf16x3", "fp64"])
    ap.add_argument("--ref-precision", default="none", choices=["bf16x15", "none"],
                    help="also run the whole domain in BF16X15 and report the difference")
    ap.add_argument("--cpu-sample", type=int, default=2, help="oracle triplets per case")
    ap.add_argument("--cpu-seconds", type=float, default=30.0)
    ap.add_argument("--fp64-sample", type=int, default=64, help="FP64-path triplets per case")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--triplet-sample", type=int, default=0,
                    help="time a seeded sample of this many triplets per case instead of the "
                         "whole domain (for domains too large to time whole, e.g. c2)")
    ap.add_argument("--tune", default=None,
                    help="tuning table (vmax bn group_cap lines) for the timed context")
    ap.add_argument("--no-keep", action="store_true",
                    help="every step builds its own operands (no keep_operands)")
    ap.add_argument("--closed-shell", action="store_true",
                    help="closed-shell domain (nocc of spin up for both spins, identical data); "
                         "both spins passed as the same arrays, so the spin-flip images run once")
    ap.add_argument("--fov", action="store_true",
                    help="restricted open-shell domain: add an f_ov block (and time the "
                         "orbital contributions too)")
    ap.add_argument("--central", action="store_true",
                    help="time the central-LMO share in the Laplace form (eq local_pt)")
    ap.add_argument("--naf", action="store_true", help="time the NAF compression (eq naf_w)")
    ap.add_argument("--shape", default=None,
                    help="custom domain nbas,nalpha,nbeta,naux (recipe of the configs, seed 5)")
    args = ap.parse_args()
    if args.shape:
        nbas_, na_, nb_, naux_ = (int(x) for x in args.shape.split(","))
        CONFIGS["custom"] = dict(nbas=nbas_, nocc=(na_, nb_), naux=naux_, L=naux_ / 4.0, seed=5)
        args.config = "custom"
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.config == "c3":
        return run_c3(args)
    if args.backward:
        return run_backward(args)
    if args.central:
        return run_central(args)
    if args.naf:
        return run_naf(args)
    return run_domain(args)


if __name__ == "__main__":
    sys.exit(main())
