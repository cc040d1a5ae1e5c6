"""Host-side logic without a GPU: flop model, batch shapes, sharding (gloo)."""
import math
import os
import socket

import numpy as np
import pytest

from paper_2311_10048_gb300 import shard
from paper_2311_10048_gb300.synth import CONFIGS, c3_shapes


def test_flop_model_matches_published_totals():
    # totals of the W contraction per configuration (counting every (b,c))
    want = {"c0": 1.87e9, "c1": 1.29e16, "c2": 9.75e17, "c4": 9.07e13}
    for name, ref in want.items():
        c = CONFIGS[name]
        got = shard.domain_cost(c["nbas"], c["nocc"])
        assert abs(got - ref) / ref < 0.01, (name, got, ref)


def test_flop_model_equals_bench_model():
    import bench
    for name, c in CONFIGS.items():
        assert math.isclose(bench.total_alg_flops(c["nocc"], c["nbas"]),
                            shard.domain_cost(c["nbas"], c["nocc"]), rel_tol=1e-12)


def test_c3_shapes_statistics():
    s = c3_shapes()
    assert len(s) == 2000
    na = np.array([d["nocc"][0] for d in s])
    nb = np.array([d["nocc"][1] for d in s])
    nv = np.array([d["nbas"] - d["nocc"][0] for d in s])
    assert na.min() >= 8 and na.max() <= 60 and np.all((na - nb >= 1) & (na - nb <= 3))
    assert nv.min() >= 60 and nv.max() <= 400
    assert all(d["naux"] == 3 * d["nbas"] for d in s)
    # the paper's LIS statistics: average 26-32 occupied, 112-131 virtual, virtual ~4-5x occupied
    assert 22 <= na.mean() <= 32 and 4.0 <= (nv / na).mean() <= 8.5
    assert s == c3_shapes()                      # deterministic
    tot = sum(shard.domain_cost(d["nbas"], d["nocc"]) for d in s)
    assert 1.3e19 < tot < 1.6e19


def test_lpt_shards_cover_and_balance():
    rng = np.random.default_rng(0)
    costs = rng.lognormal(0, 1.5, 500).tolist()
    for world in (1, 2, 3, 8):
        shards, load = shard.lpt_shards(costs, world)
        allidx = sorted(i for s in shards for i in s)
        assert allidx == list(range(len(costs)))
        assert max(load) <= (4.0 / 3.0) * max(sum(costs) / world, max(costs)) + 1e-9
        assert math.isclose(sum(load), sum(costs))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    costs = [float(c) for c in range(1, 21)]
    shards, _ = shard.lpt_shards(costs, world)
    mine = shards[rank]
    # each rank "computes" its domains: result = cost squared
    local = {i: costs[i] ** 2 for i in mine}
    merged = shard.gather_results(local, world)
    t = shard.max_over_ranks(10.0 + rank)
    q.put((rank, sorted(mine), merged, t))
    dist.destroy_process_group()


def test_two_rank_gloo_sharding_round_trip():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert sorted(res[0][1] + res[1][1]) == list(range(20))
    assert not set(res[0][1]) & set(res[1][1])
    for _, _, merged, t in res:
        assert merged == {i: float(i + 1) ** 2 for i in range(20)}
        assert t == 11.0


def test_energy_element_counts_match_published_totals():
    import bench
    want = {"c0": 2.1e6, "c1": 1.50e12, "c2": 6.45e13, "c4": 2.1e10}
    for name, ref in want.items():
        c = CONFIGS[name]
        same, mixed = bench.energy_elements(c["nocc"], c["nbas"])
        assert abs(same + mixed - ref) / ref < 0.03, (name, same + mixed, ref)
