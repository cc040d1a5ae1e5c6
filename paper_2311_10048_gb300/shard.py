"""Host-side sharding of independent LNO domains across GPUs (one process per GPU).

The per-domain (T) energies are independent (the domains of Sec. 3 are
summed in eq lno_ccsdpt_energy), so a batch is split across ranks with no
data-path collective: each rank computes whole domains, and the only
exchanges are the per-domain results (a handful of doubles) and the
max-over-ranks wall time.  Assignment is longest-processing-time first on
the W-contraction flop model, which bounds the slowest rank at 4/3 of the
optimum.
"""
from __future__ import annotations

import heapq


def domain_cost(nbas, nocc):
    """W-contraction flops of one domain (all (b,c) outputs counted)."""
    na, nb = nocc
    va, vb = nbas - na, nbas - nb
    c2 = lambda n: n * (n - 1) // 2
    c3 = lambda n: n * (n - 1) * (n - 2) // 6
    same = lambda v, o: 3.0 * (2 * v ** 4 + 2 * v ** 3 * o)
    mixed = lambda vs, vt, os_, ot: (4 * vs ** 2 * vt ** 2 + 6 * vs ** 3 * vt
                                     + 4 * vs ** 2 * vt * ot + 6 * os_ * vs ** 2 * vt)
    return (c3(na) * same(va, na) + c3(nb) * same(vb, nb)
            + c2(na) * nb * mixed(va, vb, na, nb) + c2(nb) * na * mixed(vb, va, nb, na))


def lpt_shards(costs, world):
    """Assign item indices to `world` ranks, largest cost first onto the
    least-loaded rank.  Returns (list of index lists, per-rank load)."""
    heap = [(0.0, r) for r in range(world)]
    shards = [[] for _ in range(world)]
    load = [0.0] * world
    for i in sorted(range(len(costs)), key=lambda k: (-costs[k], k)):
        l, r = heapq.heappop(heap)
        shards[r].append(i)
        load[r] = l + costs[i]
        heapq.heappush(heap, (load[r], r))
    return [sorted(s) for s in shards], load


def max_over_ranks(value, group=None):
    """Max of a float over the ranks of the default (or given) process group."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return float(value)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def gather_results(local, world, group=None):
    """All ranks' per-domain results (index -> value dict) merged on every rank."""
    import torch.distributed as dist
    if world == 1 or not dist.is_initialized():
        return dict(local)
    out = [None] * world
    dist.all_gather_object(out, dict(local), group=group)
    merged = {}
    for part in out:
        merged.update(part)
    return merged
