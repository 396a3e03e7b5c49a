"""Work split of independent problems over ranks (one GPU per rank).

The H² products of different matrices share nothing, so a batch of
independent problems shards without any data-path collective: every rank
builds and multiplies its own share, and only the timing and the work counts
are combined on the host (a max and a sum over ranks).  Shares are chosen by
longest-processing-time-first on an estimate of each problem's bytes, which
is deterministic: every rank computes the same split from the same list.
"""
from __future__ import annotations


def weight(spec):
    """Bytes estimate of one product: n k^2 (the coupling stream dominates) times the padded RHS."""
    k = int(spec["order"]) ** 3
    return int(spec["n"]) * k * k * ((int(spec["nrhs"]) + 3) // 4)


def shard_problems(specs, world):
    """Split specs over world ranks (longest first onto the least-loaded rank, ties to the lowest rank).

    Returns a list of world lists; each keeps the problems' original order.
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    owner = {}
    for s in sorted(specs, key=lambda s: (-weight(s), s["index"])):
        r = min(range(world), key=lambda i: (load[i], i))
        owner[s["index"]] = r
        load[r] += weight(s)
    return [[s for s in specs if owner[s["index"]] == r] for r in range(world)]


def combine(ms, units, group=None):
    """(max of ms, sum of units) over the ranks of the default process group (or this rank alone)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(ms), float(units)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    u = torch.tensor([float(units)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    return float(t.item()), float(u.item())
