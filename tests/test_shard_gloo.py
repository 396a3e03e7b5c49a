"""Multi-rank host logic on CPU (gloo, world size 2): the problem split and
the max / sum combination that bench.py uses for N GPUs."""
import os
import socket

import pytest

from paper_2203_05665_gb300 import inputs as I
from paper_2203_05665_gb300 import shard


def test_shard_covers_every_problem_once():
    specs = I.batch_problems(64, 1004)
    for world in (1, 2, 3, 4, 8):
        parts = shard.shard_problems(specs, world)
        assert len(parts) == world
        idx = sorted(s["index"] for p in parts for s in p)
        assert idx == list(range(64))
        for p in parts:   # original order kept
            assert [s["index"] for s in p] == sorted(s["index"] for s in p)
        loads = [sum(shard.weight(s) for s in p) for p in parts]
        # LPT: no rank exceeds the mean by more than the largest single problem
        assert max(loads) - sum(loads) / world <= max(shard.weight(s) for s in specs)
    assert shard.shard_problems(specs, 4) == shard.shard_problems(list(specs), 4)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    specs = I.batch_problems(16, 1004)
    mine = shard.shard_problems(specs, world)[rank]
    units = sum(s["n"] * s["nrhs"] for s in mine)
    ms, total = shard.combine(10.0 + rank, units)
    out.put((rank, [s["index"] for s in mine], ms, total))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    specs = I.batch_problems(16, 1004)
    want = sum(s["n"] * s["nrhs"] for s in specs)
    (r0, i0, ms0, tot0), (r1, i1, ms1, tot1) = res
    assert sorted(i0 + i1) == list(range(16)) and not set(i0) & set(i1)
    assert ms0 == ms1 == 11.0            # max over ranks
    assert tot0 == tot1 == want          # sum over ranks
