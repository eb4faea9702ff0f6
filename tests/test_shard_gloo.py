"""Multi-rank host logic on CPU: two gloo ranks shard a batch of grids
without overlap or loss, balance the load, and reduce timings the way the
benchmark does (max over ranks, sum of work)."""
import os
import socket

import pytest

from paper_1503_01563_gb300 import inputs, shard

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dims = inputs.batch_dims(512, 4)
    mine = shard.shard(dims, rank, world)
    work = torch.tensor([sum(dims[g][0] * dims[g][1] for g in mine)], dtype=torch.float64)
    elapsed = torch.tensor([1.0 + rank], dtype=torch.float64)     # stand-in per-rank time
    ids = torch.zeros(512, dtype=torch.int64)
    ids[mine] = 1
    dist.all_reduce(ids)                                          # every grid exactly once
    total = work.clone()
    dist.all_reduce(total)
    dist.all_reduce(elapsed, op=dist.ReduceOp.MAX)
    loads = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(loads, work)
    q.put((rank, ids.tolist(), float(total), float(elapsed), [float(x) for x in loads]))
    dist.destroy_process_group()


def test_two_rank_batch_shard():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    dims = inputs.batch_dims(512, 4)
    n = sum(h * w for h, w in dims)
    for rank, ids, total, elapsed, loads in res:
        assert ids == [1] * 512
        assert total == n
        assert elapsed == 2.0
        assert max(loads) - min(loads) <= max(h * w for h, w in dims)   # LPT bound


def test_assignment_deterministic_and_balanced():
    dims = inputs.batch_dims(512, 4)
    sizes = [h * w for h, w in dims]
    for world in (1, 2, 3, 8):
        own = shard.assign(sizes, world)
        assert own == shard.assign(sizes, world)
        loads = [sum(s for s, r in zip(sizes, own) if r == k) for k in range(world)]
        assert max(loads) - min(loads) <= max(sizes)
        assert sorted(sum((shard.shard(dims, r, world) for r in range(world)), [])) == list(range(512))
