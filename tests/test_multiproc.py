"""Multi-rank host logic on CPU (gloo, world size 2): each rank serves its own
shard of the request stream and the bench's max-over-ranks timing; no data
passes between ranks except the final statistics."""
import os
import socket

import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import torch
    from paper_2606_02711_gb300.serve import shard
    reqs = list(range(23))
    mine = shard(reqs, rank, world)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    t = torch.tensor([1.5 + rank])  # per-rank elapsed time
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    cells = torch.tensor([float(len(mine))])
    dist.all_reduce(cells, op=dist.ReduceOp.SUM)
    if rank == 0:
        out.put((gathered, float(t.item()), float(cells.item())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered, tmax, total = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    flat = sorted(x for g in gathered for x in g)
    assert flat == list(range(23))
    assert tmax == 2.5 and total == 23.0
