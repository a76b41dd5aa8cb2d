"""The multi-rank host logic of bench.py on CPU: world-size-2 gloo ranks.

Frames are independent work units (replicas, weak scaling): every rank draws
its own frame seed, the ranks exchange nothing on the data path, and the
timing takes the maximum over ranks while the units are summed."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, lr = bench.rank_env()
    seed = bench.rank_seed(1000, r)
    t = 1.5 + r  # rank r "took" 1.5 + r seconds
    mx = bench.reduce_max(t)
    total = bench.reduce_sum(10 * (r + 1))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, (r, w, lr), seed, mx, total))


@pytest.mark.parametrize("world", [2])
def test_rank_seeds_and_reductions(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    seeds = [o[2] for o in out]
    assert len(set(seeds)) == world  # independent frames per rank
    assert all(o[1] == (o[0], world, o[0]) for o in out)
    assert all(o[3] == 1.5 + (world - 1) for o in out)  # max over ranks
    assert all(o[4] == sum(10 * (r + 1) for r in range(world)) for o in out)


def test_single_rank_reductions_are_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(2.5) == 2.5
    assert bench.reduce_sum(3.0) == 3.0
    assert bench.rank_seed(7, 0) == 7
