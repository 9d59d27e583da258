"""The N > 1 path of bench.py on CPU: two gloo ranks run independent problems, the
job's time is the slowest rank's, and the value counts every rank's units."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 * (rank + 1)                    # rank 1 is the slowest
    t, value = bench.reduce_over_ranks(local_ms, 1000, dist, "cpu")
    seeds = [None] * world
    dist.all_gather_object(seeds, bench.rank_seed(rank))
    out.put((rank, t, value, seeds))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, value, seeds in results:
        assert t == 200.0                            # max over ranks
        assert value == pytest.approx(2 * 1000 / 0.2)  # both ranks' units over the slowest time
        assert len(set(seeds)) == 2                  # independent problems per rank


def test_single_process_reduce():
    sys.path.insert(0, ROOT)
    import bench
    t, value = bench.reduce_over_ranks(50.0, 500, None)
    assert t == 50.0 and value == pytest.approx(10000.0)
