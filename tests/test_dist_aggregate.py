"""The multi-rank path of bench.py on CPU: two gloo ranks, replicas with no data-path collective;
the job time is the slowest rank's, the work is the sum over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, vu = bench.aggregate_over_ranks(10.0 * (rank + 1), 1000 * (rank + 1), world, "cpu")
    q.put((rank, ms, vu))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_max_time_and_sum_work():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, ms, vu in res:
        assert ms == 20.0 and vu == 3000.0


def test_single_rank_is_identity():
    import bench
    assert bench.aggregate_over_ranks(5.0, 7, 1, "cpu") == (5.0, 7)
