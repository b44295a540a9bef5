"""The multi-rank logic of bench.py on CPU: two gloo ranks each time their
own share of the work; the job's time is the slowest rank's and its value
counts every rank's solves (weak scaling, no collective on the data path)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = [1000.0, 1500.0][rank]          # rank 1 is the slower one
    ms, value = bench.aggregate(ms_local, 320, dist)
    q.put((rank, ms, value, bench.rank_seed(0, rank)))
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value, seed in out:
        assert ms == 1500.0                      # max over ranks
        assert value == pytest.approx(640 / 1.5)  # all ranks' solves / slowest time
    assert out[0][3] != out[1][3]                # distinct seeded problems per rank


def test_single_process_aggregate():
    import bench
    ms, value = bench.aggregate(2000.0, 320, None)
    assert ms == 2000.0 and value == pytest.approx(160.0)
