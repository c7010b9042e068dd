"""The multi-replica host logic of bench.py on CPU: two gloo ranks, barrier and max over ranks
(the path does not shard, so every rank runs its own replica and only the timing is reduced)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import bench
    got_ws, got_rank, got_local = bench.dist_env()
    assert (got_ws, got_rank, got_local) == (ws, rank, rank)
    bench.init_dist(ws, "gloo")
    bench.barrier(ws)
    vals = bench.reduce_max([10.0 * (rank + 1), 5.0 - rank, 1.5], ws)
    out[rank] = vals
    dist.destroy_process_group()


def test_two_rank_max_reduction():
    ws = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_worker, args=(ws, port, out), nprocs=ws, start_method="spawn")
        assert out[0] == out[1] == [20.0, 5.0, 1.5]


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_max([3.0, 4.0], 1) == [3.0, 4.0]
