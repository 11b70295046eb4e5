"""CPU checks of bench.py's multi-rank bookkeeping (world_size 2, gloo):
every rank times its own replica; the job's time is the max over ranks and
the value counts the units of all ranks.  No GPU and no data-path
collective are involved."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    r, w, lr = bench.dist_env()
    assert (r, w, lr) == (rank, world, rank)
    d = bench.dist_init(world, use_cuda=False)
    bench.barrier(d)
    elapsed = 1.0 + rank  # rank 1 is the slow one
    t = bench.max_over_ranks(elapsed, d)
    out[rank] = t
    d.destroy_process_group()


def test_max_over_ranks_gloo_world_size_2():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    assert out[0] == out[1] == 2.0


def test_single_rank_is_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.dist_init(1, use_cuda=False) is None
    assert bench.max_over_ranks(3.5, None) == 3.5
