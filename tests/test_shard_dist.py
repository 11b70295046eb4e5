"""CPU checks of the row-shard bookkeeping (no GPU): the chunk layout every
rank derives, and the exchange of chunks and the assembly of the whole state
through torch.distributed with world_size 2 and 3 on gloo -- the collective
the GPU path runs on NCCL."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_chunk_layout():
    import sys
    sys.path.insert(0, ROOT)
    from paper_2112_15079_gb300.shard import chunk_layout
    for n in (1, 2, 5, 31, 1000, 1001, 10425):
        for world in (1, 2, 3, 4, 8):
            c, ranges = chunk_layout(n, world)
            assert c % 2 == 0 and c * world >= n and c >= 2
            assert c < (n + world - 1) // world + 2  # no more padding than the pair rounding needs
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            for k, (b, e) in enumerate(ranges):  # contiguous, in rank order, each inside its chunk
                assert b == min(k * c, n) and e == min(b + c, n) and b <= e
                if k:
                    assert b == ranges[k - 1][1]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, n, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2112_15079_gb300.shard import chunk_layout, exchange_chunks, gather_rows
    c, ranges = chunk_layout(n, world)
    b, e = ranges[rank]
    cb = 32 * c
    # The source buffer: this rank's chunk current (its bodies' bytes tagged
    # with the body index), every other chunk stale.
    buf = torch.full((world * cb,), 255, dtype=torch.uint8)
    for p in range(b, e):
        buf[32 * (rank * c + (p - b)): 32 * (rank * c + (p - b) + 1)] = p % 251
    exchange_chunks(buf, rank, cb)
    # Every rank's state copy is stale outside its own bodies.
    local = torch.full((6, n), -1.0, dtype=torch.float64)
    local[:, b:e] = torch.arange(b, e, dtype=torch.float64) + torch.arange(6, dtype=torch.float64)[:, None] * 1e4
    whole = gather_rows(local, (b, e), rank, world, c)
    out[rank] = (buf.numpy().tobytes(), whole.numpy().tobytes())
    dist.destroy_process_group()


@pytest.mark.parametrize("world,n", [(2, 1001), (3, 10), (3, 2)])
def test_exchange_and_gather_gloo(world, n):
    import sys
    sys.path.insert(0, ROOT)
    from paper_2112_15079_gb300.shard import chunk_layout
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, n, out), nprocs=world, join=True, start_method="spawn")
    c, ranges = chunk_layout(n, world)
    want = np.full(world * 32 * c, 255, dtype=np.uint8)  # padding entries keep what their owner had
    for k, (b, e) in enumerate(ranges):
        for p in range(b, e):
            want[32 * (k * c + (p - b)): 32 * (k * c + (p - b) + 1)] = p % 251
    whole_want = np.arange(n, dtype=np.float64) + np.arange(6, dtype=np.float64)[:, None] * 1e4
    for r in range(world):
        buf, whole = out[r]
        assert np.array_equal(np.frombuffer(buf, dtype=np.uint8), want), r
        assert np.array_equal(np.frombuffer(whole, dtype=np.float64).reshape(6, n), whole_want), r
