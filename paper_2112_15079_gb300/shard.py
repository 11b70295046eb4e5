"""Row shards of one system over several ranks (GPUs).

The distributed form of the method (Section 3: each process owns a block of
bodies, loops over all of them as sources, and the processes exchange the
new positions after every step).  Every rank holds the whole state.  Rank k
owns bodies [k C, (k + 1) C) (C = the chunk length, the last chunk padded);
each step it evaluates Eq. 1 for its own bodies against every source and
applies Eqs. 3-4 to them (``nbody_shard_step``), which stages their next
positions into its own chunk of the next step's source buffer; one
all-gather of those chunks then gives every rank all positions
(``nbody_shard_buffer``).  The collective carries 32 bytes per body per
step; no rank reads another's memory directly.

``ShardedNBody`` drives one rank.  Its ``exchange`` callback performs the
all-gather: by default ``allgather_exchange`` (torch.distributed, NCCL on
GPUs, in place, on the context's stream).  Only argument marshalling and the
collective live here; every step of the computation runs in the library.
"""
from __future__ import annotations

import ctypes

from . import nbody as _nb


def chunk_layout(n: int, world: int):
    """(C, [(begin, end) per rank]): the chunk length the library uses --
    ceil(n / world) rounded up to an even count (whole source pairs) -- and
    each rank's bodies.  Chunk k occupies source entries [k C, (k + 1) C);
    entries past n are inert padding."""
    c = ((n + world - 1) // world + 1) // 2 * 2
    return c, [(min(k * c, n), min(k * c + c, n)) for k in range(world)]


class _CudaBytes:
    """A device byte range presented through __cuda_array_interface__ (so
    torch can view it without a copy)."""

    def __init__(self, ptr: int, nbytes: int):
        self.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (ptr, False),
                                         "version": 3, "strides": None}


def exchange_chunks(buf, rank: int, chunk: int) -> None:
    """In place: chunk `rank` of the 1-D tensor `buf` (world chunks of
    `chunk` elements) from every rank into every rank's `buf`
    (torch.distributed all-gather; any backend, any device)."""
    import torch.distributed as dist

    dist.all_gather_into_tensor(buf, buf[rank * chunk:(rank + 1) * chunk])


def gather_rows(local, own, rank: int, world: int, chunk: int):
    """The whole [rows, n] array from every rank's own columns [own[0],
    own[1]) of its `local` copy (torch.distributed all-gather of padded
    chunks)."""
    torch = _nb._torch()
    import torch.distributed as dist

    rows, n = local.shape
    b, e = own
    mine = torch.zeros((world, rows, chunk), dtype=local.dtype, device=local.device)
    mine[rank, :, : e - b] = local[:, b:e]
    flat = mine.reshape(-1)
    exchange_chunks(flat, rank, rows * chunk)
    return mine.permute(1, 0, 2).reshape(rows, world * chunk)[:, :n]


def allgather_exchange(sh: "ShardedNBody") -> None:
    """Every rank's chunk of the next step's source buffer to every rank:
    one in-place all-gather on the context's stream."""
    torch = _nb._torch()
    with torch.cuda.stream(sh.body._stream):
        exchange_chunks(sh.stage_bytes(), sh.rank, sh.chunk_bytes)


class ShardedNBody:
    """One rank's row shard of a single system (velocity Verlet).

    r, v, m: the WHOLE system (every rank passes the same state).  The
    bound state of this rank advances for its own bodies only; ``own`` is
    their range, ``gather_state`` assembles the whole state from all ranks."""

    def __init__(self, r, v, m, *, G: float, dt: float, precision: str, rank: int, world: int,
                 exchange=None, device=None, stream=None):
        self.body = _nb.NBody(r, v, m, G=G, dt=dt, precision=precision, small=False, device=device, stream=stream)
        ctx = self.body._ctx
        _nb.check(_nb.nbody_shard(ctx, int(rank), int(world)), ctx)
        self.rank, self.world = int(rank), int(world)
        self.chunk, ranges = chunk_layout(self.body.n, self.world)
        self.own = ranges[self.rank]
        self.exchange = exchange if exchange is not None else allgather_exchange
        _, cb = self._buffer()
        if cb != 32 * self.chunk:
            raise RuntimeError(f"chunk layout mismatch: library {cb} bytes, expected {32 * self.chunk}")
        self.chunk_bytes = cb

    def _buffer(self):
        p = ctypes.c_void_p()
        cb = ctypes.c_int64()
        _nb.check(_nb.nbody_shard_buffer(self.body._ctx, ctypes.byref(p), ctypes.byref(cb)), self.body._ctx)
        return p.value, cb.value

    def stage_bytes(self):
        """The source buffer the next step reads, as a torch uint8 view
        (world chunks of chunk_bytes)."""
        torch = _nb._torch()
        p, cb = self._buffer()
        return torch.as_tensor(_CudaBytes(p, cb * self.world), device=self.body.device)

    def step_local(self) -> None:
        """One step of this rank's bodies, without the exchange."""
        _nb.check(_nb.nbody_shard_step(self.body._ctx), self.body._ctx)

    def step(self, n_steps: int = 1) -> None:
        for _ in range(int(n_steps)):
            self.step_local()
            self.exchange(self)

    def sync(self) -> None:
        self.body.sync()

    def gather_state(self):
        """The whole [6, N] state on every rank (torch.distributed
        all-gather of each rank's own bodies)."""
        torch = _nb._torch()
        with torch.cuda.stream(self.body._stream):
            return gather_rows(self.body.state, self.own, self.rank, self.world, self.chunk)

    def close(self) -> None:
        self.body.close()
