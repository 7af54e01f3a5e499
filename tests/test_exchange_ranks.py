"""The exchange of a row-sharded call (binding.exchange_max), run as two gloo
ranks on the CPU: each of the three arrays (int32 column maxima, int64 per-k
maxima and rule maxima, the latter two the bits of nonnegative doubles) ends
as the element-wise maximum over the ranks on every rank, and for the bits of
nonnegative doubles that is the maximum of the values."""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _arrays(rank):
    rng = np.random.default_rng(rank)
    cmax = rng.integers(0, 1 << 29, 37).astype(np.int32)
    kmax = np.abs(rng.standard_normal(23)) * 2.0 ** rng.integers(-1000, 1000, 23)
    red = np.abs(rng.standard_normal(8)) * 1e3
    return cmax, kmax.view(np.int64), red.view(np.int64)


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2602_02549_b300 import binding as B
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        arrays = [torch.from_numpy(a.copy()) for a in _arrays(rank)]
        B.exchange_max(arrays)
        q.put((rank, [a.numpy().copy() for a in arrays]))
    finally:
        dist.barrier()
        dist.destroy_process_group()


def test_exchange_max_on_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    a0, a1 = _arrays(0), _arrays(1)
    for r in (0, 1):
        got = out[r]
        assert np.array_equal(got[0], np.maximum(a0[0], a1[0]))
        for i in (1, 2):
            assert np.array_equal(got[i], np.maximum(a0[i], a1[i]))
            vals = got[i].view(np.float64)
            assert np.array_equal(vals, np.maximum(a0[i].view(np.float64), a1[i].view(np.float64)))
