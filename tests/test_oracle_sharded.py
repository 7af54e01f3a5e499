"""Row-sharded Ozaki-II on gloo CPU ranks (oracle/sharded.py): each rank holds a
block of rows of A and all of B; one all-reduce (MAX) of Cbar's column maxima
(with the bound rule's maxima in the same buffer) is the only exchange.  Every
rank's rows of C, mu and nu, and N, must equal the unsharded oracle's bit for
bit (Algorithm 2's nu_j takes max_h cbar_hj over all m rows).  A planted
mistake, the exchange left out, must break that."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (m, n, k, phi, N or 0 for the bound rule, target, world)
CASES = [(37, 23, 300, 1.0, 14, 0.0, 2), (37, 23, 300, 4.0, 0, 1e-15, 2), (50, 17, 129, 2.0, 0, 1e-12, 3),
         (2, 9, 64, 0.5, 9, 0.0, 3)]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, case, plant, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import sharded
        from paper_2602_02549_b300.inputs import paper_pair
        m, n, k, phi, N, tau, _ = case
        A, B = paper_pair(m, n, k, phi, seed=m + n)
        if case == CASES[0]:
            A[5, :] = 0.0                                  # an empty row on rank 0
        rows = np.array_split(np.arange(m), world)[rank]
        if plant:                                          # the exchange left out
            sharded.all_reduce_max = lambda buf, group=None: buf
        r = sharded.os_ii_rows(A[rows], B, N, 64, tau, 20)
        q.put((rank, rows, r["C"], r["mu"], r["nu"], r["N"]))
    finally:
        dist.barrier()
        dist.destroy_process_group()


def run_ranks(case, plant=False):
    world = case[-1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, case, plant, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return sorted(out, key=lambda o: o[0])


def reference(case):
    from oracle import ozaki2
    from paper_2602_02549_b300.inputs import paper_pair
    m, n, k, phi, N, tau, _ = case
    A, B = paper_pair(m, n, k, phi, seed=m + n)
    if case == CASES[0]:
        A[5, :] = 0.0
    if N == 0:
        s = ozaki2.scaling(A, B, 14)
        N, _ = ozaki2.choose_N(A, B, s["alpha"], s["beta"], s["cmax_row"], s["cmax_col"], tau, 20)
    return ozaki2.os_ii(A, B, N, 64), N


@pytest.mark.parametrize("case", CASES)
def test_sharded_rows_equal_unsharded(case):
    ref, N = reference(case)
    out = run_ranks(case)
    for rank, rows, C, mu, nu, Nr in out:
        assert Nr == N
        assert np.array_equal(nu, ref["nu"])
        assert np.array_equal(mu, ref["mu"][rows])
        assert np.array_equal(C.view(np.int64), ref["C"][rows].view(np.int64))


def test_planted_missing_exchange_is_caught():
    case = CASES[1]
    ref, N = reference(case)
    out = run_ranks(case, plant=True)
    same = all(np.array_equal(nu, ref["nu"]) and np.array_equal(C.view(np.int64), ref["C"][rows].view(np.int64))
               for _, rows, C, _, nu, _ in out)
    assert not same
