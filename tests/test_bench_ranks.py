"""bench.py's multi-GPU form is replicas (one emulated GEMM per GPU, nothing
sharded): its host logic, run here as two gloo ranks on the CPU, must give every
rank the slowest rank's time and a whole-job value that sums the replicas' work;
the reference arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [12.5, 20.0][rank]
    got = bench.max_over_ranks(ms, torch.device("cpu"))
    q.put((rank, got, bench.job_tflops(world, 2.0 * 1024 ** 3, got)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [20.0, 20.0]
    expect = 2 * 2.0 * 1024 ** 3 / 20e-3 / 1e12
    assert all(abs(o[2] - expect) < 1e-12 * expect for o in out)


def test_single_process_keeps_local_time():
    sys.path.insert(0, ROOT)
    import bench
    import torch
    assert bench.max_over_ranks(7.25, torch.device("cpu")) == 7.25
    assert bench.job_tflops(1, 2e12, 1000.0) == pytest.approx(2.0)


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
