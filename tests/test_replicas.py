"""The N > 1 path of bench.py on CPU: two gloo ranks stand in for two GPUs.

The FMM itself is not sharded (each rank solves an independent problem), so
the only cross-rank logic is the whole-job throughput: all particles of all
ranks divided by the slowest rank's time.  A rank that is not rank 0 prints
nothing for the reference arm.
"""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [100.0, 150.0][rank]
    value, max_ms = bench.replica_throughput(1000, 4, local_ms)
    buf = io.StringIO()
    args = type("A", (), dict(steps=1, warmup=0, workload=bench.WORKLOAD))()
    if rank == 1:
        with redirect_stdout(buf):
            bench.run_reference(args)
    out.put((rank, value, max_ms, buf.getvalue()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replica_throughput_and_rank0_only_output():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, max_ms, printed in res:
        assert max_ms == 150.0
        assert value == pytest.approx(1000 * 2 * 4 / 0.150)
        if rank == 1:
            assert printed == ""


def test_single_process_throughput():
    sys.path.insert(0, ROOT)
    import bench
    value, max_ms = bench.replica_throughput(500, 10, 250.0)
    assert max_ms == 250.0 and value == pytest.approx(500 * 10 / 0.25)
