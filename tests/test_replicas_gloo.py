"""Multi-replica bookkeeping of bench.py on CPU (gloo, world size 2).

The solves do not shard across GPUs: every rank runs an independent replica,
and the only cross-rank traffic is a barrier and the max of the elapsed
times.  This runs that path with two CPU processes.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    reps = bench.Replicas("gloo")
    reps.barrier()
    ms, value = reps.throughput(100.0 * (rank + 1), 6, "cpu")
    reps.barrier()
    out.put((rank, reps.world, ms, value))
    reps.close()


def test_two_replicas_max_time_and_aggregate_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, world, ms, value in res:
        assert world == 2
        assert ms == 200.0                       # max over ranks
        assert abs(value - 2 * 6 / 0.2) < 1e-9   # all ranks' solves / max elapsed
