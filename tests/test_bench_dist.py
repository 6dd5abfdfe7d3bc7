"""The benchmark's multi-rank path on CPU: two gloo ranks on 127.0.0.1 run
independent replicas, and the whole-job rate uses the slowest rank's time
(units of all ranks / max time)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        local_ms = 100.0 * (rank + 1)          # rank 1 is the slow one
        rate = bench.job_rate(10, local_ms, world)
        mx = bench.allmax(float(rank), world)
        q.put((rank, rate, mx))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_whole_job_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, rate, mx in out:
        assert mx == 1.0
        assert rate == pytest.approx(2 * 10 / 0.2)      # 20 units in the slowest rank's 200 ms
