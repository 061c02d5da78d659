"""The benchmark's multi-rank logic (replicas only, no data-path collective)
with world_size-2 gloo process groups on the CPU: the slowest rank's time is
every rank's timing figure, the job throughput sums the ranks' work, and the
reference arm prints only on rank 0."""
import io
import os
import sys
from contextlib import redirect_stdout

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist)
        value = bench.job_throughput(world, 1000, 50, ms)
        out = io.StringIO()

        class A:
            gpus, steps, warmup = world, 1, 3
        if rank != 0:
            with redirect_stdout(out):
                bench.run_reference(A())
        q.put((rank, ms, value, out.getvalue()))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=100) for _ in procs)
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]
    assert all(abs(r[2] - 2 * 1000 * 50 / 15e-3) < 1e-6 for r in res)
    assert res[1][3] == ""  # rank 1 of the reference arm prints nothing
