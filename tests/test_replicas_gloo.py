"""The multi-GPU path is replicas only (every rank solves its own lattice, no
data-path collective).  What ranks share is the job timing: the barrier, the
slowest rank's time, and the whole-job throughput.  This runs that logic with
two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r pretends its 5 steps took 100 (r+1) ms and moved 2^30 (r+1) bytes per step
    gbs, ms = bench.job_throughput(float(2 ** 30 * (rank + 1)), 100.0 * (rank + 1), 5, dist, "cpu")
    dist.barrier()
    q.put((rank, gbs, ms))
    dist.destroy_process_group()


def test_replica_throughput_two_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # slowest rank: 200 ms for 5 steps -> 40 ms per step; bytes summed over ranks
    want_ms = 200.0 / 5
    want_gbs = (2 ** 30 * 3) / (want_ms * 1e-3) / 1e9
    for rank, gbs, ms in out:
        assert ms == pytest.approx(want_ms)
        assert gbs == pytest.approx(want_gbs)


def test_single_rank_throughput():
    import bench
    gbs, ms = bench.job_throughput(2.0e9, 50.0, 10)
    assert ms == pytest.approx(5.0)
    assert gbs == pytest.approx(2.0e9 / 5e-3 / 1e9)
