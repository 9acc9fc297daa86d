"""The multi-GPU path of bench.py is replicas only: each rank times its own batch and the job
reports the slowest rank.  Its cross-rank pieces run here as two gloo ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    dist.barrier()
    local = 1.5 if rank == 0 else 2.5          # seconds: rank 1 is slower
    m = bench.reduce_max(local, dist)
    thr = bench.job_throughput(65536, world, 3, m)
    q.put((rank, m, thr, bench.rank_seed(rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_report_slowest_and_aggregate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, t0, s0), (r1, m1, t1, s1) = res
    assert m0 == m1 == 2.5                      # max over ranks
    assert t0 == t1 == pytest.approx(65536 * 2 * 3 / 2.5)
    assert s0 == 1 and s1 != s0                 # rank 0 runs the workload's seed; others differ
