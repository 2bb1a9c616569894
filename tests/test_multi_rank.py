"""The N > 1 host logic of bench.py with two gloo ranks on the CPU: the
job's time is the slowest rank's, replicas get distinct seeds, and sharded
jobs are each run by exactly one rank with balanced load."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_0808_2109_gb300 import workloads
    t = bench.max_over_ranks(1.5 + rank)
    jobs = workloads.batch_manifest(n=64, sweeps=10)
    mine = bench.shard_jobs(jobs, rank, world)
    out.put((rank, t, [j.seed for j in mine], sum(j.L * j.L * j.sweeps for j in mine),
             workloads.LARGE.seed + rank))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(r[1] == 2.5 for r in res)                      # max over ranks
    seeds = res[0][2] + res[1][2]
    assert sorted(seeds) == sorted(set(seeds)) and len(seeds) == 64   # each job once
    loads = [r[3] for r in res]
    assert max(loads) <= 1.1 * min(loads) + 1024 * 1024 * 10   # within one largest job
    assert res[0][4] != res[1][4]                             # distinct replica seeds


def test_single_process_is_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    from paper_0808_2109_gb300 import workloads
    assert bench.max_over_ranks(3.25) == 3.25
    jobs = workloads.batch_manifest(n=10, sweeps=5)
    assert bench.shard_jobs(jobs, 0, 1) == sorted(jobs, key=lambda j: -j.L * j.L * j.sweeps)
