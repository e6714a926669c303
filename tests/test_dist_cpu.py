"""The N > 1 benchmark path on CPU with the gloo backend (world size 2):
envs shard by rank with no data-path collective; the job's time is the
slowest rank's (max over ranks), its rate counts every rank's env-steps;
the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import numpy as np
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [12.5, 20.0][rank]
    got = bench.max_over_ranks(local_ms, world)
    wl = bench.make_workload(rank)
    # a map fingerprint and sizes for the parent
    fp = int(np.asarray(wl.maps[0], np.int64).sum())
    # the reference arm: rank 1 returns at once without work
    ran = None
    if rank == 1:
        class A:
            steps, warmup = 1, 1
        ran = bench.run_reference(A())
    dist.barrier()
    out.put((rank, got, wl.n_envs, len(wl.maps), fp, ran))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_envs_and_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, e0, n0, f0, _), (r1, m1, e1, n1, f1, ran1) = res
    assert m0 == m1 == 20.0                   # both ranks see the slowest time
    assert (e0, n0) == (e1, n1) == (4096, 16)  # same shape on every rank
    assert f0 != f1                            # its own seeded maps per rank
    assert ran1 is None


def test_job_rate_counts_every_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_rate(2, 4096, 100, 0.5) == pytest.approx(2 * 4096 * 100 / 0.5)
    assert bench.max_over_ranks(3.5, 1) == 3.5
