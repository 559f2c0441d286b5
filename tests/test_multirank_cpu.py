"""The multi-rank path of the benchmark on CPU: two gloo ranks.

With N GPUs the benchmark runs one independent replica per rank (its own
seed, no data-path collective); a barrier brackets the timed region and the
job's throughput is all ranks' particle-steps over the slowest rank's time.
Here two processes on the host exercise that logic with the gloo backend.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    from paper_1707_04232_gb300.inputs import lattice_state

    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.set_process_group(dist)

    class Args:
        n, K = 10, 50.0

    w = bench.replica_workload(Args, rank)
    q, _, _ = lattice_state(w)
    bench.barrier(world)
    ms_local = 100.0 + 50.0 * rank  # rank 1 is the slower one
    value, ms_max = bench.aggregate(w.N, 20, ms_local, world)
    bench.barrier(world)
    out.put((rank, w.N, float(q[0, 0]), value, ms_max, bench.allreduce_max(float(rank), world)))
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_replicas():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, n0, x0, v0, m0, mx0), (r1, n1, x1, v1, m1, mx1) = res
    assert n0 == n1 == 1000
    assert x0 != x1  # independent replicas: own seeds
    assert m0 == m1 == 150.0  # the slowest rank's time, on every rank
    assert v0 == v1 == pytest.approx(1000 * 20 * 2 / 0.150)
    assert mx0 == mx1 == 1.0

