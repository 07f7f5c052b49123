"""The benchmark's N > 1 path on the CPU.

A run of the measured workload fits one GPU, so `bench.py --gpus N` runs N
independent replicas (no halo or particle exchange between them) and combines
their figures with two collectives only: the slowest
rank's timed region (MAX) and the particle-steps and end-to-end rates of all
ranks (SUM).  The same function (bench.job_totals) runs here on two gloo
ranks in spawned processes, with the rank layout read from the environment
the way torchrun sets it.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


MS = [10.0, 12.5]
PS = [1.0e9, 2.0e9]
E2E = [3.0e8, 5.0e8]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    r, w, local = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        out = bench.job_totals(MS[rank], PS[rank], E2E[rank], w, device="cpu")
        q.put((rank, (r, w, local), out))
    finally:
        dist.destroy_process_group()


def test_replica_totals_on_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(k, 2, port, q)) for k in range(2)]
    for p in procs:
        p.start()
    got = {}
    try:
        for _ in range(2):
            rank, env, out = q.get(timeout=180)
            got[rank] = (env, out)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert [p.exitcode for p in procs] == [0, 0]
    for k in range(2):
        env, (ms, ps, e2e) = got[k]
        assert env == (k, 2, k)
        assert ms == max(MS)                  # the job ends with its slowest replica
        assert ps == sum(PS) and e2e == sum(E2E)
    # whole-job throughput: every rank's units over the slowest rank's time
    assert got[0][1][1] / (got[0][1][0] * 1e-3) == pytest.approx(sum(PS) / (max(MS) * 1e-3))


def test_one_rank_passes_its_figures_through():
    import bench
    assert bench.job_totals(1.5, 2.0, 3.0, 1) == (1.5, 2.0, 3.0)
