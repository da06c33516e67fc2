"""The bench's multi-rank logic with two gloo ranks on CPU.

Under torchrun every rank fuses its own trajectory (seed = rank) with no
data-path collective; the only cross-rank steps are the barrier, the max of
the timed region and the sum of the update counts.  This runs those steps in
two processes and checks the whole-job numbers."""

import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, l = bench.dist_env()
    ms = [120.0, 150.0][rank]                     # rank 1 is the slower one
    mx = bench.max_over_ranks(ms, w)
    tot = bench.sum_over_ranks(1000.0 * (rank + 1), w)
    dist.barrier()
    from synth import kinect_workload
    pose0 = kinect_workload(seed=r).pose(0)
    q.put((rank, w, r, l, mx, tot, bench.job_throughput(100, w, mx), pose0[:3, 3].tolist()))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, w, r, l, mx, tot, fps, pos in out:
        assert (w, r, l) == (2, rank, rank)
        assert mx == 150.0 and tot == 3000.0
        assert fps == pytest.approx(200 / 0.150)
    assert out[0][7] != out[1][7]                # independent trajectories per rank
