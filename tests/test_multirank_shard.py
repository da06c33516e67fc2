"""The split-scene exchange and the batched deal with two gloo ranks on CPU.

Each rank fuses the tiny sequence into its part of the scene (the oracle's
slab partition: this host has no GPU), raycasts it, and the two ranks run
the library's exchange step (shard.exchange: an all-gather of the parts'
vertex and normal maps); each merges the gathered maps by the oracle's
merge rule.  Both ranks must end with the same maps, equal to the merge of
the parts computed in one process and within the parity bar of the whole
scene's raycast.  The deal of independent items by estimated size gives each
item to exactly one rank with balanced loads.
"""

import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist

    import oracle
    from paper_1708_00783_gb300 import shard
    from synth import tiny_workload
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = tiny_workload()
    part = oracle.Scene(**w.params)
    part.set_shard(world, rank, 4)
    ia = w.intr.as_array()
    for k in range(w.n_frames):
        f = w.frame(k)
        part.allocate(f.depth, ia, f.T_wc)
        part.integrate(f.depth, ia, f.T_wc)
    H, W = f.depth.shape
    v, n = part.raycast(W, H, ia, f.T_wc)
    vparts, nparts = shard.exchange(torch.from_numpy(v), torch.from_numpy(n))
    vm, nm = oracle.merge_raycasts(vparts.numpy(), nparts.numpy(), f.T_wc)
    deal = shard.deal_by_size([5, 1, 9, 3, 3, 7, 2], world)
    q.put((rank, vparts.numpy(), vm, nm, deal))
    dist.barrier()
    dist.destroy_process_group()


def test_split_scene_exchange_on_two_gloo_ranks():
    import torch.multiprocessing as mp

    import oracle
    from synth import tiny_workload
    from tests.parity_util import compare_raycast
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, vp0, vm0, nm0, deal0), (_, vp1, vm1, nm1, deal1) = out
    assert np.array_equal(vp0, vp1)                       # both ranks hold every part's map
    assert np.array_equal(vm0, vm1) and np.array_equal(nm0, nm1)
    # the same parts and merge in one process, and the whole scene
    w = tiny_workload()
    ia = w.intr.as_array()
    full = oracle.Scene(**w.params)
    parts = [oracle.Scene(**w.params) for _ in range(2)]
    for i, p in enumerate(parts):
        p.set_shard(2, i, 4)
    for k in range(w.n_frames):
        f = w.frame(k)
        for sc in [full] + parts:
            sc.allocate(f.depth, ia, f.T_wc)
            sc.integrate(f.depth, ia, f.T_wc)
    H, W = f.depth.shape
    maps = [p.raycast(W, H, ia, f.T_wc) for p in parts]
    assert np.array_equal(vp0, np.stack([m[0] for m in maps]))
    vm, nm = oracle.merge_raycasts(np.stack([m[0] for m in maps]), np.stack([m[1] for m in maps]), f.T_wc)
    assert np.array_equal(vm0, vm) and np.array_equal(nm0, nm)
    vf, nf = full.raycast(W, H, ia, f.T_wc)
    assert compare_raycast(vm0, nm0, vf, nf, f.T_wc)["pass_frac"] >= 0.999
    # the deal: each item once, loads balanced (sizes 9 7 5 3 3 2 1: 15 and 15)
    assert deal0 == deal1
    assert sorted(deal0[0] + deal0[1]) == list(range(7))
    sizes = [5, 1, 9, 3, 3, 7, 2]
    assert sorted(sum(sizes[i] for i in d) for d in deal0) == [15, 15]
