#!/usr/bin/env python
"""Throughput of the per-frame hashed-TSDF core on synthetic Kinect-shaped data.

One step = one 640x480 frame through the whole per-frame path: uint16
millimetre depth -> float metres, allocation (enumerate, commit, overflow,
visible list), integration, raycast to vertex and normal maps.  The frames
come from the seeded 300-frame room trajectory (5 mm voxels, mu = 20 mm,
2^20 buckets + 2^17 excess, 2^19 blocks); W warm-up frames are fused
untimed, then K frames are timed, each with CUDA events on the launching
stream, with the L2 flushed (a 256 MB write) between frames outside the
timed events.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank fuses its own independent trajectory (seed = rank):
no data-path collective; the barrier and the max over ranks use
torch.distributed.  --impl reference times the CPU oracle on the same
workload (rank 0 only).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_FRAMES = 300
WORKLOAD_NAME = "kinect room 640x480, 5 mm voxels, mu 20 mm, 2^20 buckets + 2^17 excess, 2^19 blocks, 300-frame trajectory"
METRIC = "frames/s (alloc+fuse+raycast, 640x480 @ 5 mm)"
L2_FLUSH_BYTES = 256 << 20


# ----------------------------------------------------------------- inputs

def _render(args):
    seed, k = args
    from synth import kinect_workload
    w = kinect_workload(seed=seed)
    f = w.frame(k)
    return k, f.depth_u16, f.T_wc


def render_frames(seed, indices, procs=None):
    """Frames of the seeded trajectory, rendered by a spawn pool (started
    before any CUDA call)."""
    procs = procs or min(len(indices), os.cpu_count() or 1, 32)
    out = {}
    if procs > 1 and len(indices) > 4:
        ctx = mp.get_context("spawn")
        with ctx.Pool(procs) as pool:
            for k, d, T in pool.imap_unordered(_render, [(seed, k) for k in indices], chunksize=4):
                out[k] = (d, T)
    else:
        for k in indices:
            _, d, T = _render((seed, k))
            out[k] = (d, T)
    return out


# ----------------------------------------------------------------- helpers

def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash():
    p = os.path.join(ROOT, "paper_1708_00783_gb300", "csrc", "itm_integrate.cu")
    with open(p, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def committed_traffic():
    """DRAM bytes per integration launch from the committed ncu summary, if it
    was taken from the current kernel source."""
    p = os.path.join(ROOT, "profiles", "integrate_kinect_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("source_sha256_16") != kernel_source_hash():
        return None
    return d.get("dram_bytes_per_launch_scaled")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return world, rank, local


def max_over_ranks(value, world, device=None):
    """Max of a scalar over ranks (identity at world size 1)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, world, device=None):
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ----------------------------------------------------------------- CPU oracle

def cpu_oracle_sample(frames, stride=30, budget_s=30.0):
    """The oracle as it stands, single-threaded, on every `stride`-th frame of
    the trajectory from an empty volume (alloc + integrate + raycast each),
    stopping once `budget_s` of work is done."""
    import oracle
    from synth import kinect_workload
    w = kinect_workload()
    sc = oracle.Scene(**w.params)
    ia = w.intr.as_array()
    done, t0, upd = 0, time.perf_counter(), 0
    idx = list(range(0, N_FRAMES, stride))
    for k in idx:
        raw, T = frames[k]
        d = oracle.depth_u16_to_f32(raw)
        sc.allocate(d, ia, T)
        upd += sc.integrate(d, ia, T)
        sc.raycast(w.intr.width, w.intr.height, ia, T)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "frames/s", "cores": 1, "kind": "oracle",
            "sample": "%d frames (every %dth of the 300-frame trajectory from frame 0, empty volume at start), "
                      "u16->f32 + allocate + integrate over all allocated blocks + raycast, single thread"
                      % (done, stride),
            "voxel_updates_per_s": upd / dt, "seconds": dt}


def run_reference(args, world, rank):
    """Reference arm: the CPU oracle timed on this arm's workload and metric."""
    if rank != 0:
        return
    frames = render_frames(0, list(range(0, N_FRAMES, 30)))
    import oracle
    from synth import kinect_workload
    w = kinect_workload()
    sc = oracle.Scene(**w.params)
    ia = w.intr.as_array()
    order = list(range(0, N_FRAMES, 30))
    budget = 120.0
    for i in range(min(args.warmup, 2)):
        raw, T = frames[order[i % len(order)]]
        d = oracle.depth_u16_to_f32(raw)
        sc.allocate(d, ia, T)
        sc.integrate(d, ia, T)
        sc.raycast(w.intr.width, w.intr.height, ia, T)
    times, upd = [], 0
    t_start = time.perf_counter()
    for i in range(args.steps):
        raw, T = frames[order[i % len(order)]]
        t0 = time.perf_counter()
        d = oracle.depth_u16_to_f32(raw)
        sc.allocate(d, ia, T)
        upd += sc.integrate(d, ia, T)
        sc.raycast(w.intr.width, w.intr.height, ia, T)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_start > budget:
            break
    total = sum(times)
    val = len(times) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "frames/s", "n_gpus": world,
        "steps": len(times), "warmup": min(args.warmup, 2), "ms_per_step": 1000 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME, "frames": "every 30th frame of the trajectory, repeated",
                   "requested_steps": args.steps, "time_budget_s": budget},
        "cpu_baseline": {"value": val, "unit": "frames/s", "cores": 1, "kind": "oracle",
                         "sample": "%d steps of one full 640x480 frame each (frames 0,30,...,270 cycled), "
                                   "single-threaded C oracle, stopped after a %.0f s budget" % (len(times), budget)},
        "e2e": {"value": val, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "voxel_updates_per_s": upd / total,
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- GPU arm

def run_ours(args, world, rank, local):
    # render before the first CUDA call (spawn pool)
    seed = rank
    total_frames = args.warmup + args.steps
    idx = sorted({k % N_FRAMES for k in range(total_frames)})
    frames = render_frames(seed, idx)
    cpu_frames = render_frames(0, list(range(0, N_FRAMES, 30))) if (rank == 0 and world == 1 and args.cpu_baseline) else None

    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_1708_00783_gb300 as itm
    from synth import kinect_workload

    w = kinect_workload(seed=seed)
    H, W = w.intr.height, w.intr.width
    ci = itm.make_intrinsics(W, H, w.intr.fx, w.intr.fy, w.intr.cx, w.intr.cy)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    raw_dev = {k: torch.from_numpy(frames[k][0].view(np.int16)).to(dev) for k in idx}
    poses = {k: frames[k][1] for k in idx}
    depth = torch.empty((H, W), dtype=torch.float32, device=dev)
    vtx = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
    nrm = torch.empty_like(vtx)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    scene = itm.Scene(**w.params)
    n_pix = H * W

    def step(k):
        itm.itm_depth_u16_to_f32(raw_dev[k], depth, n_pix, stream)
        itm.itm_allocate(scene.handle, depth, ci, poses[k], stream)
        itm.itm_integrate(scene.handle, depth, ci, poses[k], stream)
        itm.itm_raycast(scene.handle, ci, poses[k], vtx, nrm, stream)

    for i in range(args.warmup):
        step(i % N_FRAMES)
    torch.cuda.synchronize()
    st0 = scene.stats()

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            k = (args.warmup + i) % N_FRAMES
            e = ev[i]
            e[0].record(stream)
            itm.itm_depth_u16_to_f32(raw_dev[k], depth, n_pix, stream)
            e[1].record(stream)
            itm.itm_allocate(scene.handle, depth, ci, poses[k], stream)
            e[2].record(stream)
            itm.itm_integrate(scene.handle, depth, ci, poses[k], stream)
            e[3].record(stream)
            itm.itm_raycast(scene.handle, ci, poses[k], vtx, nrm, stream)
            e[4].record(stream)
            flush.zero_()
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    st1 = scene.stats()
    if st1["status"] != 0:
        raise RuntimeError("device status %#x during the timed region" % st1["status"])
    stage = np.array([[ev[i][j].elapsed_time(ev[i][j + 1]) for j in range(4)] for i in range(args.steps)])
    step_ms = stage.sum(axis=1)
    total_ms = float(step_ms.sum())
    total_ms_max = max_over_ranks(total_ms, world, dev)
    frames_all = args.steps * world
    fps = frames_all / (total_ms_max / 1000.0)
    updated = st1["updated_voxels"] - st0["updated_voxels"]
    visited = st1["visited_voxels"] - st0["visited_voxels"]
    updated_all = sum_over_ranks(float(updated), world, dev)

    # integration roofline: algorithmic bytes = 10 B per updated voxel (4 B sdf
    # + 1 B weight, read and written) + the depth frame + 12 B per visible
    # block (list entry + coordinates)
    integ_ms = float(stage[:, 2].sum())
    visible_blocks = visited / 512.0
    alg_bytes = 10.0 * updated + 4.0 * n_pix * args.steps + 12.0 * visible_blocks
    achieved = alg_bytes / (integ_ms / 1000.0) / 1e9
    peak, peak_kind = load_peaks()
    traffic = committed_traffic()

    # end to end through the public API with host buffers: pinned u16 frame
    # in, vertex + normal maps out, every step
    e2e = None
    if not args.no_e2e:
        scene.reset(stream)
        host_raw = {k: torch.from_numpy(frames[k][0].view(np.int16)).pin_memory() for k in idx}
        host_v = torch.empty((H, W, 4), dtype=torch.float32).pin_memory()
        host_n = torch.empty_like(host_v).pin_memory()
        raw_buf = torch.empty((H, W), dtype=torch.int16, device=dev)

        def e2e_step(k):
            raw_buf.copy_(host_raw[k], non_blocking=True)
            itm.itm_depth_u16_to_f32(raw_buf, depth, n_pix, stream)
            itm.itm_process_frame(scene.handle, depth, ci, poses[k], vtx, nrm, stream)
            host_v.copy_(vtx, non_blocking=True)
            host_n.copy_(nrm, non_blocking=True)

        for i in range(args.warmup):
            e2e_step(i % N_FRAMES)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for i in range(args.steps):
            e2e_step((args.warmup + i) % N_FRAMES)
        b.record(stream)
        torch.cuda.synchronize()
        e_ms = max_over_ranks(a.elapsed_time(b), world, dev)
        e2e = {"value": frames_all / (e_ms / 1000.0), "unit": "frames/s",
               "h2d_bytes_per_step": n_pix * 2, "d2h_bytes_per_step": 2 * n_pix * 16}

    cpu = None
    if cpu_frames is not None:
        cpu = cpu_oracle_sample(cpu_frames)
        cpu = {k: v for k, v in cpu.items() if k != "seconds"}

    if rank != 0:
        return
    clocks = clk.summary()
    line = {
        "metric": METRIC,
        "value": fps,
        "unit": "frames/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms_max / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {
            "workload": WORKLOAD_NAME,
            "frames": "warm-up frames 0..%d, timed frames %d..%d (mod 300)" % (args.warmup - 1, args.warmup,
                                                                              args.warmup + args.steps - 1),
            "input": "uint16 millimetre depth resident in HBM, converted on the device each step",
            "l2": "flushed between steps (256 MB write, outside the timed events)",
            "parallelism": "independent trajectory per rank" if world > 1 else "single GPU",
            "stage_ms_mean": {"depth_u16_to_f32": float(stage[:, 0].mean()), "allocate": float(stage[:, 1].mean()),
                              "integrate": float(stage[:, 2].mean()), "raycast": float(stage[:, 3].mean())},
            "allocated_blocks": st1["allocated_blocks"],
            "visible_blocks_mean": visible_blocks / args.steps,
            "updated_voxels_per_frame": updated / args.steps,
        },
        "voxel_updates_per_s": updated_all / (total_ms_max / 1000.0),
        "roofline": {
            "kernel": "integrate_kernel<0>",
            "bound": "hbm",
            "achieved": achieved,
            "peak": peak,
            "peak_kind": peak_kind,
            "unit": "GB/s",
            "frac": achieved / peak,
            "traffic": traffic,
            "algorithmic_bytes_per_launch": alg_bytes / args.steps,
            "launch_ms_mean": integ_ms / args.steps,
        },
        "cpu_baseline": cpu,
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": 8 * args.steps,  # u16, enumerate, commit, overflow, visible, integrate, range, raycast
    }
    print(json.dumps(line), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=290)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return 0
    run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
