#!/usr/bin/env python3
"""Benchmark of the occupancy-grid ray sampler on one GB300 (or N, as
independent replicas of the per-frame work).

One step = one frame of the unbounded workload, the largest single-GPU frame
(a cascade of four 128^3 levels, level l over [-2^l, 2^l)^3, 1245x825 rays
from one of 20 seeded cameras inside the inner box, near 0.02, far 1e3, step
1.73e-3, cone 0.004): rebuild the VDB grid from the dense occupancy,
hierarchical-DDA sampling (count, scan, emit), and compositing over the
64-blob field.  Rays of all 20 cameras stay resident in HBM; the L2 is
flushed between timed steps (the flush is outside the timed windows).

Prints one JSON line (rank 0).  `value` is rays/s of the whole step; the
line also carries the sampler alone for HDDA and for the dense-DDA
baseline (rays/s, samples/s), per-kernel times, the roofline of the
dominant kernel and of the sampler, the end-to-end rate through the public
API with host buffers, and the CPU oracle's rate on a bounded sample of the
same work.  A default single-GPU run adds three summaries: the
object-centric frame (one 128^3 level, 800x800 rays) under `object`, the
batched sampler under `batch`, and the server's p50/p99 latency at a fixed
offered load under `serve`.

--impl reference times the CPU oracle (binary32 brute-force sampler plus
binary64 compositor) on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import gc
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_CAMERAS = 20
L2_FLUSH_BYTES = 256 << 20
# FP32 operations per evaluated blob in the compositor: 3 sub, 1 mul + 2 fma (squared
# distance), 1 fma (scaled exponent plus log2 amplitude), 1 add (density), 3 fma (colour);
# the exp2 runs on the MUFU pipe alongside.  The compositor evaluates two samples per
# lane with paired (f32x2) instructions, so this is 5.5 instructions per evaluation.  It
# skips blobs beyond 7 s of a chunk's points by definition; the library counts the
# evaluations it does make when its work counters are on ("composite_blob_evals"), which
# the bench does in a separate untimed pass.
COMPOSITE_FP32_PER_BLOB = 11
KERNELS_PER_TIMER = {"build_vdb": 5}   # the builder's timer spans five kernels
# L2 hit rate and warp execution efficiency (active lanes per warp instruction) per kernel
# from the ncu --set full captures (object frame, camera 0; unbounded: its first 200 image
# rows); dropped like the traffic when a kernel changes.
PROFILED_COUNTERS = {
    "object": {"hdda_walk": {"l2_hit_pct": 53.8, "active_lanes_of_32": 26.06},
               "hdda_emit": {"l2_hit_pct": 10.7, "active_lanes_of_32": 27.16},
               "composite": {"l2_hit_pct": 26.4, "active_lanes_of_32": 30.03}},
    "unbounded": {"hdda_walk": {"l2_hit_pct": 56.7, "active_lanes_of_32": 26.01},
                  "hdda_emit": {"l2_hit_pct": 10.0, "active_lanes_of_32": 30.15},
                  "composite": {"l2_hit_pct": 16.6, "active_lanes_of_32": 30.46}},
}
# DRAM bytes (read + write) per launch from ncu of a workload's step on camera 0 (the
# capture commands are kept with the profile summaries), for the roofline's "traffic"; an
# entry must be dropped whenever its kernel changes, and a workload without a capture
# reports none.
PROFILED_TRAFFIC = {
    "object": {"composite": 233_599_744, "hdda_emit": 266_574_592, "hdda_walk": 16_295_424},
    "unbounded": {"composite": 1_502_165_760, "hdda_emit": 2_182_214_144,
                  "hdda_walk": 27_365_888},
}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline workload only: no object-centric, batch or serve summaries")
    ap.add_argument("--cpu-stride", type=int, default=None,
                    help="CPU baseline sample: every n-th ray of camera 0 (default per workload)")
    ap.add_argument("--workload", choices=["object", "unbounded", "tiny", "batch", "serve"],
                    default="unbounded",
                    help="unbounded / object / tiny: the per-frame step on that scene (unbounded, "
                         "the largest single-GPU frame, is the default line and carries the "
                         "object-centric, batch and serve summaries); batch: 64 mixed jobs in one "
                         "graph launch against 64 separate launches; serve: continuous-batching "
                         "render server under Poisson load")
    ap.add_argument("--sampler-form", choices=["separate", "fused"], default="separate",
                    help="with --profile-step: the two-pass samplers' form")
    ap.add_argument("--profile-step", choices=["hdda", "dense", "render"], default=None,
                    help="profiling aid: one count-only call, one warm-up step and one step of "
                         "the given path on camera 0, no timing, no JSON line")
    ap.add_argument("--profile-rays", type=int, default=0,
                    help="with --profile-step: only the first N rays of camera 0 (whole image "
                         "rows from the top), a smaller case for multi-pass ncu captures")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def frame_workload(name: str):
    """(scene, 20 cameras, description, default CPU-baseline stride) of a per-frame workload."""
    from paper_2404_10272_gb300 import scenes
    if name == "unbounded":
        sc = scenes.unbounded_scene()
        cams = [scenes.unbounded_camera(j=j) for j in range(N_CAMERAS)]
        desc = ("unbounded: 4x128^3 cascade, level l over [-2^l,2^l)^3, 1245x825 rays from "
                "inside the inner box, 20 cameras, near 0.02, far 1e3, step 1.73e-3, cone 0.004, "
                "64-blob composite")
        return sc, cams, desc, 64
    if name == "tiny":
        sc = scenes.tiny_scene()
        cams = [scenes.tiny_camera(seed=1001 + 7 * j) for j in range(N_CAMERAS)]
        desc = ("tiny: 1x64^3 grid over [-1.5,1.5)^3, 96x96 rays, 20 cameras on a radius-4 "
                "sphere, near 2, far 6, step 5e-3, 64-blob composite")
        return sc, cams, desc, 1
    sc = scenes.object_scene()
    cams = scenes.object_cameras(n=N_CAMERAS)
    desc = ("object-centric: 1x128^3 grid over [-1.5,1.5)^3, 800x800 rays, 20 cameras on a "
            "radius-4 sphere, near 2, far 6, step 0.0050743674, 64-blob composite")
    return sc, cams, desc, 16


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args):
    """The headline line: the per-frame step on the chosen workload (the unbounded one by
    default), with the object-centric frame, the batched sampler and the server's latency
    summarised beside it on a default single-GPU run."""
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        # replicas only: no data path crosses GPUs; a host (gloo) group carries just the
        # barrier around the timed loops and the MAX of the ranks' elapsed times
        dist.init_process_group("gloo")
    import __graft_entry__
    __graft_entry__.build()
    line = measure_frame(args, args.workload, full=True)
    if world == 1 and not args.no_extras and args.workload == "unbounded":
        obj = measure_frame(args, "object", full=False)
        line["object"] = object_summary(obj)
        line["batch"] = run_batch(args, quick=True)
        line["serve"] = run_serve(args, quick=True)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def object_summary(d: dict) -> dict:
    """The object-centric frame's figures for the headline line's `object` key."""
    keep = ("ms_per_step", "value", "samples_per_step", "hdda_sampler", "dense_dda_sampler",
            "hdda_vs_dense_sampler_speedup", "roofline", "roofline_sampler", "render_only_step",
            "dense_dda_step", "grid", "candidates_per_ray", "fused_sampler_form", "ray_order")
    out = {"workload": d["config"]["workload"], "rays_per_step": d["config"]["rays_per_step"],
           "steps": d["steps"], "rays_per_s": d["value"]}
    out.update({k: d[k] for k in keep if k in d and k != "value"})
    out["kernels"] = {k: v["avg_ms"] for k, v in d["kernels"].items()}
    out["render_only_step"] = {k: v for k, v in d["render_only_step"].items()
                               if k in ("rays_per_s", "ms_per_step", "vs_step")}
    return out


def measure_frame(args, workload: str, full: bool = True) -> dict:
    """All figures of one per-frame workload.  full=False keeps the step, both samplers,
    the dense-DDA and render-only steps and the rooflines (a summary block); full=True adds
    the remaining variants, the incremental rebuild, the end-to-end loop and the CPU
    baselines."""
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2404_10272_gb300 import hdda, replicas, scenes

    rank, world, local = dist_env()
    sc, cams, desc, stride = frame_workload(workload)
    rays = [c.rays() for c in cams]
    n = rays[0][0].shape[0]
    O = torch.stack([torch.from_numpy(o) for o, _ in rays]).cuda()
    D = torch.stack([torch.from_numpy(d) for _, d in rays]).cuda()
    dense = torch.from_numpy(sc.occ).cuda()
    field = torch.from_numpy(sc.field).cuda()
    p = sc.params
    # the rays are each camera's pixels row by row: the calls pass the image width, so that
    # the walk takes them in 8 x 4 pixel blocks (same outputs); `ray_order` below times the
    # walk in index order beside it
    img_w = cams[0].width
    prm = hdda.make_params(p.near, p.far, p.step, p.cone, p.max_step, p.max_steps,
                           image_width=img_w)
    prm_index = hdda.make_params(p.near, p.far, p.step, p.cone, p.max_step, p.max_steps)
    gv = hdda.build_vdb(dense, sc.aabbs)
    gd = hdda.pack_dense(dense, sc.aabbs)
    gvp = hdda.build_vdb(dense, sc.aabbs)   # the plain VDB tree, without refinement masks
    gvp.set_refine(False)
    gvs = hdda.build_vdb(dense, sc.aabbs)   # Algorithm 2's control flow ("skip")
    gvs.set_walk(hdda.WALK_SKIP)
    gds = hdda.pack_dense(dense, sc.aabbs)
    gds.set_walk(hdda.WALK_SKIP)
    vstats = gv.stats()
    plain_bytes = int(gvp.stats().bytes)

    totals = [hdda.traverse_hdda(O[c], D[c], gv, prm, count_only=True).total
              for c in range(N_CAMERAS)]
    cap = max(totals)
    bufs = hdda.alloc_samples(n, cap)
    rgba = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def cam_of(j):
        return replicas.camera_for(rank, j, N_CAMERAS)

    tstatus = torch.zeros(1, dtype=torch.int32, device="cuda")

    def step_hdda(j):
        """The step: rebuild, stream-ordered sampling, compositing; no host round trip
        (the per-camera totals were counted above)."""
        c = cam_of(j)
        gv.rebuild(dense)
        hdda.traverse_async(O[c], D[c], gv, prm, bufs, tstatus)
        hdda.composite(O[c], D[c], bufs, field, out=rgba)
        return totals[c]

    def step_hdda_sync(j):
        """The same step through the synchronous sampler (host reads the total)."""
        c = cam_of(j)
        gv.rebuild(dense)
        s = hdda.traverse_hdda(O[c], D[c], gv, prm, out=bufs)
        hdda.composite(O[c], D[c], s, field, out=rgba)
        return s.total

    def step_dense(j):
        c = cam_of(j)
        gd.rebuild(dense)
        s = hdda.traverse_dense(O[c], D[c], gd, prm, out=bufs)
        hdda.composite(O[c], D[c], s, field, out=rgba)
        return s.total

    def sampler_hdda(j):
        c = cam_of(j)
        return hdda.traverse_hdda(O[c], D[c], gv, prm, out=bufs).total

    def sampler_hdda_plain(j):
        c = cam_of(j)
        return hdda.traverse_hdda(O[c], D[c], gvp, prm, out=bufs).total

    def sampler_hdda_skip(j):
        c = cam_of(j)
        return hdda.traverse_hdda(O[c], D[c], gvs, prm, out=bufs).total

    def sampler_dense_skip(j):
        c = cam_of(j)
        return hdda.traverse_dense(O[c], D[c], gds, prm, out=bufs).total

    def sampler_dense(j):
        c = cam_of(j)
        return hdda.traverse_dense(O[c], D[c], gd, prm, out=bufs).total

    def timed(fn, steps, warmup, profile=False, clocks=None):
        for j in range(warmup):
            fn(j)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
        if profile:
            hdda.profiler_read()
            hdda.profiler_enable(True)
        evs = []
        samples = 0
        for j in range(steps):
            flush.zero_()   # evict the previous step's data from L2 (outside the window)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            samples += fn(warmup + j)
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        kern = {}
        if profile:
            hdda.profiler_enable(False)
            kern = hdda.profiler_read()
        clk = clocks.stop() if clocks else None
        ms = replicas.max_over_ranks(sum(a.elapsed_time(b) for a, b in evs))
        return ms, samples, kern, clk

    status = torch.zeros(1, dtype=torch.int32, device="cuda")

    def render_step(j):
        c = cam_of(j)
        gv.rebuild(dense)
        hdda.render(O[c], D[c], gv, prm, field, out=rgba, status=status)
        return 0

    def fused_step(j):
        """The step's outputs (samples and frame) from hdda_traverse_composite: walk,
        scan, then one kernel that stores each sample and composites it."""
        c = cam_of(j)
        gv.rebuild(dense)
        hdda.traverse_composite(O[c], D[c], gv, prm, bufs, field, tstatus, rgba=rgba)
        return totals[c]

    K, W = args.steps, args.warmup
    # clocks are sampled over every timed loop below (the headline loop alone is
    # shorter than a few sampling periods)
    clocks = ClockSampler(local)
    clocks.start()
    # the headline loop runs without the library's per-kernel events; the per-kernel
    # breakdown comes from a second, profiled pass over the same steps
    ms, samples, _, _ = timed(step_hdda, K, W)
    ms_prof, _, kern, _ = timed(step_hdda, K, 2, profile=True)
    # the comparison loops run as many steps as the headline loop, so that they cover the
    # same cameras (with K = 20, each camera once): the unbounded cameras differ in cost
    K2 = K
    ms_dense, samples_dense, kern_dense, _ = timed(step_dense, K2, 2, profile=True)
    ms_sh, samp_sh, _, _ = timed(sampler_hdda, K, 2)
    ms_sd, samp_sd, _, _ = timed(sampler_dense, K2, 2)
    ms_r, _, kern_r, _ = timed(render_step, K, 2, profile=True)
    # the same step and sampler with the walk and the emit fused into one kernel
    hdda.set_sampler_form(hdda.SAMPLER_FUSED)
    try:
        # K steps: every camera once, as in the loops it is compared with
        ms_fu, _, kern_fu, _ = timed(step_hdda, K, 2, profile=True)
        ms_fu_s, _, _, _ = timed(sampler_hdda, K, 2)
    finally:
        hdda.set_sampler_form(hdda.SAMPLER_SEPARATE)
    # the same step and samplers with the rays walked in index order (no image width):
    # the closures above read `prm` when they run
    prm_blocks, prm = prm, prm_index
    try:
        ms_io, _, kern_io, _ = timed(step_hdda, K, 2, profile=True)
        ms_io_s, _, _, _ = timed(sampler_hdda, K, 2)
        ms_io_d, _, _, _ = timed(sampler_dense, K2, 2)
    finally:
        prm = prm_blocks
    ms_sync = ms_sp = ms_ss = ms_ds = ms_f = None
    kern_f = {}
    if full:
        ms_sync, _, _, _ = timed(step_hdda_sync, K2, 2)
        ms_sp, samp_sp, _, _ = timed(sampler_hdda_plain, K2, 2)
        ms_ss, _, _, _ = timed(sampler_hdda_skip, K2, 2)
        ms_ds, _, _, _ = timed(sampler_dense_skip, K2, 2)
        ms_f, _, kern_f, _ = timed(fused_step, K, 2, profile=True)

    # incremental rebuild: 1 % of the 8^3 blocks change (one voxel each, in partial
    # blocks, so the leaves are rewritten in place) and again 1 % with a new leaf each
    # (empty blocks gain a voxel: the structure is rebuilt), against the full rebuild
    def update_bench(occ, aabbs):
        L, R = occ.shape[0], occ.shape[1]
        B = (R + 7) // 8
        blk = occ[:, : B * 8, : B * 8, : B * 8].reshape(L, B, 8, B, 8, B, 8)
        cnt = blk.sum(axis=(2, 4, 6)).reshape(-1)
        rng = np.random.default_rng(77)
        n_pick = max(1, (L * B ** 3) // 100)
        out = {"blocks": int(L * B ** 3), "listed": n_pick}
        for kind, cand in (("in_place", np.flatnonzero((cnt > 1) & (cnt < 511))),
                           ("structural", np.flatnonzero(cnt == 0))):
            pick = np.sort(rng.choice(cand, size=min(n_pick, cand.size), replace=False))
            alt = occ.copy()
            for b in pick:
                l, r = divmod(int(b), B ** 3)
                bx, r = divmod(r, B * B)
                by, bz = divmod(r, B)
                v = alt[l, 8 * bx:8 * bx + 8, 8 * by:8 * by + 8, 8 * bz:8 * bz + 8]
                v[0, 0, 0] ^= 1
            dense_alt = torch.from_numpy(alt).cuda()
            dense_cur = torch.from_numpy(occ).cuda()
            lst = torch.from_numpy(pick.astype(np.int64)).cuda()
            gu = hdda.build_vdb(dense_cur, aabbs)
            ust = torch.zeros(1, dtype=torch.int32, device="cuda")
            srcs = (dense_alt, dense_cur)
            for j in range(4):
                gu.update(srcs[j % 2], lst, status=ust)
            torch.cuda.synchronize()
            reps = 50
            a, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for j in range(reps):
                gu.update(srcs[j % 2], lst, status=ust)
            b2.record()
            b2.synchronize()
            out[kind + "_ms"] = round(a.elapsed_time(b2) / reps, 4)
            if int(ust.item()) != 0:
                raise RuntimeError("grid update raised a device status")
            a.record()
            for j in range(reps):
                gu.rebuild(srcs[j % 2])
            b2.record()
            b2.synchronize()
            out["full_rebuild_ms"] = round(a.elapsed_time(b2) / reps, 4)
            gu.free()
            del dense_alt, dense_cur
        return out

    if int(tstatus.item()) != 0:
        raise RuntimeError(f"hdda_traverse_async raised device status {int(tstatus.item())}")
    upd = None
    if full:
        upd = {"this_grid": update_bench(sc.occ, sc.aabbs)}
        # a large cascade (2 x 512^3, 256 MiB of voxels): the update reads only the listed
        # blocks
        big_rng = np.random.default_rng(78)
        big = np.zeros((2, 512, 512, 512), np.uint8)
        big.reshape(-1)[big_rng.integers(0, big.size, size=big.size // 500)] = 1
        for l in range(2):
            for _ in range(40):
                a0 = big_rng.integers(0, 448, size=3)
                b0 = a0 + big_rng.integers(8, 64, size=3)
                big[l, a0[0]:b0[0], a0[1]:b0[1], a0[2]:b0[2]] = 1
        upd["2x512_grid"] = update_bench(big, scenes.cascade_boxes(2, 1.0))
        del big
    clk = clocks.stop()
    if int(status.item()) != 0:
        raise RuntimeError(f"hdda_render raised device status {int(status.item())}")

    def count_evals(fn, reps=3):
        """Blob evaluations per step, counted outside the timed loops (the
        counters are extra device work)."""
        torch.cuda.synchronize()
        hdda.profiler_read()
        hdda.profiler_enable(False, counters=True)
        for j in range(reps):
            fn(j)
        hdda.profiler_enable(False)
        got = hdda.profiler_read()
        return {k: v[0] / reps for k, v in got.items() if k.endswith("_blob_evals")}

    evals_step = count_evals(step_hdda).get("composite_blob_evals", 0.0)
    render_evals = count_evals(render_step).get("render_blob_evals", 0.0)

    value = replicas.aggregate_rate(n * K, ms, world)

    # --- end to end through the public API with host buffers ---------------
    # Every step uploads its rays from pinned host memory and reads its frame
    # back.  As a streaming renderer would, the uploads run on one copy stream
    # and the read-backs on another, two slots deep, so that step j+1's rays
    # travel while step j computes and step j's frame returns while step j+1
    # computes; events keep each slot's buffers from being reused early.
    e2e = None
    if full:
        o_host = [torch.from_numpy(o).pin_memory() for o, _ in rays]
        d_host = [torch.from_numpy(d).pin_memory() for _, d in rays]
        out_host = [torch.empty((n, 4), dtype=torch.float32).pin_memory() for _ in range(2)]
        o_dev = [torch.empty_like(O[0]) for _ in range(2)]
        d_dev = [torch.empty_like(D[0]) for _ in range(2)]
        frame = [torch.empty_like(rgba) for _ in range(2)]
        main = torch.cuda.current_stream()
        h2d, d2h = torch.cuda.Stream(), torch.cuda.Stream()
        ev_in = [torch.cuda.Event() for _ in range(2)]    # slot's rays uploaded
        ev_used = [torch.cuda.Event() for _ in range(2)]  # slot's step computed
        ev_out = [torch.cuda.Event() for _ in range(2)]   # slot's frame read back
        steps_e2e = K  # the same camera mix as the timed steps

        def upload(j):
            sl, c = j % 2, cam_of(j)
            h2d.wait_event(ev_used[sl])  # step j-2 is done with this slot's rays
            with torch.cuda.stream(h2d):
                o_dev[sl].copy_(o_host[c], non_blocking=True)
                d_dev[sl].copy_(d_host[c], non_blocking=True)
            ev_in[sl].record(h2d)

        def compute(j):
            sl = j % 2
            main.wait_event(ev_in[sl])
            main.wait_event(ev_out[sl])  # step j-2's frame has left this slot
            gv.rebuild(dense)
            hdda.traverse_async(o_dev[sl], d_dev[sl], gv, prm, bufs, tstatus)
            hdda.composite(o_dev[sl], d_dev[sl], bufs, field, out=frame[sl])
            ev_used[sl].record(main)
            d2h.wait_event(ev_used[sl])
            with torch.cuda.stream(d2h):
                out_host[sl].copy_(frame[sl], non_blocking=True)
            ev_out[sl].record(d2h)

        def run_e2e(steps):
            upload(0)
            for j in range(steps):
                if j + 1 < steps:
                    upload(j + 1)
                compute(j)
            torch.cuda.synchronize()

        run_e2e(3)
        t0 = time.perf_counter()
        run_e2e(steps_e2e)
        el = time.perf_counter() - t0
        # the last frame read back equals the same step run plainly (stream order check)
        last = steps_e2e - 1
        gv.rebuild(dense)
        hdda.traverse_async(O[cam_of(last)], D[cam_of(last)], gv, prm, bufs, tstatus)
        want = hdda.composite(O[cam_of(last)], D[cam_of(last)], bufs, field).cpu()
        if int(tstatus.item()) != 0 or not torch.equal(out_host[last % 2], want):
            raise RuntimeError("pipelined end-to-end frame differs from the plain step")
        e2e = {"value": n * steps_e2e * world / el, "unit": "rays/s",
               "h2d_bytes_per_step": int(2 * n * 3 * 4),
               "d2h_bytes_per_step": int(n * 4 * 4),
               "overlap": "uploads and read-backs on two copy streams, two slots deep",
               "cameras": "the same 20-camera cycle as the timed steps",
               "l2": "not flushed between steps: each step writes and reads its samples "
                     "(hundreds of MB, more than the L2)"}

    # --- roofline of the dominant kernel -----------------------------------
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    # FP32 pipe: 128 lanes per SM per clock at the maximum SM clock
    alu_peak = n_sm * 128 * sm_mhz * 1e6 / 1e12
    S_avg = samples / K
    grid_bytes = int(vstats.bytes)
    G = int(sc.field.shape[0])
    # algorithmic bytes per launch: what each kernel must move at least.  Walk: the rays
    # (24 B each) and the grid once.  Emit: the CSR offsets (8 B per ray) and the samples
    # (ray_idx, t0, t1: 12 B each).  Compositor: rays, offsets, t0/t1 (8 B per sample),
    # the pixels (16 B per ray) and the field.  The sampler as a whole: rays in, offsets
    # and samples out, grid once.
    sampler_bytes = 24 * n + 8 * (n + 1) + 12 * S_avg + grid_bytes
    alg_bytes = {
        "hdda_walk_emit": sampler_bytes,
        "hdda_walk": 24 * n + grid_bytes,
        "hdda_emit": 8 * (n + 1) + 12 * S_avg,
        "build_vdb": sc.occ.size + grid_bytes,
        "composite": 24 * n + 8 * (n + 1) + 8 * S_avg + 16 * n + 32 * G,
    }
    alg_inst = {"composite": evals_step * COMPOSITE_FP32_PER_BLOB}
    traffic = PROFILED_TRAFFIC.get(workload, {})
    per_kernel = {}
    for name, (launches, tot_ms) in kern.items():
        avg = tot_ms / max(1, launches)
        ent = {"launches": launches, "avg_ms": round(avg, 4), "share": round(tot_ms / ms_prof, 4)}
        if name in alg_bytes:
            ent["alg_bytes"] = int(alg_bytes[name])
            ent["gbs"] = round(alg_bytes[name] / (avg / 1e3) / 1e9, 1)
        if name in traffic:
            ent["traffic"] = traffic[name]
        ent.update(PROFILED_COUNTERS.get(workload, {}).get(name, {}))
        if name in alg_inst:
            ent["fp32_tops"] = round(alg_inst[name] / (avg / 1e3) / 1e12, 2)
            ent["blob_evals_per_sample"] = round(evals_step / max(S_avg, 1), 2)
        per_kernel[name] = ent

    def roof(name):
        launches, tot_ms = kern[name]
        avg = tot_ms / max(1, launches)
        if name in alg_inst:
            ach = alg_inst[name] / (avg / 1e3) / 1e12
            return {"kernel": name, "bound": "alu", "achieved": round(ach, 2),
                    "peak": round(alu_peak, 2), "unit": "T FP32 ops/s",
                    "frac": round(ach / alu_peak, 4), "traffic": traffic.get(name),
                    "alg_bytes": int(alg_bytes.get(name, 0)),
                    "peak_source": "derived: SMs x 128 FP32 lanes x max SM clock"}
        ach = alg_bytes.get(name, 0) / (avg / 1e3) / 1e9
        return {"kernel": name, "bound": "hbm", "achieved": round(ach, 1), "peak": hbm_peak,
                "unit": "GB/s", "frac": round(ach / hbm_peak, 4),
                "traffic": traffic.get(name),
                "peak_source": peak_src}

    dom = max(kern.items(), key=lambda kv: kv[1][1])[0] if kern else None
    roofline = roof(dom) if dom else None
    # the sampler as a whole (walk then emit, or one walk-and-emit kernel): rays in, CSR
    # offsets and samples out
    sam_k = (("hdda_walk_emit",) if "hdda_walk_emit" in kern
             else ("hdda_walk", "hdda_emit"))
    sam_ms = sum(kern[k][1] / max(1, kern[k][0]) for k in sam_k if k in kern)
    roofline_sampler = None
    if sam_ms > 0:
        ach = sampler_bytes / (sam_ms / 1e3) / 1e9
        roofline_sampler = {"kernels": list(sam_k), "bound": "hbm",
                            "alg_bytes": int(sampler_bytes), "ms": round(sam_ms, 4),
                            "achieved": round(ach, 1), "peak": hbm_peak, "unit": "GB/s",
                            "frac": round(ach / hbm_peak, 4), "peak_source": peak_src}

    # the build_vdb timer spans the builder's four kernels; every other timer one kernel
    launches_per_step = (sum(v[0] * KERNELS_PER_TIMER.get(k, 1) for k, v in kern.items()) / K
                         if kern else None)

    # --- CPU oracle on a bounded sample (rank 0, N = 1) -------------------
    cpu = None
    if full and rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(sc, rays[0], args.cpu_stride or stride)
        cpu["all_cores"] = cpu_baseline_all_cores(sc, rays[0],
                                                  max(1, (args.cpu_stride or stride) // 4))
    K_cand = lattice_candidates(sc.params)
    # t update (2 ops, 5 with a growing step) + midpoint 2 + position 6 + floors 3 + compares 3
    cand_ops = (5 if sc.params.cone > 0 else 2) + 2 + 6 + 3 + 3

    line = {
        "metric": "rays/sec and samples/sec, HDDA vs dense-DDA on same GB300 (bit-exact); % HBM roofline",
        "value": round(value, 1), "unit": "rays/s", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": round(ms / K, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": desc, "rays_per_step": n,
                   "occupancy": [round(float(sc.occ[l].mean()), 4) for l in range(sc.levels)],
                   "step": "vdb rebuild + hdda walk and emit (stream-ordered) + composite",
                   "ray_order": f"each camera's pixels row by row, image width {img_w} passed "
                                "(hdda_params.image_width: the walk takes 8x4 pixel blocks)",
                   "l2": "flushed between steps (256 MiB write), flush outside timed windows",
                   "parallelism": f"replicas x{world}"},
        "samples_per_s": round(samples * world / (ms / 1e3), 1),
        "samples_per_step": int(S_avg),
        "candidates_per_ray": K_cand,
        "candidate_alu_bound": {
            "fp32_ops_per_candidate": cand_ops,
            "ms_per_frame_at_peak": round(n * K_cand * cand_ops / (alu_peak * 1e12) * 1e3, 4),
            "note": "FP32 issue alone of stepping every lattice candidate (t update, midpoint, "
                    "position, 3 floors, 3 compares) at the derived FP32 peak; both walks "
                    "cross regions instead and touch a candidate only to confirm a crossing "
                    "or to write a kept sample"},
        "hdda_sampler": {"rays_per_s": round(n * K * world / (ms_sh / 1e3), 1),
                         "samples_per_s": round(samp_sh * world / (ms_sh / 1e3), 1),
                         "candidates_per_s": round(n * K_cand * K * world / (ms_sh / 1e3), 1),
                         "ms_per_frame": round(ms_sh / K, 4)},
        "dense_dda_sampler": {"rays_per_s": round(n * K2 * world / (ms_sd / 1e3), 1),
                              "samples_per_s": round(samp_sd * world / (ms_sd / 1e3), 1),
                              "candidates_per_s": round(n * K_cand * K2 * world
                                                        / (ms_sd / 1e3), 1),
                              "ms_per_frame": round(ms_sd / K2, 4)},
        "dense_dda_step": {"rays_per_s": round(n * K2 * world / (ms_dense / 1e3), 1),
                           "ms_per_step": round(ms_dense / K2, 4)},
        "render_only_step": {
            "note": "vdb rebuild + hdda_render: the walk, then runs expanded from the lattice "
                    "table and composited in one kernel; no sample, scan or host read-back",
            "rays_per_s": round(n * K * world / (ms_r / 1e3), 1),
            "ms_per_step": round(ms_r / K, 4),
            "vs_step": round(ms / ms_r, 3),
            "kernels": {k: {"launches": v[0], "avg_ms": round(v[1] / max(1, v[0]), 4)}
                        for k, v in kern_r.items()},
            "render_fp32_tops": (round(render_evals * COMPOSITE_FP32_PER_BLOB
                                     / (kern_r["hdda_render"][1] / kern_r["hdda_render"][0] / 1e3)
                                     / 1e12, 2) if "hdda_render" in kern_r else None)},
        "fused_sampler_form": {
            "note": "the same step and sampler with the walk and the emit in one persistent "
                    "kernel (hdda_set_sampler_form(HDDA_SAMPLER_FUSED)); same samples",
            "step_ms": round(ms_fu / K, 4),
            "sampler_ms_per_frame": round(ms_fu_s / K, 4),
            "speedup_vs_separate": round(ms_sh / ms_fu_s, 3),
            "kernels": {k: {"launches": v[0], "avg_ms": round(v[1] / max(1, v[0]), 4)}
                        for k, v in kern_fu.items()}},
        "ray_order": {
            "note": "the same step and samplers without the image width: the walk takes "
                    "32 consecutive rays (an image-row segment) per warp; same outputs",
            "step_ms": round(ms_io / K, 4),
            "hdda_sampler_ms_per_frame": round(ms_io_s / K, 4),
            "dense_sampler_ms_per_frame": round(ms_io_d / K2, 4),
            "walk_ms": (round(kern_io["hdda_walk"][1] / max(1, kern_io["hdda_walk"][0]), 4)
                        if "hdda_walk" in kern_io else None),
            "hdda_sampler_speedup_of_blocks": round(ms_io_s / ms_sh, 3),
            "dense_sampler_speedup_of_blocks": round(ms_io_d / ms_sd, 3)},
        "hdda_vs_dense_sampler_speedup": round(ms_sd / K2 / (ms_sh / K), 3),
        "grid": {"vdb_bytes": grid_bytes, "vdb_plain_bytes": plain_bytes,
                 "dense_bytes": int(vstats.dense_bytes),
                 "n_leaves": int(vstats.n_leaves), "n_tiles": int(vstats.n_tiles)},
        "kernels": per_kernel,
        "kernels_dense_step": {k: {"launches": v[0], "avg_ms": round(v[1] / max(1, v[0]), 4)}
                               for k, v in kern_dense.items()},
        "roofline": roofline,
        "roofline_sampler": roofline_sampler,
        "gpu_launches": int(round(launches_per_step * K)) if launches_per_step else 0,
        "clocks": clk,
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    if full:
        line.update({
            "hdda_plain_vdb_sampler": {"rays_per_s": round(n * K2 * world / (ms_sp / 1e3), 1),
                                       "ms_per_frame": round(ms_sp / K2, 4),
                                       "note": "HDDA on the plain VDB tree (8^3 leaves, 16^3-block "
                                               "nodes), refinement masks off"},
            "skip_form_samplers": {
                "note": "Algorithm 2 control flow (leading empty regions in an inner loop); "
                        "same samples",
                "hdda_ms_per_frame": round(ms_ss / K2, 4),
                "dense_ms_per_frame": round(ms_ds / K2, 4)},
            "synchronous_step": {"note": "the same step through hdda_traverse_hdda, which reads "
                                         "the sample total back to the host before compositing",
                                 "ms_per_step": round(ms_sync / K2, 4)},
            "incremental_update": upd,
            "fused_step": {
                "note": "vdb rebuild + hdda_traverse_composite: the walk and the tile scan, then "
                        "one kernel that writes every sample at its CSR position and composites "
                        "it (the same samples as the step, the render-only path's frame)",
                "rays_per_s": round(n * K * world / (ms_f / 1e3), 1),
                "ms_per_step": round(ms_f / K, 4),
                "vs_step": round(ms / ms_f, 3),
                "kernels": {k: {"launches": v[0], "avg_ms": round(v[1] / max(1, v[0]), 4)}
                            for k, v in kern_f.items()}},
        })
    return line


def cpu_baseline(sc, ray_pair, stride):
    """Oracle (as it stands) on every stride-th ray of camera 0: sampler + compositor."""
    import numpy as np
    import oracle

    o, d = ray_pair
    sel = np.arange(0, o.shape[0], stride)
    so, sd = np.ascontiguousarray(o[sel]), np.ascontiguousarray(d[sel])
    p = sc.params
    t0 = time.perf_counter()
    off, idx, a, b = oracle.sample(so, sd, sc.occ, sc.aabbs, p.near, p.far, p.step, p.cone,
                                   p.max_step, p.max_steps)
    t1 = time.perf_counter()
    oracle.composite(so, sd, off, a, b, sc.field)
    t2 = time.perf_counter()
    return {"value": round(sel.size / (t2 - t0), 1), "unit": "rays/s", "cores": 1,
            "kind": "oracle",
            "sample": f"every {stride}th ray of camera 0 ({sel.size} rays, {int(off[-1])} samples)",
            "sampler_rays_per_s": round(sel.size / (t1 - t0), 1), "seconds": round(t2 - t0, 2)}


def _oracle_chunk(job):
    """One worker's share of the all-cores CPU baseline (runs in a spawned process)."""
    import oracle
    o, d, occ, aabbs, p, field = job
    if o.shape[0] == 0:
        return 0.0, 0
    t0 = time.perf_counter()
    off, _, a, b = oracle.sample(o, d, occ, aabbs, *p)
    oracle.composite(o, d, off, a, b, field)
    return time.perf_counter() - t0, int(off[-1])


def cpu_baseline_all_cores(sc, ray_pair, stride):
    """The same oracle on every host core: the rays dealt round-robin into one share per
    process (spawned, so no process inherits the CUDA context)."""
    import multiprocessing as mp

    import numpy as np
    cores = len(os.sched_getaffinity(0))
    o, d = ray_pair
    sel = np.arange(0, o.shape[0], stride)
    p = sc.params
    prm = (p.near, p.far, p.step, p.cone, p.max_step, p.max_steps)
    parts = [sel[i::cores] for i in range(cores)]
    jobs = [(np.ascontiguousarray(o[s]), np.ascontiguousarray(d[s]), sc.occ, sc.aabbs, prm,
             sc.field) for s in parts]
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_chunk, [(j[0][:1], j[1][:1]) + j[2:] for j in jobs])  # warm the workers
        t0 = time.perf_counter()
        res = pool.map(_oracle_chunk, jobs)
        wall = time.perf_counter() - t0
    return {"value": round(sel.size / wall, 1), "unit": "rays/s", "cores": cores,
            "kind": "oracle",
            "sample": f"every {stride}th ray of camera 0 ({sel.size} rays, "
                      f"{sum(r[1] for r in res)} samples), split over {cores} processes",
            "seconds": round(wall, 2)}


def lattice_candidates(p) -> int:
    """Candidates per ray: the length of the shared lattice, by the binary32 recurrence."""
    import numpy as np
    f32 = np.float32
    t, far = f32(p.near), f32(p.far)
    step, cone, mx = f32(p.step), f32(p.cone), f32(p.max_step)
    k = 0
    while True:
        tn = f32(t + min(max(f32(t * cone), step), mx))
        if tn > far:
            return k
        k += 1
        t = tn


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle on bounded samples of the same workload
# ---------------------------------------------------------------------------

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np
    import oracle
    from paper_2404_10272_gb300 import scenes

    oracle.build()
    sc, cams, desc, cpu_stride = frame_workload(args.workload)
    stride = 16 * cpu_stride  # each step: a bounded sample of one camera's rays

    def step(j):
        o, d = cams[j % N_CAMERAS].rays()
        sel = np.arange(j % stride, o.shape[0], stride)
        so, sd = np.ascontiguousarray(o[sel]), np.ascontiguousarray(d[sel])
        p = sc.params
        t0 = time.perf_counter()
        off, idx, a, b = oracle.sample(so, sd, sc.occ, sc.aabbs, p.near, p.far, p.step, p.cone,
                                       p.max_step, p.max_steps)
        oracle.composite(so, sd, off, a, b, sc.field)
        return sel.size, time.perf_counter() - t0

    for j in range(args.warmup):
        step(j)
    rays = 0
    el = 0.0
    for j in range(args.steps):
        r, t = step(args.warmup + j)
        rays += r
        el += t
    v = rays / el
    print(json.dumps({
        "impl": "reference",
        "metric": "rays/sec and samples/sec, HDDA vs dense-DDA on same GB300 (bit-exact); % HBM roofline",
        "value": round(v, 1), "unit": "rays/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(el / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": desc, "parallelism": "cpu, 1 thread"},
        "cpu_baseline": {"value": round(v, 1), "unit": "rays/s", "cores": 1, "kind": "oracle",
                         "sample": f"each step: every {stride}th ray of one camera"},
        "e2e": {"value": round(v, 1), "unit": "rays/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def profile_step(args):
    """Kernel launch order: sample (count only), build, sample, composite (warm-up),
    build, sample, composite (the step to capture).  For "render": build, render
    (warm-up), build, render."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2404_10272_gb300 import hdda

    sc, cams, _, _ = frame_workload(args.workload)
    o, d = cams[0].rays()
    if args.profile_rays > 0:
        o, d = o[:args.profile_rays].copy(), d[:args.profile_rays].copy()
    O, D = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    dense = torch.from_numpy(sc.occ).cuda()
    field = torch.from_numpy(sc.field).cuda()
    p = sc.params
    # the rays in image order with the image width, as the bench's timed loops pass them
    # (a ray prefix of --profile-rays keeps it: whole rows and a partial last one)
    prm = hdda.make_params(p.near, p.far, p.step, p.cone, p.max_step, p.max_steps,
                           image_width=cams[0].width)
    vdb = args.profile_step in ("hdda", "render")
    hdda.set_sampler_form(hdda.SAMPLER_FUSED if args.sampler_form == "fused"
                          else hdda.SAMPLER_SEPARATE)
    grid = hdda.build_vdb(dense, sc.aabbs) if vdb else hdda.pack_dense(dense, sc.aabbs)
    trav = hdda.traverse_hdda if vdb else hdda.traverse_dense
    rgba = torch.empty((o.shape[0], 4), dtype=torch.float32, device="cuda")
    if args.profile_step == "render":
        # the render-only step twice: rebuild, walk, run-level compositing
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        for _ in range(2):
            grid.rebuild(dense)
            hdda.render(O, D, grid, prm, field, out=rgba, status=status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        print(f"profile step done: {o.shape[0]} rays, render only")
        return
    cap = trav(O, D, grid, prm, count_only=True).total
    bufs = hdda.alloc_samples(o.shape[0], cap)
    for _ in range(2):
        grid.rebuild(dense)
        s = trav(O, D, grid, prm, out=bufs)
        hdda.composite(O, D, s, field, out=rgba)
    torch.cuda.synchronize()
    print(f"profile step done: {o.shape[0]} rays, {s.total} samples")


def run_batch(args, quick: bool = False) -> dict:
    """64 (scene, camera) jobs, 64^2..800^2 rays each, 1-4 cascade levels: one autotuned,
    graph-captured batch launch per step against 64 separate single-call launches.  quick:
    a reduced tuning space (walk block 256, 32 or 64 rays per fetch, 2 or 4 emit warps, then
    the control flow) and fewer timed launches, for the summary in the headline line."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2404_10272_gb300 import autotune, hdda, scenes

    sc, specs = scenes.batch_jobs(seed=1004, n=64)
    grids = {k: hdda.build_vdb(torch.from_numpy(s.occ).cuda(), s.aabbs) for k, s in sc.items()}
    jobs = []
    for sp in specs:
        s = sc[sp["scene"]]
        p = s.params
        prm = hdda.make_params(p.near, p.far, p.step, p.cone, p.max_step, p.max_steps)
        O = torch.from_numpy(sp["rays_o"]).cuda()
        D = torch.from_numpy(sp["rays_d"]).cuda()
        tot = hdda.traverse_hdda(O, D, grids[sp["scene"]], prm, count_only=True).total
        jobs.append(dict(rays_o=O, rays_d=D, grid=grids[sp["scene"]], params=prm,
                         out=hdda.alloc_samples(O.shape[0], max(1, tot))))
    n_rays = sum(int(j["rays_o"].shape[0]) for j in jobs)

    def make(cfg):
        return hdda.Batch(jobs, config=cfg, use_graph=True)

    space = autotune.SPACE
    if quick:
        space = [(256, rpf, ew, autotune.WALK_BRANCH) for rpf in (32, 64) for ew in (2, 4)]
    t_tune = time.perf_counter()
    best, timings = autotune.tune(make, autotune.signature(jobs), space=space,
                                  reps=3 if quick else 5, warmup=2, use_cache=False)
    t_tune = time.perf_counter() - t_tune
    b = make(best)
    K = min(args.steps, 20) if quick else args.steps
    W = args.warmup
    for _ in range(W):
        b.launch()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(K):
        b.launch()
    e1.record()
    e1.synchronize()
    ms_batch = e0.elapsed_time(e1) / K
    clk = clocks.stop()
    totals, _ = b.results()
    samples = sum(totals)

    def separate():
        for j in jobs:
            hdda.traverse_hdda(j["rays_o"], j["rays_d"], j["grid"], j["params"], out=j["out"])

    for _ in range(2):
        separate()
    torch.cuda.synchronize()
    reps = max(3, K // 4)
    e0.record()
    for _ in range(reps):
        separate()
    e1.record()
    e1.synchronize()
    ms_sep = e0.elapsed_time(e1) / reps
    b.free()
    return {
        "metric": "batched sampling: total rays/s of 64 mixed jobs in one graph launch",
        "value": round(n_rays / (ms_batch / 1e3), 1), "unit": "rays/s", "n_gpus": 1, "steps": K,
        "warmup": W, "ms_per_step": round(ms_batch, 4), "higher_is_better": True,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "64 jobs: tiny-type 64^3 and object-type 128^3 scenes with 1-4 "
                               "cascade levels, images uniform 64..800 per side (seed 1004)",
                   "rays_per_step": n_rays, "samples_per_step": int(samples),
                   "autotuned": {"walk_block": best[0], "rays_per_fetch": best[1],
                                 "emit_warps": best[2],
                                 "walk_form": "skip" if len(best) > 3 and best[3] else "branch"},
                   "l2": "not flushed: 64 jobs' outputs exceed the L2 each step"},
        "samples_per_s": round(samples / (ms_batch / 1e3), 1),
        "separate_launches": {"ms_per_step": round(ms_sep, 4),
                              "rays_per_s": round(n_rays / (ms_sep / 1e3), 1)},
        "speedup_vs_separate": round(ms_sep / ms_batch, 3),
        "autotune": {"seconds": round(t_tune, 2), "candidates": len(timings),
                     "median_ms": {"/".join(str(x) for x in k): round(sorted(v)[len(v) // 2], 4)
                                   for k, v in sorted(timings.items())},
                     "key": "walk_block/rays_per_fetch/emit_warps/walk_variant (1 = skip)"},
        "clocks": clk,
    }


# Offered load of the serving measurement: a stated constant, below the capacity of both
# executor modes, so that the tail reflects queueing at a known load rather than a noisy
# capacity estimate.
SERVE_LOAD = 400.0   # requests per second


def run_serve(args, quick: bool = False) -> dict:
    """Continuous-batching server: 8 resident scenes, Poisson arrivals of 200x200..1920x1080
    requests (log-uniform sides) at SERVE_LOAD requests/s; p50/p99 latency over three repeats
    of the same request sequence, for both executor modes, and each mode's closed-loop
    capacity (a burst, context only).  An unmeasured repeat comes first.  quick: 2.5 s of
    arrivals per repeat instead of 6 s."""
    import math
    import random

    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2404_10272_gb300 import scenes, serve

    scene_list = ([scenes.tiny_scene(seed=2001 + i) for i in range(4)]
                  + [scenes.object_scene(seed=3001 + i) for i in range(4)])
    rng = np.random.default_rng(1005)
    pool = []
    for i in range(16):
        W = int(round(math.exp(rng.uniform(math.log(200), math.log(1920)))))
        H = int(round(math.exp(rng.uniform(math.log(200), math.log(1080)))))
        o, d = scenes.orbit_camera(rng, 4.0, W, H, 0.69).rays()
        pool.append((torch.from_numpy(o).pin_memory(), torch.from_numpy(d).pin_memory(), W))
    slots = 4
    budget = 8 << 30
    seconds = 2.5 if quick else 6.0
    pick = random.Random(7)

    def make(rid):
        o, d, w = pool[pick.randrange(len(pool))]
        return serve.Request(rid=rid, scene=pick.randrange(len(scene_list)), rays_o=o, rays_d=d,
                             width=w)

    def capacity(ex):
        srv = serve.RenderServer(ex, slots=slots, budget_bytes=budget)
        for i in range(16):
            srv.submit(make(i))
        srv.drain()
        burst = [make(100 + i) for i in range(48 if quick else 96)]
        t0 = time.perf_counter()
        for r in burst:
            srv.submit(r)
        srv.drain()
        cap = len(burst) / (time.perf_counter() - t0)
        srv.close()
        return cap

    lat_ms = []  # latencies of the measured requests of the current mode's repeats

    def at_load(ex, lam):
        """One repeat: the same Poisson arrival sequence (seed 1006) and request mix (seed 7).
        Python's cyclic garbage collector is paused during the repeat (as a latency-bound
        server would run it) and run in between."""
        gc.collect()
        gc.disable()
        try:
            return _at_load(ex, lam)
        finally:
            gc.enable()

    def _at_load(ex, lam):
        pick.seed(7)
        n_req = max(60, int(lam * seconds))
        gaps = np.random.default_rng(1006).exponential(1.0 / lam, size=n_req)
        srv = serve.RenderServer(ex, slots=slots, budget_bytes=budget, samples_per_ray_hint=40)
        reqs = [make(1000 + i) for i in range(n_req)]
        t_start = time.perf_counter()
        t_next = t_start
        for r, g in zip(reqs, gaps):
            t_next += g
            delay = t_next - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            r.arrival = t_next
            srv.submit(r)
        srv.drain(timeout=300)
        wall = max(r.done for r in reqs) - t_start
        srv.close()
        measured = reqs[len(reqs) // 10:]   # drop the first 10 % (warm-up of the queue)
        summ = serve.summary(measured, wall * len(measured) / len(reqs))
        lat_ms.extend(r.latency * 1e3 for r in measured if r.error is None)
        return {"p50_ms": summ["p50_ms"], "p99_ms": summ["p99_ms"], "mean_ms": summ["mean_ms"],
                "frames_per_s": summ["frames_per_s"], "rays_per_s": summ["rays_per_s"],
                "re_runs": summ["retries"], "errors": summ["errors"],
                "max_concurrent": srv.max_concurrent, "admission_ticks": srv.ticks}

    clocks = ClockSampler(0)
    clocks.start()
    modes = {}
    for mode in ("samples", "batched", "render"):
        pick.seed(7)
        ex = serve.GpuExecutor(scene_list, slots=slots, mode=mode)
        ex.warm()
        cap = capacity(ex)
        at_load(ex, SERVE_LOAD)   # warm-up repeat: the allocator's pools grow to the mix
        lat_ms.clear()
        reps = [at_load(ex, SERVE_LOAD) for _ in range(3)]
        p99 = [r["p99_ms"] for r in reps]
        p50 = [r["p50_ms"] for r in reps]
        modes[mode] = {
            "p50_ms": round(statistics.median(p50), 3), "p99_ms": round(statistics.median(p99), 3),
            "p99_spread": round((max(p99) - min(p99)) / statistics.median(p99), 3),
            # the three repeats' requests together: a p99 over three times the samples
            "p99_pooled_ms": round(serve.percentile(lat_ms, 0.99), 3),
            "repeats": reps, "capacity_frames_per_s": round(cap, 1)}
    clk = clocks.stop()
    return {
        "metric": "serving: p50/p99 latency and frames/s at a fixed offered load",
        "value": modes["samples"]["p99_pooled_ms"],
        "unit": "ms (p99 latency over the three repeats' requests)", "n_gpus": 1,
        "higher_is_better": False, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "8 resident scenes (4 tiny-type 64^3, 4 object-type 128^3), "
                               "requests 200x200..1920x1080 log-uniform",
                   "slots": slots, "memory_budget_bytes": budget,
                   "offered_load_frames_per_s": SERVE_LOAD,
                   "seconds_per_repeat": seconds, "repeats": 3,
                   "arrivals": "Poisson (seed 1006), the same sequence in every repeat, after "
                               "one unmeasured repeat"},
        "samples_mode": dict(modes["samples"], note="traversal + compositing through sample "
                                                    "buffers, one request per slot"),
        "batched_mode": dict(modes["batched"], note="a slot samples every ready request (up to "
                                                    "8) in one hdda_batch launch, then "
                                                    "composites each frame"),
        "render_mode": dict(modes["render"], note="hdda_render: no sample buffers, no re-runs"),
        "clocks": clk,
    }


def main():
    args = parse_args()
    if args.profile_step:
        profile_step(args)
        return
    if args.workload == "batch" and args.impl == "ours":
        print(json.dumps(run_batch(args)), flush=True)
        return
    if args.workload == "serve" and args.impl == "ours":
        print(json.dumps(run_serve(args)), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
