#!/usr/bin/env python
"""Benchmark of the bricked ray caster on the HI-survey workload.

One step = one frame of the whole hot path at a pose of a 120-pose orbit about
the y axis: host plan (rendering rectangles, empty-space skipping, view order),
ray march of every (brick, tile) item, sort-last 'over' composite.  K timed
steps visit K poses evenly spaced over the orbit (all 120 when K = 120), so the
frame rate is an orbit mean; warm-up frames render poses spread over the orbit
too.

Workload (default): float32 cube 1024 x 1024 x 2048 (8 GiB; noise + 2000 line
sources + 50 continuum sources), 128^3 bricks, 1920 x 1080 image, step 0.5
voxel, 16-point transfer function TF-A, termination at alpha >= 0.99.  The cube
is larger than L2, so no L2 flush is needed between frames.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on the same workload instead (a bounded pixel sample per step).
Multi-GPU (torchrun): each rank renders its own share of the orbit (no data
exchange), the job time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "ray samples/s & 1080p FPS vs HBM roofline; learned vs plain FPS @>=45 dB PSNR"
UNIT = "ray samples/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=120)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", choices=["hi", "mid", "tiny", "xl"], default="hi",
                    help="xl (with --learned): the 4096x4096x3200 (~200 GiB) cube, generated brick by brick "
                         "on request, learned against plain out-of-core at the same device budgets")
    ap.add_argument("--tf", choices=["a", "b"], default="a")
    ap.add_argument("--width", type=int, default=0, help="override the image width")
    ap.add_argument("--height", type=int, default=0, help="override the image height")
    ap.add_argument("--kernel", choices=["auto", "tma", "direct", "tex"], default="auto")
    ap.add_argument("--precision", choices=["f32", "f16", "f8"], default="f32",
                    help="storage of the texture march's cube copies (FP32, FP16, FP8 E4M3 per-brick scale)")
    ap.add_argument("--tex-slab-layers", type=int, default=0,
                    help="texture march: layers per slab of the layered copies (0: the device limit)")
    ap.add_argument("--mip", action="store_true",
                    help="maximum intensity projection + colour map (the paper's mode, Section 2.3.3)")
    ap.add_argument("--dynamic-step", action="store_true",
                    help="dynamic step: samples `step` voxels apart along each ray's dominant axis")
    ap.add_argument("--shard", type=int, default=1,
                    help="render each frame as this many virtual ranks on one GPU (k-d leaves, one "
                         "stream each, root fold of the rectangle-clipped sub-images)")
    ap.add_argument("--ooc", action="store_true",
                    help="out-of-core: the cube stays in host memory, bricks stream into a device cache")
    ap.add_argument("--budget-gib", type=float, default=0.0,
                    help="device brick-cache budget for --ooc in GiB (0: every brick)")
    ap.add_argument("--ooc-march", choices=["auto", "direct", "tex", "texz", "texxz"], default="auto",
                    help="out-of-core and learned marches: direct on the blocks, texture march on three "
                         "layered copies of the slots, on one copy along z, or on the copies along x and z "
                         "(VR_OPT_OOC_MARCH)")
    ap.add_argument("--serve", action="store_true",
                    help="serving loop: Poisson arrivals of camera/TF/resolution requests, p50/p99 latency")
    ap.add_argument("--rate", type=float, default=200.0, help="--serve: mean arrivals per second")
    ap.add_argument("--serve-seconds", type=float, default=10.0, help="--serve: length of the arrival window")
    ap.add_argument("--arena-gib", type=float, default=16.0, help="--serve: device arena (two batch halves)")
    ap.add_argument("--max-batch", type=int, default=32, help="--serve: frames per batch at most")
    ap.add_argument("--learned", action="store_true",
                    help="learned brick codec: train latents + MLP on the cube, render from decoded bricks, PSNR")
    ap.add_argument("--train-steps", type=int, default=3000)
    ap.add_argument("--train-batch", type=int, default=262144)
    ap.add_argument("--train-lr", type=float, default=3e-3)
    ap.add_argument("--psnr-poses", type=int, default=12)
    ap.add_argument("--codec-brick", type=int, default=0,
                    help="--learned: brick edge of the codec and of the learned render; --ooc: brick edge "
                         "of the streamed bricks (0: the workload's)")
    ap.add_argument("--active-frac", type=float, default=0.5,
                    help="--learned: share of training points drawn from voxels the transfer function can show")
    ap.add_argument("--fallback-bound", type=float, default=None,
                    help="--learned: bricks whose decode error (above the TF floor, in data units) exceeds "
                         "this are copied from pinned plain blocks instead of decoded")
    ap.add_argument("--xl-budgets-gib", default="32,96",
                    help="--config xl: device brick-cache budgets (GiB) at which both forms render")
    ap.add_argument("--xl-frames", type=int, default=4, help="--config xl: timed frames per form and budget")
    ap.add_argument("--xl-slab-layers", type=int, default=4,
                    help="--config xl: brick layers per training slab (generated on the host, copied to the device)")
    ap.add_argument("--xl-decoder-slabs", type=int, default=3,
                    help="--config xl: slabs the shared decoder is trained on (--train-steps each)")
    ap.add_argument("--xl-slab-steps", type=int, default=1500,
                    help="--config xl: steps fitting each slab's latents to the trained decoder")
    ap.add_argument("--xl-scale", type=int, default=1,
                    help="--config xl: divide each axis by this and the source counts by its cube (quick checks)")
    ap.add_argument("--protocol-repeats", type=int, default=10,
                    help="after the timed orbit, render every pose this many times and report the per-pose "
                         "median and the 75th percentile over poses (0: skip)")
    ap.add_argument("--e2e-steps", type=int, default=120)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def workload(args):
    spec, tf, poses, desc = _workload(args)
    if args.width or args.height:
        W = args.width or spec["width"]
        H = args.height or spec["height"]
        spec["width"], spec["height"] = W, H
        poses = [dict(c, width=W, height=H) for c in poses]
        desc += f", image overridden to {W}x{H}"
    if args.ooc and args.codec_brick:
        spec["brick"] = (args.codec_brick,) * 3
        desc += f", bricks overridden to {args.codec_brick}^3"
    return spec, tf, poses, desc


def _workload(args):
    if args.config == "hi":
        spec = dict(synth.HI)
        tf = synth.tf_hi_a() if args.tf == "a" else synth.tf_hi_b()
        poses = synth.orbit(spec["shape_xyz"], 120, 15.0, spec["width"], spec["height"])
        desc = ("HI-survey cube 1024x1024x2048 f32 (noise + 2000 line + 50 continuum sources), "
                f"128^3 bricks, 1920x1080, step 0.5, 16-point TF-{args.tf.upper()}, "
                "tau 0.99, 120-pose orbit about y at 15 deg elevation")
    elif args.config == "mid":
        spec = dict(synth.MID)
        tf = synth.tf_hi_a() if args.tf == "a" else synth.tf_hi_b()
        poses = synth.orbit(spec["shape_xyz"], 120, 15.0, spec["width"], spec["height"])
        desc = ("mid-size HI-like cube 512x512x1024 f32 (1 GiB), 128^3 bricks, 1920x1080, "
                f"step 0.5, 16-point TF-{args.tf.upper()}, profiling case")
    else:
        spec = dict(synth.TINY)
        tf = synth.tf_tiny()
        poses = synth.tiny_views()
        desc = "tiny 64^3 cube, 32^3 bricks, 256x256, step 0.5, 8-point TF, 4 views"
    return spec, tf, poses, desc


def make_cube(spec):
    if spec["name"] == "hi":
        return synth.hi_cube()
    if spec["name"] == "mid":
        return synth.hi_cube(seed=4, shape_xyz=spec["shape_xyz"], n_line=250, n_cont=25)
    return synth.tiny_cube()


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "utilization.gpu",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) != len(self.FIELDS):
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[3], parts[4:]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        loaded = [r for r in rows if r[2] not in ("0", "[N/A]")] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in loaded for k, v in enumerate(r[3]) if v == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in loaded),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows), "samples_loaded": len(loaded)}


# ------------------------------------------------------------------ roofline inputs

def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


KERNEL_SOURCES = ("vr_kernels.cu", "vr_march_tma.cu", "vr_march_tex.cu", "vr_device.cuh",
                  "vr_internal.cuh", "df.cuh")


def kernel_source_hash():
    """Hash of the device sources; a recorded ncu traffic figure is reported only
    while this hash matches the one stored with it."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_1205_0282_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def recorded_inst_per_sample(kernel, workload_name):
    """Thread instructions per composited sample of the march kernel from a
    committed ncu capture (smsp__thread_inst_executed.sum over the frame's
    samples), only if the kernel source is unchanged since that capture."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    e = json.load(open(p)).get(kernel, {}).get(workload_name)
    if not e or e.get("kernel_source_sha") != kernel_source_hash():
        return None
    return e.get("thread_inst_per_sample")


def recorded_traffic(kernel, workload_name):
    """DRAM bytes per launch from a committed ncu capture, only if the kernel
    source is unchanged since that capture."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(kernel, {}).get(workload_name)
    if not e or e.get("kernel_source_sha") != kernel_source_hash():
        return None
    return e.get("dram_bytes_per_launch")


# ------------------------------------------------------------------ CPU oracle timing

def oracle_rate(cube, tf, poses, brick, seconds, crop=64, keep=False, regions=None, step_mode=0, mode="ea"):
    """Samples/s of the FP64 oracle on centre crops of successive poses, for
    about `seconds` of wall time (at least one crop).  With keep, also returns
    the crops as (camera, pixel indices, RGBA) for the image-quality check.
    regions: the k-d leaf of every brick when frames are rendered as virtual
    ranks (the oracle then folds per leaf first, as the ranks do)."""
    import oracle
    total = 0
    t0 = time.perf_counter()
    k = 0
    crops = []
    while True:
        cam = poses[k % len(poses)]
        W, H = cam["width"], cam["height"]
        x0, y0 = W // 2 - crop // 2, H // 2 - crop // 2
        jj, ii = np.meshgrid(np.arange(y0, y0 + crop), np.arange(x0, x0 + crop), indexing="ij")
        pix = (jj * W + ii).reshape(-1)
        ref, amb, ns = oracle.render(cube, tf, cam, brick=brick, pixels=pix,
                                     amb_alpha=QUALITY_AMB_ALPHA, amb_steps=QUALITY_AMB_STEPS,
                                     regions=regions, step_mode=step_mode, mode=mode)
        total += int(ns.sum())
        crops.append((cam, pix, ref, amb) if keep else None)
        k += 7
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return (total / dt, dt, len(crops), crops) if keep else (total / dt, dt, len(crops))


# A pixel is "ambiguous" for the image-quality figures when the oracle's compositing
# alpha comes within this distance of the termination threshold, or a sample
# position within QUALITY_AMB_STEPS voxel of the ray's exit: there a perturbation
# of that size (FP16/FP8 storage moves voxel values by up to 2^-11 / 2^-4
# relative) may legitimately stop the ray one sample earlier or later.
QUALITY_AMB_ALPHA = 1e-3
QUALITY_AMB_STEPS = 1e-4


def image_quality(render_pose, crops):
    """Per-pixel error of the GPU image against the FP64 oracle's crops (oracle
    on the FP32 cube).  PSNR = 10 log10(1 / MSE) over the RGBA channels, whose
    values lie in [0, 1]; max_abs over all pixels and over the unambiguous ones."""
    errs, ambs = [], []
    for cam, pix, ref, amb in crops:
        errs.append(render_pose(cam, pix).astype(np.float64) - ref.reshape(-1, 4))
        ambs.append(amb.reshape(-1) != 0)
    e = np.concatenate(errs)
    amb = np.concatenate(ambs)
    mse = float(np.mean(e * e))
    per_px = np.abs(e).max(axis=1)
    return {"against": "FP64 oracle on the FP32 cube", "pixels": int(e.shape[0]),
            "sub_views": f"the CPU-baseline crops: {len(crops)} poses",
            "max_abs": float(per_px.max()), "rms": mse ** 0.5,
            "psnr_db": (10 * np.log10(1.0 / mse)) if mse > 0 else None,
            "ambiguous_pixels": int(amb.sum()),
            "ambiguity": f"oracle alpha within {QUALITY_AMB_ALPHA:g} of tau or a sample within "
                         f"{QUALITY_AMB_STEPS:g} voxel of the exit",
            "max_abs_unambiguous": float(per_px[~amb].max()) if (~amb).any() else None,
            "pixels_over_1e-3": int((per_px > 1e-3).sum())}


def cpu_cores():
    n = os.environ.get("OMP_NUM_THREADS")
    return int(n) if n else (os.cpu_count() or 1)


# ------------------------------------------------------------------ ranks

def my_share(items, rank: int, world: int):
    """The orbit poses this rank renders: every world-th pose from its rank
    (replicas: each rank renders whole frames of its own, no data exchange)."""
    return list(items[rank::world]) if world > 1 else list(items)


def orbit_index(k: int, count: int, n: int) -> int:
    """Pose of frame k of `count` frames over an orbit of n poses: evenly spaced
    (floor(k n / count)) when count < n, else every pose in turn, so that the
    timed frames cover the whole orbit whatever the step count."""
    return (k * n) // count % n if count < n else k % n


def job_totals(dist, elapsed: float, counts, device="cpu"):
    """Whole-job numbers over ranks: the slowest rank's time (max) and the summed
    counts (samples, frames, launches ...).  dist is torch.distributed or None."""
    if dist is None:
        return elapsed, [int(c) for c in counts]
    import torch
    t = torch.tensor([elapsed], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(x) for x in counts], dtype=torch.float64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), [int(round(x)) for x in c.tolist()]


# ------------------------------------------------------------------ main

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    spec, tf, poses, desc = workload(args)
    cube = make_cube(spec)
    brick = spec["brick"]
    import oracle
    oracle.build()
    crop = 64 if spec["name"] == "hi" else 128
    for k in range(args.warmup):
        oracle_rate(cube, tf, poses[k:k + 1], brick, 0.0, crop=16)
    total_samples, t = 0, 0.0
    for k in range(args.steps):
        rate, dt, _ = oracle_rate(cube, tf, poses[k % len(poses):] + poses, brick, 0.0, crop=crop)
        total_samples += rate * dt
        t += dt
    value = total_samples / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "sample": f"{crop}x{crop} centre crop of one pose per step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                             "sample": f"{crop}x{crop} centre crop per step, {args.steps} steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    local_world = int(os.environ.get("LOCAL_WORLD_SIZE", str(world)))
    if local_world > 1:
        # the replicas generate their cubes at once: share the host cores (the
        # launcher's default of one thread per process would leave most idle)
        os.environ["OMP_NUM_THREADS"] = str(max(1, (os.cpu_count() or 1) // local_world))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_1205_0282_gb300 import VolumeRenderer

    spec, tf, poses, desc = workload(args)
    cube = make_cube(spec)
    my_poses = my_share(poses, rank, world)
    W, H = spec["width"], spec["height"]

    r = VolumeRenderer(local)
    from paper_1205_0282_gb300 import vr as vrmod
    t_load = time.perf_counter()
    if args.ooc:
        r.load_cube_host(cube)
        r.set_option(vrmod.VR_OPT_OOC_MARCH, OOC_MARCH[args.ooc_march])
        if args.budget_gib > 0:
            r.set_option(vrmod.VR_OPT_DEVICE_BUDGET, int(args.budget_gib * 2 ** 30))
    else:
        dcube = torch.from_numpy(cube).cuda()
        r.load_cube(dcube)
        del dcube
        torch.cuda.empty_cache()
    r.brick(*spec["brick"])
    load_s = time.perf_counter() - t_load
    r.set_transfer_function(tf)
    from paper_1205_0282_gb300 import vr as vrmod
    r.set_option(vrmod.VR_OPT_KERNEL, {"auto": vrmod.VR_KERNEL_AUTO, "tma": vrmod.VR_KERNEL_TMA,
                                       "direct": vrmod.VR_KERNEL_DIRECT, "tex": vrmod.VR_KERNEL_TEX}[args.kernel])
    r.set_option(vrmod.VR_OPT_PRECISION, {"f32": vrmod.VR_PRECISION_F32, "f16": vrmod.VR_PRECISION_F16,
                                          "f8": vrmod.VR_PRECISION_F8}[args.precision])
    r.set_option(vrmod.VR_OPT_STEP_MODE, 1 if args.dynamic_step else 0)
    r.set_option(vrmod.VR_OPT_MODE, 1 if args.mip else 0)
    if args.tex_slab_layers > 0:
        r.set_option(vrmod.VR_OPT_TEX_SLAB_LAYERS, args.tex_slab_layers)
    out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    if args.shard > 1:
        from paper_1205_0282_gb300 import vr as vrm
        leaves = vrm.vr_kd_partition(spec["shape_xyz"], spec["brick"], args.shard)
        leaf_streams = [torch.cuda.Stream() for _ in range(args.shard)]
        leaf_bufs = [torch.empty((H, W, 4), dtype=torch.float32, device="cuda") for _ in range(args.shard)]

    def orbit_pose(k, count):
        return my_poses[orbit_index(k, count, len(my_poses))]

    def frame(k):
        draw(orbit_pose(k, args.steps))

    def draw(cam):
        r.set_camera(cam)
        if args.shard <= 1:
            r.render(out, stream)
            return
        # virtual ranks: leaf j on its own stream into a rectangle-sized buffer,
        # then the root stream folds the sub-images in visibility order
        subs, rects = [], []
        for j in range(args.shard):
            r.set_region(leaves[j, :3], leaves[j, 3:])
            rect = r.region_rect()
            n_px = max(int(rect[2] - rect[0] + 1), 0) * max(int(rect[3] - rect[1] + 1), 0)
            leaf_streams[j].wait_stream(stream)
            sub = None
            if n_px:
                sub = leaf_bufs[j].view(-1)[:n_px * 4].view(int(rect[3] - rect[1] + 1), int(rect[2] - rect[0] + 1), 4)
                r.render_rect(rect, sub, leaf_streams[j])
            subs.append(sub)
            rects.append(rect)
        for s_ in leaf_streams:
            stream.wait_stream(s_)
        order = vrm.vr_kd_order(spec["shape_xyz"], spec["brick"], args.shard, cam["eye"])
        vrm.vr_composite_subimages(r.ctx, [subs[j] for j in order], np.stack([rects[j] for j in order]), out,
                                   stream)

    for k in range(args.warmup):
        draw(orbit_pose(2 * k + 1, 2 * max(args.warmup, 1)))   # spread over the orbit
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    r.reset_stats()
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        gpu_id = local
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    with ClockSampler(gpu_id) as clocks:
        torch.cuda.synchronize()
        evs[0].record(stream)
        for k in range(args.steps):
            frame(k)
            evs[k + 1].record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    st = r.stats()
    elapsed_ms = evs[0].elapsed_time(evs[-1])
    frame_ms = [evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)]
    # the root fold of --shard is one more launch per frame
    fold_launches = args.steps if args.shard > 1 else 0
    elapsed_ms, (samples, frames, launches) = job_totals(
        dist, elapsed_ms, [st["samples"], args.steps, st["launches"] + fold_launches], "cuda")

    # the paper's timing protocol (Section 3.1: each pose rendered repeatedly, its
    # median frame time kept, the 75th percentile over poses as the estimate),
    # after the timed region: every pose of this rank's orbit, repeated
    protocol = None
    if args.protocol_repeats > 0 and args.shard <= 1:
        per_pose = []
        for cam in my_poses:
            draw(cam)                                  # warm the pose's plan buffers
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.protocol_repeats + 1)]
            ev[0].record(stream)
            for k in range(args.protocol_repeats):
                draw(cam)
                ev[k + 1].record(stream)
            ev[-1].synchronize()
            per_pose.append(float(np.median([ev[k].elapsed_time(ev[k + 1]) for k in range(args.protocol_repeats)])))
        med = np.asarray(per_pose)
        protocol = {"repeats_per_pose": args.protocol_repeats, "poses": len(per_pose),
                    "rule": "per pose the median of the repeated frames; over the orbit the mean fps of those "
                            "medians and the 75th percentile of the median frame times",
                    "mean_fps": float(np.mean(1e3 / med)), "frame_ms_p75": float(np.percentile(med, 75)),
                    "frame_ms_median": float(np.median(med)), "frame_ms_max": float(med.max())}

    # end to end: host output buffer, copies inside the timed region
    e2e = None
    if args.e2e_steps > 0 and args.shard <= 1:
        # (1) synchronous: each call returns with its image in host memory;
        # (2) pipelined (VR_OPT_HOST_OUTPUT_ASYNC): each call enqueues its image's
        #     copy into one of two page-locked buffers and returns, the host plans
        #     the next frame meanwhile; one synchronise ends the timed region, so
        #     every image is in host memory inside it
        hosts = [torch.empty((H, W, 4), dtype=torch.float32, pin_memory=True).numpy() for _ in range(2)]
        runs = {}
        for mode in ("sync", "async"):
            r.set_option(vrmod.VR_OPT_HOST_OUTPUT_ASYNC, 1 if mode == "async" else 0)
            r.reset_stats()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for k in range(args.e2e_steps):
                r.set_camera(my_poses[orbit_index(k, args.e2e_steps, len(my_poses))])
                r.render(hosts[k % 2])
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            runs[mode] = (t1 - t0, r.stats())
        r.set_option(vrmod.VR_OPT_HOST_OUTPUT_ASYNC, 0)
        e2e_t, se = runs["async"]
        sync_t, _ = runs["sync"]
        e2e_t, (e2e_samples,) = job_totals(dist, e2e_t, [se["samples"]], "cuda")
        sync_t, _ = job_totals(dist, sync_t, [0], "cuda")
        e2e = {"value": e2e_samples / e2e_t, "unit": UNIT,
               "h2d_bytes_per_step": se["h2d_bytes"] // max(se["frames"], 1),
               "d2h_bytes_per_step": se["d2h_bytes"] // max(se["frames"], 1),
               "steps": args.e2e_steps,
               "fps": args.e2e_steps * (world if dist else 1) / e2e_t,
               "mode": "vr_render into page-locked host buffers (two, alternating) with VR_OPT_HOST_OUTPUT_ASYNC: "
                       "frames pipelined, one synchronise at the end of the timed region",
               "fps_synchronous": args.e2e_steps * (world if dist else 1) / sync_t}

    if rank != 0:
        r.close()
        if dist:
            dist.destroy_process_group()
        return

    def render_pose(cam, pix):
        """RGBA of pixels pix (flat indices) of the frame at pose cam."""
        draw(cam)
        return out.view(-1, 4)[torch.from_numpy(pix).cuda()].cpu().numpy()

    per_frame = max(st["frames"], 1) if args.shard <= 1 else args.steps   # stats count leaf renders
    peak, peak_kind = peaks()
    avg_march_ms = st["march_ms"] / max(st["frames"], 1)
    bytes_per_launch = st["touched_bytes"] / max(st["frames"], 1)
    achieved = bytes_per_launch / (avg_march_ms * 1e-3) / 1e9
    kname = {"tma": "march_tma_kernel", "direct": "march_kernel", "tex": "march_tex_kernel",
             "auto": "march_tex_kernel" if st["chunks_staged"] == 0 else "march_tma_kernel"}[args.kernel]
    roofline = {"bound": "hbm", "kernel": kname,
                "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak,
                # recorded for the fixed-step emission-absorption march of each storage
                "traffic": None if (args.mip or args.dynamic_step or args.ooc or args.width or args.height
                                    or args.tf != "a" or args.config != "hi")
                else recorded_traffic(kname, spec["name"] + ("" if args.precision == "f32" else "_" + args.precision)),
                "peak_kind": peak_kind,
                "algorithmic_bytes_per_launch": bytes_per_launch,
                "avg_launch_ms": avg_march_ms,
                "frame_bytes_per_step": bytes_per_launch + W * H * 16,
                "frame_frac": (bytes_per_launch + W * H * 16) / (elapsed_ms / args.steps * 1e-3) / 1e9 / peak}

    # secondary (ALU) roofline: lane instructions per second during the march
    # against the issue peak, 128 lanes per SM per cycle at the sampled SM clock
    ips = recorded_inst_per_sample(kname, spec["name"] + ("" if args.precision == "f32"
                                                         else "_" + args.precision))
    roofline_alu = None
    if ips and not args.mip and not args.dynamic_step:
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        mhz = clocks.summary().get("sm_mhz") or 0.0
        if mhz:
            alu_peak = sms * 128 * mhz * 1e6
            alu_ach = samples / max(frames, 1) * ips / (avg_march_ms * 1e-3)
            roofline_alu = {"bound": "alu", "kernel": kname, "achieved": alu_ach / 1e12, "peak": alu_peak / 1e12,
                            "unit": "T lane-instructions/s", "frac": alu_ach / alu_peak,
                            "thread_instructions_per_sample": ips,
                            "peak_kind": f"{sms} SMs x 128 lanes x median SM clock under load ({mhz:.0f} MHz)"}

    cpu = quality = None
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        regions = None
        if args.shard > 1:
            nb = [(n - 1 + b - 1) // b for n, b in zip(spec["shape_xyz"], spec["brick"])]
            ids = np.arange(nb[0] * nb[1] * nb[2])
            idx = np.stack([ids % nb[0], (ids // nb[0]) % nb[1], ids // (nb[0] * nb[1])], axis=1)
            regions = np.zeros(len(ids), dtype=np.int32)
            for j, lf in enumerate(leaves):
                regions[((idx >= lf[:3]) & (idx < lf[3:])).all(axis=1)] = j
        rate, secs, n_crops, crops = oracle_rate(cube, tf, poses, spec["brick"], args.cpu_seconds, keep=True,
                                                 regions=regions, step_mode=1 if args.dynamic_step else 0,
                                                 mode="mip" if args.mip else "ea")
        cpu = {"value": rate, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
               "sample": f"{n_crops} centre crops of 64x64 pixels on successive orbit poses, "
                         f"{secs:.1f} s of FP64 CPU work"}
        # the GPU image's error on the same crops (per-pixel error, PSNR)
        quality = image_quality(render_pose, crops)

    value = samples / (elapsed_ms * 1e-3)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": desc, "cube_xyz": list(spec["shape_xyz"]),
                       "brick": list(spec["brick"]), "image": [W, H], "step": 0.5,
                       "tf": args.tf.upper(), "term_alpha": 0.99,
                       "step_mode": "dynamic (step along the dominant axis)" if args.dynamic_step else "fixed",
                       "mode": "MIP + colour map" if args.mip else "emission-absorption",
                       "tex_slab_layers": args.tex_slab_layers or "device limit",
                       "storage": {"f32": "FP32", "f16": "FP16",
                                   "f8": "FP8 E4M3, per-brick absmax/448 scale"}[args.precision],
                       "residency": ("out-of-core: pinned host brick store, device brick cache of "
                                     + (f"{args.budget_gib:g} GiB" if args.budget_gib > 0 else "every brick")
                                     if args.ooc else "in-core: cube resident in HBM"),
                       "l2": ("inputs larger than L2, no flush" if spec["name"] != "tiny"
                              else "tiny cube fits in L2 (not a bench line)"),
                       "parallelism": f"replicas x{world}: orbit poses split across ranks"
                                      + (f"; each frame as {args.shard} virtual ranks (k-d leaves) on one GPU"
                                         if args.shard > 1 else "")},
            "fps": frames / (elapsed_ms * 1e-3),
            "orbit": {"poses": len(poses), "timed_poses": min(args.steps, len(my_poses)),
                      "rule": "timed frame k renders pose floor(k * poses / steps) (evenly spaced over "
                              "the orbit; each pose once when steps is a multiple of the pose count)",
                      "mean_fps": frames / (elapsed_ms * 1e-3),
                      "frame_ms_p75": float(np.percentile(frame_ms, 75))},
            "paper_protocol": protocol,
            "frame_ms_p50": float(np.percentile(frame_ms, 50)),
            "frame_ms_p75": float(np.percentile(frame_ms, 75)),
            "samples_per_frame": samples / max(frames, 1),
            "bricks_rendered_per_frame": st["bricks_rendered"] / per_frame,
            "bricks_skipped_per_frame": st["bricks_skipped"] / per_frame,
            "plan_ms_per_frame": st["plan_ms"] / per_frame,
            "composite_ms_per_frame": st["composite_ms"] / per_frame,
            "roofline": roofline, "roofline_alu": roofline_alu, "cpu_baseline": cpu, "e2e": e2e,
            "quality": quality,
            "march_kernel": args.kernel,
            "chunks_staged_per_frame": st["chunks_staged"] / per_frame,
            "chunks_direct_per_frame": st["chunks_direct"] / per_frame,
            "gpu_launches": launches, "clocks": clocks.summary(),
            "load_and_brick_s": load_s,
            "ooc": ({"bricks_uploaded_per_frame": st["bricks_uploaded"] / per_frame,
                     "bricks_cached_per_frame": st["bricks_cached"] / per_frame,
                     "upload_gb_per_s": (st["h2d_bytes"] / (elapsed_ms * 1e-3) / 1e9)}
                    if args.ooc else None),
            "device_errors": st["device_errors"]}
    print(json.dumps(line), flush=True)
    r.close()
    if dist:
        dist.destroy_process_group()


def tf_floor(tf):
    """The largest value below which the transfer function's opacity is zero
    (its first control point with nonzero opacity, or the one before it)."""
    tf = np.asarray(tf, dtype=np.float64).reshape(-1, 5)
    first = int(np.argmax(tf[:, 4] > 0))
    return float(tf[max(first - 1, 0), 0]) if tf[first, 4] > 0 else float(tf[-1, 0])


def run_learned(args):
    """Learned brick codec on the workload's cube: per brick an 8^3 x 16 latent grid
    and one shared MLP (28 inputs, two hidden layers of 64, SiLU) trained on the
    GPU by the tensor-core kernels on voxels clipped below the transfer
    function's transparent floor; frames rendered from bricks decoded into the
    device cache; PSNR against the plain (in-core FP32) render of the same poses."""
    import torch

    from paper_1205_0282_gb300 import vr as vrm

    torch.cuda.set_device(0)
    spec, tf, poses, desc = workload(args)
    cube = make_cube(spec)
    shape = spec["shape_xyz"]
    brick = (args.codec_brick,) * 3 if args.codec_brick else spec["brick"]
    nb = int(np.prod([(n - 1 + b - 1) // b for n, b in zip(shape, brick)]))
    dcube = torch.from_numpy(cube).cuda()
    W, H = spec["width"], spec["height"]
    q = max(1, len(poses) // args.psnr_poses)
    psnr_poses = poses[::q][:args.psnr_poses]
    # plain reference images (in-core, FP32 texture path, the same bricking)
    plain = []
    with vrm.VolumeRenderer(0) as r:
        r.load_cube(dcube)
        r.brick(*brick)
        r.set_transfer_function(tf)
        for cam in psnr_poses:
            r.set_camera(cam)
            plain.append(r.render().cpu().numpy().astype(np.float64))
    # train
    floor = tf_floor(tf)
    codec = vrm.Codec(nb, brick)
    rng = np.random.default_rng(3)
    H_, K_ = vrm.Codec.HIDDEN, vrm.Codec.K_IN
    W1 = rng.uniform(-1, 1, (H_, K_)) / np.sqrt(28.0)
    W1[:, 28:] = 0.0
    params = {"W1": W1, "b1": np.zeros(H_), "W2": rng.uniform(-1, 1, (H_, H_)) / np.sqrt(H_),
              "b2": np.zeros(H_), "w3": rng.uniform(-1, 1, H_) / np.sqrt(H_), "b3": np.zeros(1)}
    lat = rng.normal(0.0, 0.1, (nb, 8, 8, 8, 16))
    codec.set_params(codec.pack(params, lat), np.zeros(nb), np.ones(nb))
    codec.fit_stats(dcube, floor)
    th, m, s = codec.get_params()
    codec.set_params(th, m, s)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    chunk = 250
    losses = []
    done = 0
    while done < args.train_steps:
        k = min(chunk, args.train_steps - done)
        lr = args.train_lr * (0.1 if done >= 0.8 * args.train_steps else 1.0)
        losses.append(codec.train(dcube, k, args.train_batch, lr, seed=1000 + done, active_frac=args.active_frac))
        done += k
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    # decode throughput: every brick once (tensor-core MLP at every voxel)
    V = (brick[0] + 1) * (brick[1] + 1) * (brick[2] + 1)
    ids = torch.arange(nb, dtype=torch.int32, device="cuda")
    dec_batch = min(nb, 256)
    blocks = torch.empty(dec_batch * V, dtype=torch.float32, device="cuda")
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    codec.decode_bricks(ids[:dec_batch], blocks)      # warm-up
    ev0.record()
    for b0 in range(0, nb, dec_batch):
        codec.decode_bricks(ids[b0:b0 + dec_batch], blocks)
    ev1.record()
    torch.cuda.synchronize()
    dec_ms = ev0.elapsed_time(ev1)
    del blocks
    points = nb * V
    mac_tensor = 32 * 64 + 64 * 64           # per point, on the tensor cores
    dec_tflops = points * 2 * mac_tensor / (dec_ms * 1e-3) / 1e12
    del dcube
    torch.cuda.empty_cache()

    fb = {}

    def render_learned(budget_gib, steps):
        r = vrm.VolumeRenderer(0)
        r.load_cube_codec(codec, shape)
        r.set_option(vrm.VR_OPT_OOC_MARCH, OOC_MARCH[args.ooc_march])
        if budget_gib > 0:
            r.set_option(vrm.VR_OPT_DEVICE_BUDGET, int(budget_gib * 2 ** 30))
        if args.fallback_bound is not None:
            r.set_codec_fallback(cube, args.fallback_bound, floor)
        t_scan = time.perf_counter()
        r.brick(*brick)
        if args.fallback_bound is not None:
            err, n_plain = r.codec_brick_errors()
            fb.update({"bound": args.fallback_bound, "bricks_plain": n_plain, "bricks": nb,
                       "pinned_gib": n_plain * V * 4 / 2 ** 30, "scan_and_store_s": time.perf_counter() - t_scan,
                       "brick_error_p50_p90_max": [float(np.percentile(err, 50)), float(np.percentile(err, 90)),
                                                   float(err.max())]})
        r.set_transfer_function(tf)
        imgs = []
        for cam in psnr_poses:
            r.set_camera(cam)
            imgs.append(r.render().cpu().numpy().astype(np.float64))
        out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
        for k in range(args.warmup):
            r.set_camera(poses[k % len(poses)])
            r.render(out)
        torch.cuda.synchronize()
        r.reset_stats()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for k in range(steps):
            r.set_camera(poses[k % len(poses)])
            r.render(out)
        e1.record()
        torch.cuda.synchronize()
        st = r.stats()
        r.close()
        ms = e0.elapsed_time(e1)
        return imgs, st, ms

    gpu_id = "GPU-" + str(torch.cuda.get_device_properties(0).uuid)
    with ClockSampler(gpu_id) as clocks:
        imgs, st, ms = render_learned(args.budget_gib, args.steps)
    mse = float(np.mean([np.mean((a - b) ** 2) for a, b in zip(imgs, plain)]))
    psnr = 10 * np.log10(1.0 / mse) if mse > 0 else None
    maxerr = float(max(np.abs(a - b).max() for a, b in zip(imgs, plain)))
    codec.close()
    frames = args.steps
    line = {"metric": METRIC, "value": st["samples"] / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / frames, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (decoder bf16 x bf16 -> f32)", "data": "synthetic",
            "config": {"workload": desc, "codec_brick": list(brick),
                       "form": "learned: 8^3 x 16 BF16 latents per brick + shared MLP "
                       "(28 -> 64 -> 64 -> 1, SiLU), bricks decoded on the tensor cores into the device cache",
                       "device_budget_gib": args.budget_gib or "every brick",
                       "train": {"steps": args.train_steps, "batch": args.train_batch, "lr": args.train_lr,
                                 "floor": floor, "active_frac": args.active_frac}},
            "fps": frames / (ms * 1e-3),
            "learned": {"psnr_db_vs_plain": psnr, "max_abs_vs_plain": maxerr, "psnr_poses": len(psnr_poses),
                        "train_s": train_s, "loss_trace": losses,
                        "latent_bytes": nb * 8 * 8 * 8 * 16 * 2, "cube_bytes": int(cube.nbytes),
                        "compression": cube.nbytes / (nb * 8 * 8 * 8 * 16 * 2),
                        "decode_ms_all_bricks": dec_ms, "decode_points_per_s": points / (dec_ms * 1e-3),
                        "decode_tensor_tflops": dec_tflops,
                        "bricks_decoded_per_frame": st["bricks_uploaded"] / max(st["frames"], 1),
                        "bricks_cached_per_frame": st["bricks_cached"] / max(st["frames"], 1),
                        "h2d_gb_per_frame": st["h2d_bytes"] / max(st["frames"], 1) / 1e9,
                        "fallback": fb or None},
            "roofline": {"bound": "tensor", "kernel": "codec_kernel (decode)", "achieved": dec_tflops,
                         "peak": json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"]
                         if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 1900.0,
                         "unit": "TFLOP/s", "traffic": None},
            "gpu_launches": st["launches"], "clocks": clocks.summary(), "cpu_baseline": None, "e2e": None}
    line["roofline"]["frac"] = line["roofline"]["achieved"] / line["roofline"]["peak"]
    print(json.dumps(line), flush=True)


OOC_MARCH = {"direct": 0, "tex": 1, "auto": 2, "texz": 3, "texxz": 4}


def xl_slabs(nbz: int, layers: int):
    """Brick-layer ranges [bz0, bz1) of the training slabs, in order."""
    return [(b, min(b + layers, nbz)) for b in range(0, nbz, layers)]


def spread(items, k: int):
    """k items evenly spaced over the list (all of them when k >= len)."""
    if k >= len(items):
        return list(items)
    return [items[(i * len(items)) // k + len(items) // (2 * k)] for i in range(k)]


def run_learned_xl(args):
    """The learned form on the 4096x4096x3200 (~200 GiB) cube, which never exists
    whole: its bricks are generated on request by the seeded block source.  The
    codec is trained slab by slab (a slab of brick layers generated on the host
    into pinned memory and copied to the device): first the shared decoder with
    the latents of a few slabs, then every slab's latents fitted to the fixed
    decoder.  Learned (latents on the device, fallback bricks' plain blocks in
    pinned host memory) and plain out-of-core (every missing brick from the
    provider) render the same orbit poses at each device budget; PSNR of the
    learned frames against the plain ones."""
    import torch

    from paper_1205_0282_gb300 import vr as vrm

    torch.cuda.set_device(0)
    k = max(1, args.xl_scale)
    spec = dict(synth.XL)
    shape = tuple(n // k for n in spec["shape_xyz"])
    n_line, n_cont = spec["n_line"] // k ** 3, max(1, spec["n_cont"] // k ** 3)
    src = synth.BlockSource(shape, spec["seed"], synth.hi_sources(spec["seed"], shape, n_line, n_cont))
    brick = (args.codec_brick or 64,) * 3
    tf = synth.tf_hi_a() if args.tf == "a" else synth.tf_hi_b()
    floor = tf_floor(tf)
    W = args.width or spec["width"]
    H = args.height or spec["height"]
    poses = synth.orbit(shape, 60, 15.0, W, H)
    nbs = [(n - 2 + b) // b for n, b in zip(shape, brick)]
    nb = int(np.prod(nbs))
    V = (brick[0] + 1) * (brick[1] + 1) * (brick[2] + 1)
    cube_bytes = 4 * int(np.prod(shape))
    bound = 2.0 if args.fallback_bound is None else args.fallback_bound
    desc = (f"XL cube {shape[0]}x{shape[1]}x{shape[2]} f32 ({cube_bytes / 2 ** 30:.0f} GiB; noise + {n_line} line + "
            f"{n_cont} continuum sources), generated brick by brick on request, {brick[0]}^3 bricks, {W}x{H}, "
            f"step 0.5, 16-point TF-{args.tf.upper()}, tau 0.99, 60-pose orbit")

    # ---- codec training, slab by slab
    codec = vrm.Codec(nb, brick)
    rng = np.random.default_rng(3)
    H_, K_ = vrm.Codec.HIDDEN, vrm.Codec.K_IN
    W1 = rng.uniform(-1, 1, (H_, K_)) / np.sqrt(28.0)
    W1[:, 28:] = 0.0
    params = {"W1": W1, "b1": np.zeros(H_), "W2": rng.uniform(-1, 1, (H_, H_)) / np.sqrt(H_),
              "b2": np.zeros(H_), "w3": rng.uniform(-1, 1, H_) / np.sqrt(H_), "b3": np.zeros(1)}
    lat = rng.standard_normal((nb, 8, 8, 8, 16), dtype=np.float32) * np.float32(0.1)
    codec.set_params(codec.pack(params, lat), np.zeros(nb), np.ones(nb))
    del lat
    slabs = xl_slabs(nbs[2], args.xl_slab_layers)
    max_planes = min(args.xl_slab_layers * brick[2], shape[2] - 1) + 1
    host = torch.empty((max_planes, shape[1], shape[0]), dtype=torch.float32, pin_memory=True)
    dev = torch.empty((max_planes, shape[1], shape[0]), dtype=torch.float32, device="cuda")
    t_gen = 0.0

    def load(bz0, bz1):
        nonlocal t_gen
        z0, z1 = bz0 * brick[2], min(bz1 * brick[2], shape[2] - 1)
        t = time.perf_counter()
        src.fill_planes(host.data_ptr(), z0, z1)
        t_gen += time.perf_counter() - t
        d = dev[: z1 - z0 + 1]
        d.copy_(host[: z1 - z0 + 1])
        return d

    t0 = time.perf_counter()
    losses_a, losses_b = [], []
    fitted = set()
    for i, (bz0, bz1) in enumerate(spread(slabs, args.xl_decoder_slabs)):
        d = load(bz0, bz1)
        codec.fit_stats_slab(d, shape, bz0, bz1, floor)
        fitted.add((bz0, bz1))
        done = 0
        while done < args.train_steps:
            n = min(250, args.train_steps - done)
            lr = args.train_lr * (0.1 if done >= 0.8 * args.train_steps else 1.0)
            losses_a.append(codec.train_slab(d, shape, bz0, bz1, n, args.train_batch, lr, lr,
                                             seed=7919 * i + done))
            done += n
    for j, (bz0, bz1) in enumerate(slabs):
        d = load(bz0, bz1)
        codec.fit_stats_slab(d, shape, bz0, bz1, floor)
        done = 0
        while done < args.xl_slab_steps:
            n = min(500, args.xl_slab_steps - done)
            lr = args.train_lr * (0.1 if done >= 0.8 * args.xl_slab_steps else 1.0)
            last = codec.train_slab(d, shape, bz0, bz1, n, args.train_batch, lr, 0.0, seed=104729 + 7919 * j + done)
            done += n
        losses_b.append(last)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    del host, dev, d
    torch.cuda.empty_cache()

    # ---- both forms at each budget
    budgets = [float(b) for b in args.xl_budgets_gib.split(",") if b.strip()]
    frame_poses = [poses[(i * len(poses)) // args.xl_frames] for i in range(args.xl_frames)]
    results = []
    learned_line = None

    def timed(r, cam, out):
        r.set_camera(cam)
        torch.cuda.synchronize()
        t = time.perf_counter()
        r.render(out)
        torch.cuda.synchronize()
        return time.perf_counter() - t

    gpu_id = "GPU-" + str(torch.cuda.get_device_properties(0).uuid)
    out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
    with ClockSampler(gpu_id) as clocks:
        for budget in budgets:
            row = {"budget_gib": budget}
            for form in ("plain", "learned"):
                r = vrm.VolumeRenderer(0)
                if form == "plain":
                    r.load_cube_provider(src, shape)
                else:
                    r.load_cube_codec(codec, shape)
                    r.set_codec_fallback_provider(src, bound, floor)
                r.set_option(vrm.VR_OPT_DEVICE_BUDGET, int(budget * 2 ** 30))
                r.set_option(vrm.VR_OPT_OOC_MARCH, OOC_MARCH[args.ooc_march])
                t = time.perf_counter()
                r.brick(*brick)
                setup_s = time.perf_counter() - t
                r.set_transfer_function(tf)
                info = {"setup_s": setup_s}
                if form == "learned":
                    err, n_plain = r.codec_brick_errors()
                    info.update(bricks_plain=n_plain, bricks=nb, pinned_gib=n_plain * V * 4 / 2 ** 30,
                                bound=bound)
                cold = timed(r, frame_poses[0], out)
                r.reset_stats()
                secs, imgs = [], []
                for cam in frame_poses:
                    secs.append(timed(r, cam, out))
                    imgs.append(out.cpu().numpy())
                st = r.stats()
                # the same poses back to back (repeated to at least 16 frames, so that
                # the first frame's planning, which nothing overlaps, weighs little),
                # one synchronisation at the end: the planning of a frame overlaps the
                # device work of the ones before it
                piped = frame_poses * max(1, -(-16 // len(frame_poses)))
                torch.cuda.synchronize()
                t = time.perf_counter()
                for cam in piped:
                    r.set_camera(cam)
                    r.render(out)
                torch.cuda.synchronize()
                fps_pipelined = len(piped) / (time.perf_counter() - t)
                r.close()
                info.update(cold_first_frame_s=cold, frame_s=secs, fps=len(secs) / sum(secs),
                            fps_pipelined=fps_pipelined, frames_pipelined=len(piped),
                            samples_per_s=st["samples"] / sum(secs),
                            bricks_rendered_per_frame=st["bricks_rendered"] / max(st["frames"], 1),
                            bricks_filled_per_frame=st["bricks_uploaded"] / max(st["frames"], 1),
                            plan_ms_per_frame=st["plan_ms"] / max(st["frames"], 1),
                            items_per_frame=st["items"] / max(st["frames"], 1),
                            launches=st["launches"], device_errors=st["device_errors"])
                row[form] = info
                row[form + "_imgs"] = imgs
            a = np.stack(row.pop("learned_imgs")).astype(np.float64)
            b = np.stack(row.pop("plain_imgs")).astype(np.float64)
            mse = float(np.mean((a - b) ** 2))
            row["psnr_db_learned_vs_plain"] = 10 * np.log10(1.0 / mse) if mse > 0 else None
            row["max_abs_learned_vs_plain"] = float(np.abs(a - b).max())
            results.append(row)
            print(json.dumps({"xl_budget": row}), flush=True)
            if learned_line is None:
                learned_line = row
    codec.close()
    L = learned_line["learned"]
    line = {"metric": METRIC, "value": L["samples_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.xl_frames,
            "warmup": 1, "ms_per_step": 1e3 / L["fps"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (decoder bf16 x bf16 -> f32)", "data": "synthetic",
            "config": {"workload": desc, "codec_brick": list(brick),
                       "form": "learned: 8^3 x 16 BF16 latents per brick + shared MLP (28 -> 64 -> 64 -> 1, SiLU), "
                               "bricks over the error bound from pinned plain blocks; plain: out-of-core, every "
                               "missing brick generated on request (no host copy of the cube)",
                       "train": {"decoder_slabs": args.xl_decoder_slabs, "decoder_steps_per_slab": args.train_steps,
                                 "latent_steps_per_slab": args.xl_slab_steps, "slab_layers": args.xl_slab_layers,
                                 "batch": args.train_batch, "lr": args.train_lr, "floor": floor},
                       "ooc_march": args.ooc_march,
                       "timing": "wall clock per frame with a device synchronise on both sides (host generation "
                                 "and uploads included); the first frame after vr_brick fills the cache (cold)"},
            "fps": L["fps"],
            "xl": {"cube_bytes": cube_bytes, "latent_bytes": nb * 8 * 8 * 8 * 16 * 2, "bricks": nb,
                   "train_s": train_s, "host_generation_s_in_training": t_gen,
                   "loss_decoder_last": losses_a[-1] if losses_a else None,
                   "loss_latents_last_per_slab": losses_b,
                   "budgets": results},
            "gpu_launches": L["launches"], "clocks": clocks.summary(), "roofline": None, "cpu_baseline": None,
            "e2e": None}
    print(json.dumps(line), flush=True)


SERVE_RESOLUTIONS = [(512, 512), (1280, 720), (1920, 1080), (3840, 2160)]


def run_serve(args):
    """Serving workload: requests arrive as a Poisson process (mean ``--rate`` per
    second) for ``--serve-seconds``; each asks for an orbit pose at a resolution
    drawn uniformly from 512x512, 1280x720, 1920x1080 and 3840x2160, and one in
    ten switches the transfer function (TF-A <-> TF-B).  The cube is resident
    (FP16 storage unless --precision says otherwise).  Latency = completion time
    minus arrival time of each request."""
    import threading

    import torch
    from paper_1205_0282_gb300 import vr as vrm

    torch.cuda.set_device(0)
    spec, tf, poses, desc = workload(args)
    cube = make_cube(spec)
    r = vrm.VolumeRenderer(0)
    dcube = torch.from_numpy(cube).cuda()
    r.load_cube(dcube)
    del dcube
    torch.cuda.empty_cache()
    r.brick(*spec["brick"])
    tfs = [synth.tf_hi_a(), synth.tf_hi_b()]
    r.set_transfer_function(tfs[0])
    r.set_camera(poses[0])
    prec = {"f32": vrm.VR_PRECISION_F32, "f16": vrm.VR_PRECISION_F16, "f8": vrm.VR_PRECISION_F8}[
        args.precision if args.precision != "f32" else "f16"]
    r.set_option(vrm.VR_OPT_PRECISION, prec)
    r.render()   # builds the layered copies
    torch.cuda.synchronize()

    rng = np.random.default_rng(7)
    n = int(rng.poisson(args.rate * args.serve_seconds))
    arrivals = np.sort(rng.uniform(0.0, args.serve_seconds, n))
    res = [SERVE_RESOLUTIONS[k] for k in rng.integers(0, len(SERVE_RESOLUTIONS), n)]
    tf_switch = rng.uniform(size=n) < 0.1
    # output buffers: enough that none is reused while its request can be in flight
    pool = {wh: [torch.empty((wh[1], wh[0], 4), dtype=torch.float32, device="cuda") for _ in range(48)]
            for wh in SERVE_RESOLUTIONS}
    used = {wh: 0 for wh in SERVE_RESOLUTIONS}

    srv = vrm.Server(r, int(args.arena_gib * 2 ** 30), args.max_batch)
    # warm the loop up (untimed): one request per resolution
    for wh in SERVE_RESOLUTIONS:
        cam = dict(poses[0], width=wh[0], height=wh[1])
        srv.wait(srv.submit(cam, pool[wh][0]), 120.0)
    st0 = srv.stats()
    tickets = [None] * n
    lat = [None] * n
    done = threading.Event()

    def waiter():
        for k in range(n):
            while tickets[k] is None:
                time.sleep(0.0002)
            lat[k] = srv.wait(tickets[k], 300.0)
        done.set()

    th = threading.Thread(target=waiter)
    th.start()
    tf_cur = 0
    clocks_id = "GPU-" + str(torch.cuda.get_device_properties(0).uuid)
    with ClockSampler(clocks_id) as clocks:
        t0 = time.perf_counter()
        for k in range(n):
            dt = t0 + arrivals[k] - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            wh = res[k]
            cam = dict(poses[k % len(poses)], width=wh[0], height=wh[1])
            buf = pool[wh][used[wh] % len(pool[wh])]
            used[wh] += 1
            new_tf = None
            if tf_switch[k]:
                tf_cur ^= 1
                new_tf = tfs[tf_cur]
            tickets[k] = srv.submit(cam, buf, new_tf)
        done.wait()
        t_end = time.perf_counter()
    th.join()
    st = srv.stats()
    srv.close()
    r.close()
    wall = t_end - t0
    lat = np.array(lat)
    frames = st["completed"] - st0["completed"]
    samples = st["samples"] - st0["samples"]
    batches = st["batches"] - st0["batches"]
    line = {"metric": METRIC, "value": samples / wall, "unit": UNIT, "n_gpus": 1, "steps": n,
            "warmup": len(SERVE_RESOLUTIONS), "ms_per_step": 1e3 * wall / max(n, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": desc.split(", image overridden")[0] + "; serving: Poisson arrivals "
                       f"{args.rate:g}/s for {args.serve_seconds:g} s, resolutions uniform over "
                       "512x512/1280x720/1920x1080/3840x2160, 10% transfer-function switches (TF-A/TF-B)",
                       "storage": {"f32": "FP16", "f16": "FP16", "f8": "FP8 E4M3, per-brick scale"}[args.precision],
                       "arena_gib": args.arena_gib, "max_batch": args.max_batch,
                       "l2": "inputs larger than L2, no flush"},
            "serving": {"requests": n, "completed": frames, "failed": st["failed"] - st0["failed"],
                        "fps": frames / wall, "wall_s": wall,
                        "latency_ms_p50": float(np.percentile(lat, 50)),
                        "latency_ms_p99": float(np.percentile(lat, 99)),
                        "latency_ms_mean": float(lat.mean()), "latency_ms_max": float(lat.max()),
                        "batches": batches, "mean_batch": (frames / batches) if batches else None},
            "gpu_launches": 2 * batches, "clocks": clocks.summary(), "roofline": None, "cpu_baseline": None,
            "e2e": None}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.serve and args.impl == "ours":
        return run_serve(args)
    if args.learned and args.impl == "ours":
        return run_learned_xl(args) if args.config == "xl" else run_learned(args)
    if args.config == "xl":
        raise SystemExit("--config xl runs with --learned (the cube never exists whole in host or device memory)")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
