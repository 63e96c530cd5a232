#!/usr/bin/env python
"""Benchmark of the data-parallel volume rendering hot path on one GB300.

One step = one composited frame: the per-brick emission-absorption march of
all bricks plus the sort-last "over" composite, at the next of 8 orbit views.

Workload (default): 512^3 float32 volume (6-octave value noise + 16 Gaussian
blobs, seed 1) split into 36 bricks (4x3x3 grid), 1920x1080 perspective image
(60 degree field of view) orbiting the volume, step 0.5 voxel, early ray
termination at alpha 0.99, radix-k composite 4x3x3. Synthetic stand-in for the
paper's distributed data set (36 GPUs in the paper's run, one brick each).

value = executed ray samples per second over the timed frames (samples counted
per view in an untimed pass). Inputs (560 MB of bricks) exceed the 129 MB L2.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun each rank renders its own views of a replica of the volume
(weak scaling, no data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ray samples/s and composited frames/s at 1 GB300; % HBM roofline; vs FP64 oracle"
UNIT = "samples/s"
# FP32 operations the method performs per executed sample (position 8,
# trilinear reconstruction 30, classification 19, accumulation 8, termination
# test 1).
FLOPS_PER_SAMPLE = 66
FP32_LANES = 128  # FP32 lanes per SM (sm_100 family)
# kernel durations come from a separate pass after the timed region, with event
# pairs around every march and composite launch (they cost about 10 us per
# frame, so the timed region itself carries none): at least KT_FRAMES frames
KT_FRAMES = 64


def args_parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="paper",
                    choices=["paper", "small", "precision", "grad", "batch", "stream", "mesh"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--layout", default="quads", choices=["quads", "octets"],
                    help="batch workload: 16-bit cells as xy-quads or as octets (vr_set_cell_layout)")
    ap.add_argument("--split", default="views", choices=["views", "bricks"],
                    help="multi-GPU: replicas over views (weak scaling) or bricks as ranks with a radix-k "
                         "image exchange (strong scaling)")
    return ap.parse_args()


def shard_views(rank: int, world: int, n_views: int, n_frames: int):
    """View index of each frame a rank renders: rank r takes views r, r+N,
    r+2N, ... of the orbit (replicas of the volume over views, no data-path
    exchange)."""
    return [(rank + world * i) % n_views for i in range(n_frames)]


def reduce_job(ms: float, e2e_s: float, samples: float, world: int, device: str = "cuda"):
    """Whole-job numbers over ranks: the slowest rank's times, the sum of the
    samples."""
    if world <= 1:
        return ms, e2e_s, samples
    import torch
    import torch.distributed as dist
    mx = torch.tensor([ms, e2e_s], dtype=torch.float64, device=device)
    sm = torch.tensor([samples], dtype=torch.float64, device=device)
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(mx[1]), float(sm[0])


def source_key(sources) -> str:
    """First 16 hex digits of the sha256 of the kernel sources with comments and
    whitespace removed (a recorded measurement stays valid across comment edits)."""
    import hashlib
    import re
    csrc = os.path.join(ROOT, "paper_2501_01628_gb300", "csrc")
    h = hashlib.sha256()
    for f in sources:
        text = open(os.path.join(csrc, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        h.update(re.sub(r"\s+", "", text).encode())
    return h.hexdigest()[:16]


def recorded_value(field: str, summary: str = "march_paper_workload.md",
                   sources=("vr_kernels.cu", "vr_device.cuh", "vr_internal.h")):
    """A figure (`field: value` line) of a kernel's committed ncu summary, if
    the summary was taken on the current kernel code (else None)."""
    import re
    try:
        text = open(os.path.join(ROOT, "profiles", summary)).read()
        key = source_key(sources)
    except OSError:
        return None
    m = re.search(re.escape(field) + r":\s*([0-9.eE+]+)", text)
    k = re.search(r"kernel_source_key:\s*([0-9a-f]+)", text)
    if not m or not k or k.group(1) != key:
        return None
    return float(m.group(1))


def recorded_traffic(summary: str = "march_paper_workload.md",
                     sources=("vr_kernels.cu", "vr_device.cuh", "vr_internal.h")):
    """DRAM bytes per launch of a kernel from its committed ncu summary."""
    return recorded_value("traffic_bytes_per_launch", summary, sources)


MESH_SOURCES = ("vr_mesh.cu", "vr_mesh.h", "vr_device.cuh", "vr_internal.h")


def workload(name: str):
    import numpy as np
    from paper_2501_01628_gb300 import synth
    if name == "small":
        vol, tf = synth.small_blob_scene()
        cams = [synth.ortho_camera_z(256, 256)]
        return dict(name="small: 64^3 f32 blobs (8, seed 0), 2x2x2 bricks, 256x256 orthographic +z, "
                         "step 0.5 voxel, no early termination, direct composite",
                    vol=vol, tf=tf, part=dict(kind="grid", grid=(2, 2, 2)), cams=cams, step=0.5,
                    ert=1.0, schedule=(), grid=(2, 2, 2))
    vol, tf = synth.noise_blob_scene()
    cams = [synth.orbit_camera(1920, 1080, az) for az in synth.ORBIT_AZIMUTHS]
    return dict(name="paper-shaped: 512^3 f32 value noise (6 octaves) + 16 blobs (seed 1), 36 bricks "
                     "(4x3x3), 1920x1080 perspective 60 deg orbit (8 views), step 0.5 voxel, "
                     "early termination at alpha 0.99, radix-k composite 4x3x3",
                vol=vol, tf=tf, part=dict(kind="grid", grid=(4, 3, 3)), cams=cams, step=0.5,
                ert=0.99, schedule=(4, 3, 3), grid=(4, 3, 3))


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.path = tempfile.mktemp(prefix="clocks", suffix=".csv")
        self.proc = None
        self.dev = device_index

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "20"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[4:8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------
# CPU baseline: the FP64 oracle, as it stands, on the host cores
# --------------------------------------------------------------------------


def oracle_rate_1thread(wl, budget_s: float = 3.0):
    """Oracle samples/s on one host thread: centred 64x64 crops of successive
    views until about budget_s of host time is spent."""
    import oracle
    vol, tf = wl["vol"], wl["tf"]
    lo, hi = float(vol.min()), float(vol.max())
    boxes = oracle.grid_partition(vol.shape[::-1], wl["grid"])
    n = 0
    k = 0
    t = time.perf_counter()
    while time.perf_counter() - t < budget_s and k < 64:
        cam = wl["cams"][k % len(wl["cams"])]
        W, H = cam["width"], cam["height"]
        w, h = min(W, 64), min(H, 64)
        n += oracle.render(vol, boxes, tf, lo, hi, cam, wl["step"], wl["ert"],
                           crop=((W - w) // 2, (H - h) // 2, w, h), threads=1)["nsamples"]
        k += 1
    dt = time.perf_counter() - t
    return dict(value=n / dt, unit=UNIT, cores=1, kind="oracle",
                sample="%d centred 64x64 crops of successive views (%d samples, %.1f s, FP64, 1 thread)"
                       % (k, n, dt))


def oracle_rate(wl, budget_s: float = 12.0):
    """Oracle samples/s over whole frames of successive views, until about
    budget_s of host time is spent (every host core)."""
    import oracle
    vol, tf = wl["vol"], wl["tf"]
    lo, hi = float(vol.min()), float(vol.max())
    boxes = oracle.grid_partition(vol.shape[::-1], wl["grid"])
    cores = os.cpu_count() or 1
    n = 0
    frames = 0
    t = time.perf_counter()
    while time.perf_counter() - t < budget_s and frames < 64:
        cam = wl["cams"][frames % len(wl["cams"])]
        n += oracle.render(vol, boxes, tf, lo, hi, cam, wl["step"], wl["ert"], threads=cores)["nsamples"]
        frames += 1
    dt = time.perf_counter() - t
    W, H = wl["cams"][0]["width"], wl["cams"][0]["height"]
    return dict(value=n / dt, unit=UNIT, cores=cores, kind="oracle",
                frames_per_s=frames / dt,
                sample="%d full %dx%d frames of successive orbit views (%d samples, %.1f s, FP64, %d threads)"
                       % (frames, W, H, n, dt, cores)), n, dt


def run_reference(a):
    """The oracle as the reference arm: each step a bounded crop of the view."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    wl = workload(a.workload)
    vol, tf = wl["vol"], wl["tf"]
    lo, hi = float(vol.min()), float(vol.max())
    boxes = oracle.grid_partition(vol.shape[::-1], wl["grid"])
    cores = os.cpu_count() or 1
    crop = 48

    def step(i):
        cam = wl["cams"][i % len(wl["cams"])]
        W, H = cam["width"], cam["height"]
        w, h = min(W, crop), min(H, crop)
        r = oracle.render(vol, boxes, tf, lo, hi, cam, wl["step"], wl["ert"],
                          crop=((W - w) // 2, (H - h) // 2, w, h), threads=cores)
        return r["nsamples"]

    for i in range(a.warmup):
        step(i)
    t = time.perf_counter()
    n = sum(step(a.warmup + i) for i in range(a.steps))
    dt = time.perf_counter() - t
    v = n / dt
    line = dict(impl="reference", metric=METRIC, value=v, unit=UNIT, n_gpus=0, steps=a.steps,
                warmup=a.warmup, ms_per_step=dt / a.steps * 1e3, higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=wl["name"], sample="centred %dx%d crop per step" % (crop, crop)),
                cpu_baseline=dict(value=v, unit=UNIT, cores=cores, kind="oracle",
                                  sample="%d steps of a centred %dx%d crop, FP64, %d threads"
                                         % (a.steps, crop, crop, cores)),
                e2e=dict(value=v, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line))


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------


def run_ours(a):
    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    from paper_2501_01628_gb300 import vr

    wl = workload(a.workload)
    vol, tf = wl["vol"], wl["tf"]
    lo, hi = float(vol.min()), float(vol.max())
    cams = wl["cams"]
    ctx = vr.vr_create(local)
    v = vr.vr_volume_create(ctx, vol, "f32", wl["part"])
    vr.vr_set_transfer_function(ctx, tf, lo, hi)
    vr.vr_set_render_params(ctx, wl["step"], wl["ert"])
    vr.vr_set_composite_schedule(ctx, wl["schedule"])
    W, H = cams[0]["width"], cams[0]["height"]
    out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    # executed samples per view (untimed, counting launch variant)
    counts = []
    rect_px = []
    vr.vr_set_count_samples(ctx, True)
    for cam in cams:
        vr.vr_set_camera(ctx, cam)
        vr.vr_render_frame(ctx, v, out)
        counts.append(vr.vr_get_sample_count(ctx))
        _, rects = vr.vr_plan_view(vol.shape[::-1], wl["part"], cam)
        rect_px.append(int(sum(int(r[2]) * int(r[3]) for r in rects)))
    vr.vr_set_count_samples(ctx, False)
    views = shard_views(rank, world, len(cams), a.warmup + a.steps)

    # ray-packet shape: time one pass over the views per candidate, keep the fastest
    stream = torch.cuda.current_stream()
    tune = {}
    for pw in (4, 8, 16):
        vr.vr_set_packet_width(ctx, pw)
        for cam in cams:
            vr.vr_set_camera(ctx, cam)
            vr.vr_render_frame(ctx, v, out)
        t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0e.record(stream)
        for _ in range(2):
            for cam in cams:
                vr.vr_set_camera(ctx, cam)
                vr.vr_render_frame(ctx, v, out)
        t1e.record(stream)
        torch.cuda.synchronize()
        tune[pw] = t0e.elapsed_time(t1e) / (2 * len(cams))
    best_pw = min(tune, key=tune.get)
    vr.vr_set_packet_width(ctx, best_pw)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for i in range(a.warmup):
        vr.vr_set_camera(ctx, cams[views[i]])
        vr.vr_render_frame(ctx, v, out)
    torch.cuda.synchronize()

    # ---- device-resident timed region -----------------------------------
    timed_views = views[a.warmup:]
    clocks = ClockSampler(local)
    clocks.start()
    vr.vr_get_kernel_timing(ctx)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for vi in timed_views:
        vr.vr_set_camera(ctx, cams[vi])
        vr.vr_render_frame(ctx, v, out)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()

    # ---- per-kernel durations: a separate pass with event pairs on every launch
    vr.vr_set_kernel_timing(ctx, True)
    kt_frames = max(KT_FRAMES, len(timed_views))
    for i in range(kt_frames):  # the orbit views in turn
        vr.vr_set_camera(ctx, cams[i % len(cams)])
        vr.vr_render_frame(ctx, v, out)
    kt = vr.vr_get_kernel_timing(ctx)
    vr.vr_set_kernel_timing(ctx, False)

    # ---- the same frames without pipelining (one frame's march, then its
    # composite with one block per tile, then the next frame's march)
    vr.vr_set_frame_pipelining(ctx, False)
    for i in range(a.warmup):
        vr.vr_set_camera(ctx, cams[views[i]])
        vr.vr_render_frame(ctx, v, out)
    torch.cuda.synchronize()
    e0.record(stream)
    for vi in timed_views:
        vr.vr_set_camera(ctx, cams[vi])
        vr.vr_render_frame(ctx, v, out)
    e1.record(stream)
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1)
    vr.vr_set_frame_pipelining(ctx, True)

    # ---- end to end through the C ABI into pinned host images -------------
    # asynchronous host output: frame i's 33 MB copy (own copy stream, two
    # staging images) overlaps frame i+1's rendering; two host images in turn
    hosts = [torch.empty((H, W, 4), dtype=torch.float32).pin_memory() for _ in range(2)]
    vr.vr_set_host_output_async(ctx, True)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i, vi in enumerate(timed_views):
        vr.vr_set_camera(ctx, cams[vi])
        vr.vr_render_frame(ctx, v, hosts[i & 1])
    vr.vr_sync(ctx)  # every image is in host memory
    e2e_s = time.perf_counter() - t0
    vr.vr_set_host_output_async(ctx, False)
    barrier()

    samples = float(sum(counts[vi] for vi in timed_views))
    ms, e2e_s, samples = reduce_job(ms, e2e_s, samples, world)

    # precision form on the same workload: bfloat16 brick storage, FP32
    # accumulation; frame time against the f32 frames above, and the largest
    # image difference to the f32 render of one view
    forms = None
    if world == 1 and a.workload == "paper":
        vb = vr.vr_volume_create(ctx, vol, "bf16", wl["part"])
        vr.vr_set_camera(ctx, cams[0])
        vr.vr_render_frame(ctx, v, out)
        ref0 = out.clone()
        for i in range(a.warmup):
            vr.vr_set_camera(ctx, cams[views[i]])
            vr.vr_render_frame(ctx, vb, out)
        nb16 = min(len(timed_views), 400)
        torch.cuda.synchronize()
        e0.record(stream)
        for vi in timed_views[:nb16]:
            vr.vr_set_camera(ctx, cams[vi])
            vr.vr_render_frame(ctx, vb, out)
        e1.record(stream)
        torch.cuda.synchronize()
        bms = e0.elapsed_time(e1) / nb16
        vr.vr_set_camera(ctx, cams[0])
        vr.vr_render_frame(ctx, vb, out)
        diff = (out - ref0).abs()
        fms = ms / len(timed_views)
        forms = dict(bf16=dict(ms_per_frame=bms, frames=nb16, speedup_vs_f32=fms / bms,
                               samples_per_s=sum(counts[vi] for vi in timed_views[:nb16]) / (bms * nb16 / 1e3),
                               image_diff_vs_f32=dict(max=float(diff.max()), mean=float(diff.mean())),
                               note="bfloat16 brick storage (8-byte quads), FP32 accumulation; accuracy against "
                                    "the FP64 oracle is checked on the 1024^3 precision workload"))
        vr.vr_volume_release(vb)
        # the same with the octet cell layout (both planes of a cell per 16-byte
        # element: one load per sample; the image is bit-identical to the quads')
        vr.vr_set_cell_layout(ctx, 1)
        vo = vr.vr_volume_create(ctx, vol, "bf16", wl["part"])
        vr.vr_set_cell_layout(ctx, 0)
        for i in range(a.warmup):
            vr.vr_set_camera(ctx, cams[views[i]])
            vr.vr_render_frame(ctx, vo, out)
        torch.cuda.synchronize()
        e0.record(stream)
        for vi in timed_views[:nb16]:
            vr.vr_set_camera(ctx, cams[vi])
            vr.vr_render_frame(ctx, vo, out)
        e1.record(stream)
        torch.cuda.synchronize()
        oms = e0.elapsed_time(e1) / nb16
        forms["bf16_octets"] = dict(ms_per_frame=oms, frames=nb16, speedup_vs_f32=fms / oms,
                                    samples_per_s=sum(counts[vi] for vi in timed_views[:nb16]) / (oms * nb16 / 1e3),
                                    note="bfloat16 storage as octets (vr_set_cell_layout 1): one 16-byte load per "
                                         "sample, storage as large as float32 xy-quads")
        vr.vr_volume_release(vo)

    # ray-state cycling on the same frames (rays carry (C, T) through the bricks,
    # global early termination): executed samples and frame time
    cyc = None
    if world == 1:
        vr.vr_set_render_mode(ctx, 1)
        vr.vr_set_count_samples(ctx, True)
        ccounts = []
        for cam in cams:
            vr.vr_set_camera(ctx, cam)
            vr.vr_render_frame(ctx, v, out)
            ccounts.append(vr.vr_get_sample_count(ctx))
        vr.vr_set_count_samples(ctx, False)
        for i in range(a.warmup):
            vr.vr_set_camera(ctx, cams[views[i]])
            vr.vr_render_frame(ctx, v, out)
        torch.cuda.synchronize()
        e0.record(stream)
        for vi in timed_views:
            vr.vr_set_camera(ctx, cams[vi])
            vr.vr_render_frame(ctx, v, out)
        e1.record(stream)
        torch.cuda.synchronize()
        cms = e0.elapsed_time(e1)
        vr.vr_set_frame_pipelining(ctx, False)  # the same frames in sequence
        e0.record(stream)
        for vi in timed_views:
            vr.vr_set_camera(ctx, cams[vi])
            vr.vr_render_frame(ctx, v, out)
        e1.record(stream)
        torch.cuda.synchronize()
        cms_plain = e0.elapsed_time(e1)
        vr.vr_set_frame_pipelining(ctx, True)
        csamp = float(sum(ccounts[vi] for vi in timed_views))
        cyc = dict(ms_per_frame=cms / len(timed_views), frames_per_s=len(timed_views) / (cms / 1e3),
                   samples_per_s=csamp / (cms / 1e3), samples_per_frame=csamp / len(timed_views),
                   speedup_vs_sort_last=ms / cms, plain_ms_per_frame=cms_plain / len(timed_views))
        vr.vr_set_render_mode(ctx, 0)
    vr.vr_volume_release(v)
    vr.vr_destroy(ctx)
    if rank != 0:
        return

    K = a.steps
    value = samples / (ms / 1e3)
    frames = world * K / (ms / 1e3)
    per_frame_samples = samples / (world * K)
    march_ms = kt["march_ms"] / max(1, kt["march_launches"])
    comp_ms = kt["composite_ms"] / max(1, kt["composite_launches"])
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    hbm = peaks.get("hbm_gbs")
    hbm_src = "of measured" if hbm else "of fallback"
    hbm = hbm or 6800.0
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    sms = torch.cuda.get_device_properties(local).multi_processor_count  # read from the device
    fp32_peak = sms * FP32_LANES * 2 * sm_max * 1e6 / 1e12  # TFLOP/s, FMA = 2 flops
    march_tflops = FLOPS_PER_SAMPLE * per_frame_samples / (march_ms / 1e3) / 1e12
    mean_rect = sum(rect_px[vi] for vi in timed_views) / len(timed_views)
    comp_bytes = (mean_rect + W * H) * 16
    comp_gbs = comp_bytes / (comp_ms / 1e3) / 1e9
    vol_bytes = vol.size * 4
    march_hbm_gbs = (vol_bytes + mean_rect * 16) / (march_ms / 1e3) / 1e9
    cpu = None
    if not a.no_cpu_baseline and world == 1:
        import oracle
        oracle.build()
        cpu, _, _ = oracle_rate(wl)
        cpu["single_thread"] = oracle_rate_1thread(wl)
    line = dict(
        metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=K, warmup=a.warmup,
        ms_per_step=ms / K, higher_is_better=True, scaling="weak", vs_baseline=None,
        dtype="f32", data="synthetic",
        config=dict(workload=wl["name"], volume=list(vol.shape[::-1]), bricks=len(counts) and
                    int(np.prod(wl["grid"])), image=[W, H], views=len(cams),
                    l2="inputs larger than L2: %.0f MB of bricked volume vs 129 MB L2" % (vol_bytes / 1e6)
                    if vol_bytes > 129e6 else "small workload fits in L2",
                    parallelism="replicas over views" if world > 1 else "1 GPU"),
        frames_per_s=frames,
        samples_per_frame=per_frame_samples,
        gpu_launches=2 * K,
        clocks=clk,
        roofline=dict(bound="alu", kernel="march", achieved=march_tflops, peak=fp32_peak, unit="TFLOP/s",
                      frac=march_tflops / fp32_peak,
                      traffic=recorded_traffic() if a.workload == "paper" else None,
                      sms=sms,
                      note="FP32 %d flops/sample x executed samples / mean march launch; peak = %d SMs "
                           "(cudaDeviceProp.multiProcessorCount) x 128 lanes x 2 x %.0f MHz (derived)"
                           % (FLOPS_PER_SAMPLE, sms, sm_max)),
        roofline_l1=dict(frac=recorded_value("l1_wavefronts_frac") if a.workload == "paper" else None,
                         unit="fraction of peak L1 data-pipe wavefronts",
                         note="ncu --set full on the march of this kernel code (null once the code changes): "
                              "the L1/shared data pipe is the march's busiest unit; see profiles/"),
        roofline_issue=dict(frac=recorded_value("issue_active_frac") if a.workload == "paper" else None,
                            unit="fraction of peak warp-instruction issue (smsp__issue_active)",
                            note="ncu --set full on the march of this kernel code (null once the code changes): "
                                 "the march is bound by issue and the latency of its dependent loads"),
        roofline_hbm=dict(march=dict(achieved=march_hbm_gbs, peak=hbm, unit="GB/s", frac=march_hbm_gbs / hbm,
                                     note="compulsory bytes (volume once + partial writes) / march time, %s"
                                          % hbm_src),
                          composite=dict(achieved=comp_gbs, peak=hbm, unit="GB/s", frac=comp_gbs / hbm,
                                         note="partial reads + image write / composite time, %s" % hbm_src)),
        kernel_ms=dict(march=march_ms, composite=comp_ms,
                       note="event pairs on every launch of %d frames over the orbit views; with timing on, "
                            "frames run the plain sequence (composite: one block per 32x8 tile)" % kt_frames),
        pipelining=dict(ms_per_frame=ms / K, plain_ms_per_frame=plain_ms / K,
                        speedup=plain_ms / ms,
                        note="timed region: pipelined frames (vr_set_frame_pipelining, the default): the "
                             "composite runs as a persistent grid of 2 blocks per SM and the next frame's "
                             "march starts in this frame's tail; plain: the same frames, march then "
                             "composite then march"),
        packet=dict(width=best_pw, ms_per_frame_by_width={str(k): v_ for k, v_ in tune.items()}),
        ray_state_cycling=cyc,
        cpu_baseline=cpu,
        e2e=dict(value=samples / e2e_s, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=W * H * 16,
                 note="vr_render_frame into pinned host memory: render + %.1f MB device-to-host copy + wait "
                      "per frame. h2d_bytes_per_step is 0 by design: the volume is resident library state and "
                      "the one per-step input, the camera, travels as kernel parameters (no copy)"
                      % (W * H * 16 / 1e6)),
        forms=forms,
    )
    print(json.dumps(line))


def run_precision(a):
    """Precision form: the 1024^3 blob volume (seed 2, 64 kd bricks, 2048^2
    perspective) stored as float32, bfloat16 and float16 (the 16-bit types as
    xy-quads and as octets); frame time of each and,
    for the 16-bit forms, the error against the FP64 oracle on the centre 256^2
    crop (accumulation error: oracle on the same quantised values; total error:
    oracle on the float32 source)."""
    import numpy as np
    import torch
    import __graft_entry__
    import oracle
    from paper_2501_01628_gb300 import synth, vr
    __graft_entry__.build()
    n = 1024
    vol, tf, cuts = synth.precision_scene(n=n)
    lo, hi = synth.volume_range(vol)
    part = dict(kind="kd", n_bricks=64, cut_fracs=cuts)
    boxes = oracle.kd_partition((n,) * 3, 64, cuts)
    cam = synth.orbit_camera(2048, 2048, 30.0)
    crop = (896, 896, 256, 256)
    tfs = dict(workload=tf, ramp=synth.ramp_tf())
    ref_total = {k: oracle.render(vol, boxes, t, lo, hi, cam, 0.5, crop=crop)["img"] for k, t in tfs.items()}
    quantised = {s: synth.quantize(vol, s) for s in ("bf16", "f16")}
    vol_dev = torch.from_numpy(vol).cuda()
    out = torch.empty((2048, 2048, 4), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    forms = {}
    for form in ("f32", "bf16", "f16", "bf16_octets", "f16_octets"):
        storage = form.split("_")[0]
        ctx = vr.vr_create(0)
        vr.vr_set_cell_layout(ctx, 1 if form.endswith("octets") else 0)
        v = vr.vr_volume_create(ctx, vol_dev, storage, part)
        vr.vr_set_transfer_function(ctx, tf, lo, hi)
        vr.vr_set_render_params(ctx, 0.5, 1.0)
        vr.vr_set_camera(ctx, cam)
        vr.vr_set_count_samples(ctx, True)
        vr.vr_render_frame(ctx, v, out)
        nsamp = vr.vr_get_sample_count(ctx)
        vr.vr_set_count_samples(ctx, False)
        for _ in range(a.warmup):
            vr.vr_render_frame(ctx, v, out)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(a.steps):
            vr.vr_render_frame(ctx, v, out)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / a.steps
        _, nbytes = vr.vr_volume_info(v)
        f = dict(ms_per_frame=ms, samples_per_s=nsamp / (ms / 1e3), storage_bytes=nbytes)
        for kind, t in tfs.items():
            vr.vr_set_transfer_function(ctx, t, lo, hi)
            vr.vr_render_frame(ctx, v, out)
            img = out[896:1152, 896:1152].cpu().numpy().astype(np.float64)
            e = dict(err_total_mean=float(np.mean(np.abs(img - ref_total[kind]))),
                     err_total_max=float(np.max(np.abs(img - ref_total[kind]))))
            if storage != "f32":
                code = oracle.BF16 if storage == "bf16" else oracle.F16
                ref_q = oracle.render(quantised[storage], boxes, t, lo, hi, cam, 0.5, crop=crop,
                                      dtype=code)["img"]
                e["err_accumulation_max"] = float(np.max(np.abs(img - ref_q)))
            f["tf_" + kind] = e
        forms[form] = f
        vr.vr_volume_release(v)
        vr.vr_destroy(ctx)
    for s in ("bf16", "f16", "bf16_octets", "f16_octets"):
        forms[s]["speedup_vs_f32"] = forms["f32"]["ms_per_frame"] / forms[s]["ms_per_frame"]
    line = dict(metric=METRIC, value=forms["bf16"]["samples_per_s"], unit=UNIT, n_gpus=1, steps=a.steps,
                warmup=a.warmup, ms_per_step=forms["bf16"]["ms_per_frame"], higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="bf16 storage, f32 arithmetic", data="synthetic",
                config=dict(workload="precision: 1024^3 blobs (seed 2), 64 kd bricks, 2048x2048 perspective "
                                     "(azimuth 30 deg), step 0.5 voxel; error on the centre 256^2 crop"),
                forms=forms, gpu_launches=2 * a.steps)
    print(json.dumps(line))


def run_grad(a):
    """Differentiation form: one training step = forward of 16 views (512^2) of
    the 256^3 blob volume (seed 4, 8 bricks), mean-squared image loss against
    targets of the perturbed volume density*(1 + 0.05 xi), and the backward pass
    through the adjoint kernels to the 256x4 table and every voxel."""
    import numpy as np
    import torch
    import __graft_entry__
    from paper_2501_01628_gb300 import synth, vr
    from paper_2501_01628_gb300.autograd import Renderer
    __graft_entry__.build()
    n = 256
    rng = np.random.default_rng(4)
    vol = synth.blob_volume(n, synth.draw_blobs(rng, 8))
    tf = synth.random_tf(rng)
    xi = np.random.default_rng(5).standard_normal(vol.shape).astype(np.float32)
    vol_t = vol * (np.float32(1.0) + np.float32(0.05) * xi)
    lo, hi = float(min(vol.min(), vol_t.min())), float(max(vol.max(), vol_t.max()))
    part = dict(kind="grid", grid=(2, 2, 2))
    cams = [synth.orbit_camera(512, 512, 22.5 * i, elevation_deg=20.0 if i % 2 else -10.0) for i in range(16)]
    r = Renderer(part, lo, hi)
    tft = torch.from_numpy(tf).cuda().requires_grad_(True)
    dens = torch.from_numpy(vol).cuda().requires_grad_(True)
    with torch.no_grad():
        dt_ = torch.from_numpy(vol_t).cuda()
        targets = [r.render(tft.detach(), dt_, c).clone() for c in cams]
    # executed forward samples per step
    ctx = vr.vr_create(0)
    v = vr.vr_volume_create(ctx, dens.detach(), "f32", part)
    vr.vr_set_transfer_function(ctx, tf, lo, hi)
    vr.vr_set_render_params(ctx, 0.5, 1.0)
    vr.vr_set_count_samples(ctx, True)
    tmp = torch.empty((512, 512, 4), device="cuda")
    for c in cams:
        vr.vr_set_camera(ctx, c)
        vr.vr_render_frame(ctx, v, tmp)
    fwd_samples = vr.vr_get_sample_count(ctx)
    vr.vr_volume_release(v)
    vr.vr_destroy(ctx)

    def step():
        tft.grad = None
        dens.grad = None
        loss = sum(((r.render(tft, dens, c) - t) ** 2).mean() for c, t in zip(cams, targets)) / len(cams)
        loss.backward()
        return loss

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        loss = step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.steps
    # forward only, for the split
    e0.record(stream)
    with torch.no_grad():
        for _ in range(a.steps):
            for c in cams:
                r.render(tft, dens, c)
    e1.record(stream)
    torch.cuda.synchronize()
    fwd_ms = e0.elapsed_time(e1) / a.steps
    r.close()
    line = dict(metric=METRIC, value=fwd_samples / (ms / 1e3), unit=UNIT, n_gpus=1, steps=a.steps, warmup=a.warmup,
                ms_per_step=ms, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32",
                data="synthetic",
                config=dict(workload="differentiation: 256^3 blobs (seed 4), 8 bricks, 16 views at 512x512, "
                                     "MSE against the density*(1+0.05 xi) renders; gradients for the 256x4 table "
                                     "and all 256^3 voxels; value = forward samples per second of training steps"),
                forward_ms_per_16_views=fwd_ms, backward_ms=ms - fwd_ms,
                forward_samples_per_step=fwd_samples, loss=float(loss.detach()),
                gpu_launches=a.steps * 16 * 4)
    print(json.dumps(line))


def run_batch(a):
    """Batching form: 6 time steps x 3 fields of 768^3 stored as f16 (advected
    blobs + lattice noise, seed 3), 48 kd bricks, 32 views at 1024^2: the 576
    renders and their compositing in one persistent CUDA-graph launch, packet
    shape and residency autotuned; compared with 576 plain vr_render_frame
    calls on the same volumes and views."""
    import numpy as np
    import torch
    import __graft_entry__
    from paper_2501_01628_gb300 import synth, vr
    __graft_entry__.build()
    n, steps, nfields, nviews = 768, 6, 3, 32
    draws = synth.draw_fields(seed=3, n_fields=nfields)
    rng = np.random.default_rng(3)
    tf = synth.random_tf(rng)
    cuts = synth.kd_cut_fractions(rng, 48)
    part = dict(kind="kd", n_bricks=48, cut_fracs=cuts)
    cams = [synth.orbit_camera(1024, 1024, 360.0 * w / nviews, elevation_deg=20.0 * np.cos(w))
            for w in range(nviews)]
    ctx = vr.vr_create(0)
    vr.vr_set_cell_layout(ctx, 1 if a.layout == "octets" else 0)
    vols, ranges = [], []
    for st in range(steps):
        for f in range(nfields):
            src = synth.field_volume_torch(draws[f], st, n)
            ranges.append((float(src.min()), float(src.max())))
            vols.append(vr.vr_volume_create(ctx, src, "f16", part))
            del src
    torch.cuda.empty_cache()
    storage = sum(vr.vr_volume_info(v)[1] for v in vols)
    vr.vr_set_transfer_function(ctx, tf, 0.0, 1.0)
    vr.vr_set_render_params(ctx, 0.5, 1.0)
    nr = len(vols) * nviews
    out = torch.empty((nr, 1024, 1024, 4), device="cuda")
    b = vr.vr_batch_create(ctx, vols, cams, out, vmins=[r[0] for r in ranges], vmaxs=[r[1] for r in ranges])
    t0 = time.perf_counter()
    chosen = vr.vr_batch_autotune(b)
    tune_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    for _ in range(max(1, a.warmup)):
        vr.vr_batch_launch(b)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        vr.vr_batch_launch(b)
    e1.record(stream)
    torch.cuda.synchronize()
    vr.vr_sync(ctx)
    batch_ms = e0.elapsed_time(e1) / a.steps
    # the plain form: one vr_render_frame per render (and the executed-sample count)
    img = torch.empty((1024, 1024, 4), device="cuda")
    vr.vr_set_count_samples(ctx, True)
    for v, (lo, hi) in zip(vols, ranges):
        vr.vr_set_transfer_function(ctx, tf, lo, hi)
        for c in cams:
            vr.vr_set_camera(ctx, c)
            vr.vr_render_frame(ctx, v, img)
    samples = vr.vr_get_sample_count(ctx)
    vr.vr_set_count_samples(ctx, False)
    torch.cuda.synchronize()
    e0.record(stream)
    for v, (lo, hi) in zip(vols, ranges):
        vr.vr_set_transfer_function(ctx, tf, lo, hi)
        for c in cams:
            vr.vr_set_camera(ctx, c)
            vr.vr_render_frame(ctx, v, img)
    e1.record(stream)
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1)
    vr.vr_batch_release(b)
    for v in vols:
        vr.vr_volume_release(v)
    vr.vr_destroy(ctx)
    line = dict(metric=METRIC, value=samples / (batch_ms / 1e3), unit=UNIT, n_gpus=1, steps=a.steps,
                warmup=a.warmup, ms_per_step=batch_ms, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f16 storage, f32 arithmetic", data="synthetic",
                config=dict(workload="batching: 6 steps x 3 fields x 768^3 f16 (seed 3), 48 kd bricks, 32 views at "
                                     "1024x1024 = 576 renders + compositing in one persistent CUDA-graph launch"),
                renders_per_s=nr / (batch_ms / 1e3), samples_per_batch=samples, storage_bytes=storage,
                cell_layout=a.layout,
                autotune=dict(packet_width=chosen[0], blocks_per_sm=chosen[1], ring_slots=chosen[2],
                              order="brick-major per volume" if chosen[3] == 1 else "render-major",
                              seconds=tune_s),
                plain=dict(ms_for_576_renders=plain_ms, samples_per_s=samples / (plain_ms / 1e3)),
                speedup_vs_plain=plain_ms / batch_ms, gpu_launches=a.steps)
    print(json.dumps(line))


def run_stream(a):
    """Time-step streaming: 8 time steps of a 512^3 float32 field (advected blobs
    + lattice noise, seed 3) in pinned host memory, 36 bricks, 2 device slots;
    each step renders 4 orbit views at 1920x1080 (ERT 0.99) while the next step
    is uploaded and packed on a copy stream. Compared with uploading each step
    and only then rendering it."""
    import numpy as np
    import torch
    import __graft_entry__
    from paper_2501_01628_gb300 import synth, vr
    from paper_2501_01628_gb300.streaming import TimeSeriesRenderer
    __graft_entry__.build()
    n, steps = 512, 8
    draws = synth.draw_fields(seed=3, n_fields=1)[0]
    host = []
    for t in range(steps):
        host.append(synth.field_volume_torch(draws, t, n).cpu().pin_memory())
    rng = np.random.default_rng(3)
    tf = synth.random_tf(rng)
    lo = min(float(h.min()) for h in host)
    hi = max(float(h.max()) for h in host)
    part = dict(kind="grid", grid=(4, 3, 3))
    cams = [synth.orbit_camera(1920, 1080, az) for az in (0.0, 90.0, 180.0, 270.0)]
    ctx = vr.vr_create(0)
    vr.vr_set_transfer_function(ctx, tf, lo, hi)
    vr.vr_set_render_params(ctx, 0.5, 0.99)
    outs = [torch.empty((1080, 1920, 4), device="cuda") for _ in cams]
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        torch.cuda.synchronize()
        ev0.record(stream)
        fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1)

    r = TimeSeriesRenderer(ctx, host, part, slots=2)
    for t in range(2):  # warm
        r.render_step(t, cams, outs)
    r.close()
    res = {}
    for prefetch in (True, False):
        r = TimeSeriesRenderer(ctx, host, part, slots=2)

        def run():
            for t in range(steps):
                r.render_step(t, cams, outs, prefetch=prefetch)
                if not prefetch:
                    # no overlap: wait for each step's upload before its renders
                    torch.cuda.synchronize()
        # the first two steps are resident at creation; time steps 0..7
        res[prefetch] = timed(run)
        vr.vr_sync(ctx)  # raises if a bounded device-side wait gave up
        r.close()
    # upload + pack of one step alone
    v = vr.vr_volume_create(ctx, host[0], "f32", part)
    up_ms = timed(lambda: vr.vr_volume_update_async(v, host[1]))
    vr.vr_volume_release(v)
    vr.vr_destroy(ctx)
    nbytes = host[0].numel() * 4
    line = dict(metric=METRIC, value=steps * len(cams) / (res[True] / 1e3), unit="frames/s", n_gpus=1,
                steps=steps, warmup=2, ms_per_step=res[True] / steps, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f32", data="synthetic",
                config=dict(workload="time-step streaming: 8 steps of 512^3 f32 in pinned host memory, 2 device "
                                     "slots, 36 bricks, 4 views of 1920x1080 per step, ERT 0.99"),
                overlapped_ms=res[True], sequential_ms=res[False], speedup_vs_sequential=res[False] / res[True],
                upload_pack_ms_per_step=up_ms, upload_GBps=nbytes / (up_ms / 1e3) / 1e9,
                device_budget_bytes_f32_quads="2 volumes", gpu_launches=steps * len(cams) * 2)
    print(json.dumps(line))


MESH_NAME = ("unstructured elements: 25.0M-tetrahedron graded jittered mesh of a 512^3 nominal domain "
             "(seed 5; 0.20M..2.60M elements per brick), 36 bricks (4x3x3), 1920x1080 perspective 60 deg "
             "orbit (8 views), step 0.5 voxel, early termination at alpha 0.99, radix-k composite 4x3x3")


def mesh_oracle_rate(verts, vals, tets, boxes, tf, cams, step, ert, n_pix: int = 3000):
    """Oracle samples/s on n_pix pixels spread over one view (one call: the
    oracle builds its element index, then renders the pixels; both timed)."""
    import numpy as np
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    cam = cams[1]
    W, H = cam["width"], cam["height"]
    rng = np.random.default_rng(9)
    pix = np.stack([rng.integers(0, W, n_pix), rng.integers(0, H, n_pix)], axis=1)
    mesh = oracle.Mesh(verts, vals, tets, (512, 512, 512))
    t = time.perf_counter()
    r = oracle.render(mesh, boxes, tf, 0.0, 1.0, cam, step, ert, pixels=pix, threads=cores)
    dt = time.perf_counter() - t
    return dict(value=r["nsamples"] / dt, unit=UNIT, cores=cores, kind="oracle",
                sample="%d random pixels of one 1920x1080 view (%d samples, %.1f s incl. the oracle's element "
                       "index build, FP64, %d threads)" % (n_pix, r["nsamples"], dt, cores)), r["nsamples"], dt


def run_mesh(a):
    """Tetrahedral-mesh volumes (the paper's data set is an unevenly distributed
    mixed-element mesh, Sec. 5): one step = one composited frame of the next
    orbit view; per-brick BVH point location + face-neighbour walk, then the
    sort-last composite."""
    import numpy as np
    from paper_2501_01628_gb300 import synth
    verts, vals, tets, tf, boxes = synth.mesh_scene()
    cams = [synth.orbit_camera(1920, 1080, az) for az in synth.ORBIT_AZIMUTHS]
    step, ert = 0.5, 0.99
    if a.impl == "reference":
        if int(os.environ.get("RANK", "0")) != 0:
            return
        cpu, n, dt = mesh_oracle_rate(verts, vals, tets, boxes, tf, cams, step, ert, n_pix=1500)
        line = dict(impl="reference", metric=METRIC, value=cpu["value"], unit=UNIT, n_gpus=0, steps=1, warmup=0,
                    ms_per_step=dt * 1e3, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64",
                    data="synthetic", config=dict(workload=MESH_NAME, sample=cpu["sample"]), cpu_baseline=cpu,
                    e2e=dict(value=cpu["value"], unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
        print(json.dumps(line))
        return
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2501_01628_gb300 import vr
    part = dict(kind="grid", grid=(4, 3, 3))
    ctx = vr.vr_create(0)
    t0 = time.perf_counter()
    m = vr.vr_mesh_create(ctx, verts, vals, tets, (512, 512, 512), part)
    create_s = time.perf_counter() - t0
    per_brick, mesh_bytes = vr.vr_mesh_info(m)
    vr.vr_set_transfer_function(ctx, tf, 0.0, 1.0)
    vr.vr_set_render_params(ctx, step, ert)
    vr.vr_set_composite_schedule(ctx, (4, 3, 3))
    W, H = 1920, 1080
    out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    counts = []
    vr.vr_set_count_samples(ctx, True)
    for cam in cams:
        vr.vr_set_camera(ctx, cam)
        vr.vr_render_mesh_frame(ctx, m, out)
        counts.append(vr.vr_get_sample_count(ctx))
    vr.vr_set_count_samples(ctx, False)
    views = [i % len(cams) for i in range(a.warmup + a.steps)]
    for i in range(a.warmup):
        vr.vr_set_camera(ctx, cams[views[i]])
        vr.vr_render_mesh_frame(ctx, m, out)
    vr.vr_sync(ctx)
    timed_views = views[a.warmup:]
    clocks = ClockSampler(0)
    clocks.start()
    vr.vr_get_kernel_timing(ctx)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for vi in timed_views:
        vr.vr_set_camera(ctx, cams[vi])
        vr.vr_render_mesh_frame(ctx, m, out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    vr.vr_set_kernel_timing(ctx, True)  # per-kernel durations: a separate pass
    for i in range(max(KT_FRAMES // 4, len(timed_views))):
        vr.vr_set_camera(ctx, cams[i % len(cams)])
        vr.vr_render_mesh_frame(ctx, m, out)
    kt = vr.vr_get_kernel_timing(ctx)
    vr.vr_set_kernel_timing(ctx, False)
    hosts = [torch.empty((H, W, 4), dtype=torch.float32).pin_memory() for _ in range(2)]
    vr.vr_set_host_output_async(ctx, True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i, vi in enumerate(timed_views):
        vr.vr_set_camera(ctx, cams[vi])
        vr.vr_render_mesh_frame(ctx, m, hosts[i & 1])
    vr.vr_sync(ctx)
    e2e_s = time.perf_counter() - t0
    vr.vr_set_host_output_async(ctx, False)
    vr.vr_mesh_release(m)
    vr.vr_destroy(ctx)
    K = a.steps
    samples = float(sum(counts[vi] for vi in timed_views))
    march_ms = kt["march_ms"] / max(1, kt["march_launches"])
    comp_ms = kt["composite_ms"] / max(1, kt["composite_launches"])
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = peaks.get("hbm_gbs") or 6800.0
    hbm_src = "of measured" if peaks.get("hbm_gbs") else "of fallback"
    # compulsory bytes of one march: every element record, neighbour entry and
    # BVH node read at most once (upper bound: the whole mesh) + partial writes
    rects_sum = 0
    for vi in timed_views[:len(cams)]:
        _, rects = vr.vr_plan_view((512, 512, 512), part, cams[vi])
        rects_sum += int(sum(int(r[2]) * int(r[3]) for r in rects))
    mean_rect = rects_sum / min(len(cams), len(timed_views))
    march_bytes = mesh_bytes + mean_rect * 16
    march_gbs = march_bytes / (march_ms / 1e3) / 1e9
    cpu = None
    if not a.no_cpu_baseline:
        cpu, _, _ = mesh_oracle_rate(verts, vals, tets, boxes, tf, cams, step, ert)
    line = dict(
        metric=METRIC, value=samples / (ms / 1e3), unit=UNIT, n_gpus=1, steps=K, warmup=a.warmup,
        ms_per_step=ms / K, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32",
        data="synthetic",
        config=dict(workload=MESH_NAME, elements=int(tets.shape[0]), vertices=int(verts.shape[0]),
                    elements_per_brick=[int(min(per_brick)), int(max(per_brick))], bricks=36, image=[W, H],
                    views=len(cams), l2="inputs larger than L2: %.2f GB of mesh records vs 129 MB L2"
                    % (mesh_bytes / 1e9), parallelism="1 GPU"),
        frames_per_s=K / (ms / 1e3), samples_per_frame=samples / K, gpu_launches=2 * K, clocks=clk,
        roofline=dict(bound="hbm", kernel="march_mesh", achieved=march_gbs, peak=hbm, unit="GB/s",
                      frac=march_gbs / hbm, traffic=recorded_traffic("mesh_workload.md", MESH_SOURCES),
                      note="upper-bound compulsory bytes (whole mesh once + partial writes) / mean march "
                           "launch, %s; the walk is latency-bound (dependent element loads)" % hbm_src),
        kernel_ms=dict(march=march_ms, composite=comp_ms), mesh_create_s=create_s, mesh_device_bytes=mesh_bytes,
        cpu_baseline=cpu,
        e2e=dict(value=samples / e2e_s, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=W * H * 16,
                 note="vr_render_mesh_frame into pinned host memory (asynchronous double-buffered copies), "
                      "all frames waited for"))
    print(json.dumps(line))


def prime_factors(n: int):
    out, f = [], 2
    while n > 1:
        while n % f == 0:
            out.append(f)
            n //= f
        f += 1
    return out or [1]


def run_bricks(a):
    """Bricks as ranks: each rank holds a share of the 36 bricks (kd split of
    the partition), marches it, and the ranks' images are composited by a
    radix-k exchange over NCCL (factors: the prime factors of the rank count)
    and gathered on rank 0. One step = one composited frame of the whole
    volume; the work per frame is fixed as ranks are added (strong scaling).
    value = executed samples of all ranks per second."""
    import socket
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    else:  # one rank: a single-process group, so the same code path runs
        with socket.socket() as sk:
            sk.bind(("127.0.0.1", 0))
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            os.environ.setdefault("MASTER_PORT", str(sk.getsockname()[1]))
        dist.init_process_group("gloo", rank=0, world_size=1)
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    dist.barrier()
    from paper_2501_01628_gb300 import sharded, vr
    wl = workload(a.workload)
    vol, tf = wl["vol"], wl["tf"]
    lo, hi = float(vol.min()), float(vol.max())
    cams = wl["cams"]
    ctx = vr.vr_create(local)
    vr.vr_set_transfer_function(ctx, tf, lo, hi)
    vr.vr_set_render_params(ctx, wl["step"], wl["ert"])
    vr.vr_set_composite_schedule(ctx, wl["schedule"])  # each rank's own bricks (empty partials elsewhere)
    factors = prime_factors(world)
    r = sharded.ShardedRenderer(ctx, torch.from_numpy(vol).cuda(), wl["part"], factors=factors)
    W, H = cams[0]["width"], cams[0]["height"]
    frame = torch.empty((H, W, 4), device="cuda") if rank == 0 else None
    counts = []
    vr.vr_set_count_samples(ctx, True)
    for cam in cams:
        r.render(cam, frame)
        counts.append(vr.vr_get_sample_count(ctx))
    vr.vr_set_count_samples(ctx, False)
    for i in range(a.warmup):
        r.render(cams[i % len(cams)], frame)
    torch.cuda.synchronize()
    dist.barrier()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    e0.record(stream)
    for i in range(a.steps):
        r.render(cams[(a.warmup + i) % len(cams)], frame)
    e1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    # end to end: the same frames, each read back to pinned host memory on rank 0
    host = torch.empty((H, W, 4)).pin_memory() if rank == 0 else None
    dist.barrier()
    t0 = time.perf_counter()
    for i in range(a.steps):
        out = r.render(cams[(a.warmup + i) % len(cams)], frame)
        if rank == 0:
            host.copy_(out)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    samples = float(sum(counts[(a.warmup + i) % len(cams)] for i in range(a.steps)))
    ms, e2e_s, samples = reduce_job(ms, e2e_s, samples, world, device="cuda" if world > 1 else "cpu")
    r.close()
    vr.vr_destroy(ctx)
    dist.destroy_process_group()
    if rank != 0:
        return
    line = dict(metric=METRIC, value=samples / (ms / 1e3), unit=UNIT, n_gpus=world, steps=a.steps,
                warmup=a.warmup, ms_per_step=ms / a.steps, higher_is_better=True, scaling="strong",
                vs_baseline=None, dtype="f32", data="synthetic",
                config=dict(workload=wl["name"], parallelism="bricks as ranks, radix-k %s over %s"
                            % ("x".join(map(str, factors)), "NCCL" if world > 1 else "one rank"),
                            l2="inputs larger than L2" if vol.nbytes > 129e6 else "fits in L2"),
                frames_per_s=a.steps / (ms / 1e3),
                gpu_launches=a.steps * (2 + (len(factors) if world > 1 else 0)), clocks=clk,
                e2e=dict(value=samples / e2e_s, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=W * H * 16,
                         note="frame gathered on rank 0 and copied to pinned host memory"))
    print(json.dumps(line))


def main():
    a = args_parse()
    if a.split == "bricks":
        run_bricks(a)
        return
    if a.workload == "mesh":
        run_mesh(a)
        return
    if a.workload == "stream":
        run_stream(a)
        return
    if a.workload == "batch":
        run_batch(a)
        return
    if a.workload == "grad":
        run_grad(a)
        return
    if a.workload == "precision":
        run_precision(a)
        return
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
