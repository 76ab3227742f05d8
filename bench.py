#!/usr/bin/env python3
"""Benchmark of the hybrid depth-of-field pass (one JSON line on stdout).

A step is one frame of the pass (dof_frame: CoC, tiles, prefilter, 81-tap gather,
median, ray mask + compaction, thin-lens rays through the device BVH, accumulation,
variance blur, median, mips, reconstruction, composite) on the 1920x1080 workload:
495,802-triangle lawn scene, 35 mm f/2 focused at 20 m, CoC radius <= 32 px, 1 spp,
16-frame camera dolly.  The 16 G-buffers (produced on the device beforehand) are
cycled, so each step reads inputs that are not in L2 (16 x 41 MB > 129 MB L2).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--config c1|c2|c3|batch|serve]
                    [--impl ours|reference] [--size WxH]

N > 1 (torchrun): every rank renders its own session (replicas; the sessions are
independent, there is no data exchange); the value is all ranks' frames over the
max-over-ranks time.  --impl reference times the FP64 oracle on the host cores.
"""

from __future__ import annotations

import argparse
import ctypes as C
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "hybrid-DoF frames/s at 1080p/4K, %HBM roofline; served p50/p99 frame latency"
CYCLE = 16
C3_STEPS = 32        # timed 4K frames of the default run's c3 sub-record

# FP32 operations of the traversal (FMA = 2): a binary node visit tests two child
# boxes (per box 6 FMA slab products = 12, 10 min/max, 1 compare -> 23, x2 = 46)
# and orders them (1); a 4-wide node visit tests four boxes (6 FMA slab products = 12,
# 10 min/max, 1 compare -> 23, x4 = 92) and sorts them (5 compares); a watertight
# triangle test (Woop et al. 2013) is 9 subtractions, 6 shears (sub, mul) = 12,
# 3 edge functions (2 mul + sub) = 9, 6 sign tests, det (2), T (3 mul + 3 FMA = 9),
# 1 division -> 48.  Warp packets (k_trace_packets) count, per lane, every binary node
# and triangle its lane tested: the union of the warp's rays' nodes.
FLOP_PER_NODE = {2: 47.0, 4: 97.0}
# The 81-tap gathers are bound by issue slots and L1 together; their roofline, when one of
# them is the frame's dominant kernel, counts FP32 operations (FMA = 2) per pixel that takes
# taps against the FP32 peak.
# * Main filter (every hpx N), per tap: position 5 (product, 2 FMA), fractions 2, weights 6,
#   sample 4 texels x 4 channels FMA = 32, depth 8, weight W 14 (difference, product,
#   max, reciprocal-multiply, 2 coverage FMA, 3 clamps as 6 min/max, blend), 4 colour and
#   1 bright accumulation FMA = 10, luminance 5 -> 82.
# * Reconstruction (hpx with rays M; the Eq. 5 blend below 2^-24 skips its taps, so this
#   is an upper bound of the work), per tap: position 5, per level (two levels) fractions
#   2 + weights 7 + 4 texels x (4 colour + 2 coverage) FMA = 48 -> 57 x 2 = 114, coverage
#   ratio 1, weight D 4, 4 + 1 accumulation FMA = 10 -> 134.
FLOP_PER_GATHER = {"k_main_filter": ("N", 81 * 82.0), "k_recon": ("M", 81 * 134.0)}
FLOP_PER_TRI = 48.0
FP32_LANES_PER_SM = 128

# DRAM bytes (read + write) per launch from the last ncu capture of each kernel on the
# workload (profiles/tracer_c3_1080p.md, profiles/tracer_packets.md, profiles/recon_c2_1080p.md); a kernel or
# workload changed since its capture has None.  The 4K tracers were captured at
# 1920x1080 (same scene, lens, 4 spp, rays grouped by lens cell) and are scaled by the
# rays of a full launch (6.73M / 1.78M); their DRAM writes are the rays they keep for the
# shader that L2 does not hold, so the scaled figures are estimates.
PROFILED_TRAFFIC = {"c2": {"k_trace_rays<1>": None, "k_trace_rays<0>": None, "k_trace_packets": 7.486e6 + 0.0,
                           "k_recon": 27.234e6 + 13.8e3, "k_main_filter": None, "k_accumulate": None, "k_composite": None,
                           "k_downscale_tiles": None},
                    "c3": {"k_trace_rays<0>": (21.68e6 + 10.87e6) * 6.72 / 1.78,
                           "k_trace_packets": (19.363e6 + 3.338e6) * 6.723 / 1.778}}

# Algorithmic (compulsory) DRAM bytes of each kernel per unit (FP32 layouts): per
# half-resolution pixel N, per masked pixel M, per ray R, per full-resolution pixel P.
BYTES = {
    "k_downscale_tiles": ("N", 100.0),   # 4 x (colour 16 + depth 4) read, pp_in 16 + z 4 written
    "k_prefilter": ("N", 32.0),
    "k_main_filter": ("N", 36.0),        # pre 16 + z 4 read, 16 written (neighbour taps from cache)
    "k_median_pp": ("N", 32.0),
    "k_mask_compact": [("N", 4.0), ("M", 8.0), ("R", 4.0)],   # ray count per hpx; queue entry and
                                         # first-ray index per masked hpx; ray list entry per ray
                                         # (+ 4 B/N of x_f read in the adaptive mode, not counted)
    "k_trace_rays": ("R", 36.0),              # per ray: ray list 4 read, hit 8 + kept ray 24 written (BVH reads hit L2)
    "k_shade": [("M", 76.0), ("R", 32.0)],  # queue, count, first ray read, 4 x float4 written; hits + kept rays read
    "k_accumulate": ("N", 192.0),        # rt 64 + z 4 + nrays 4 + history 48 read; history 48 + 24 written
    "k_median_rt": ("N", 80.0),          # fused: variance blur (var 4 read, 4 written), RT median
                                         # (crt 16 + nrays 4 read, 16 written), mip 0 (ct 4 read,
                                         # 24 written), mip levels 1-3 (24 x (1/4 + 1/16 + 1/64) written)
    "k_recon": ("N", 44.0),
    "k_composite": ("P", 45.0),          # colour 16 + depth 4 read, 16 written, + hpx inputs / 4
                                         # (one thread per hpx writes its 2x2 fpx)
    "k_taa": ("P", 68.0),                # composite 16 + depth 4 + history 16 read, out 16 + history 16 written
}


def algo_bytes(kernel, units):
    """Algorithmic bytes of one launch: the sum over the kernel's (unit, bytes per unit) terms."""
    terms = BYTES[kernel]
    if isinstance(terms, tuple):
        terms = [terms]
    return sum(units[u] * b for u, b in terms)


# HBM-bound streaming passes and the gather passes of a frame.  The mask kernel (ray
# count, compaction, and, when the tracer takes rays grouped by lens cell, one Philox
# lens sample per ray) is reported apart: with the grouping it is bound by that
# arithmetic, not by its few bytes.
STREAMING = ["k_downscale_tiles", "k_median_pp", "k_accumulate", "k_median_rt", "k_composite", "k_taa"]
RAY_LIST = ["k_mask_compact"]
GATHERS = ["k_prefilter", "k_main_filter", "k_recon"]


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def max_over_ranks(x: float) -> float:
    """Largest value over the ranks of the default process group (identity alone)."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def job_value(steps: int, ms: float, world: int) -> float:
    """Whole-job frames/s: every rank renders `steps` frames; time = max over ranks."""
    return world * steps / (ms / 1e3)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded sample of the workload
# ---------------------------------------------------------------------------

def oracle_sample(w, budget_s=15.0, steps=None):
    """Time oracle frames on full-width bands of the workload's frame (same scene,
    lens and camera path).  Returns (frames/s scaled to the full frame, description,
    threads, per-step list)."""
    import oracle
    oracle.build()
    osc = oracle.Scene(w.scene)
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    H_band = max(16, (w.H // 8) // 2 * 2)
    from synth import make_workload
    band = make_workload(w.name, W=w.W, H=H_band)
    cams = [band.camera(k % band.n_frames) for k in range(CYCLE)]
    gbs = {}
    times = []
    t_total = time.time()
    n = 0
    while True:
        k = n % min(CYCLE, band.n_frames)
        if k not in gbs:
            gbs[k] = oracle.gbuffer_f32(oracle.gbuffer(osc, cams[k], band.params, band.W, band.H))
        hist = oracle.History(band.W, band.H)
        t0 = time.perf_counter()
        oracle.frame(osc, cams[k], band.params, band.W, band.H, gbs[k], hist, keep_rays=False)
        times.append(time.perf_counter() - t0)
        n += 1
        if steps is not None:
            if n >= steps:
                break
        elif time.time() - t_total > budget_s or n >= 8:
            break
    frac = (band.W * band.H) / (w.W * w.H)
    per_frame = statistics.median(times) / frac
    desc = (f"{w.W}x{H_band} bands (1/{round(1 / frac)} of a {w.W}x{w.H} frame) of the same scene and lens, "
            f"{len(times)} frames, oracle frame only (G-buffer precomputed), scaled to a full frame")
    return 1.0 / per_frame, desc, threads, times, frac


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(w, budget_s=15.0, single_steps=2):
    """The FP64 oracle on the host cores: all threads (OpenMP over rows), then one
    thread, on bands of the workload's frame (same output for any thread count)."""
    import oracle
    fps, desc, threads, _, _ = oracle_sample(w, budget_s=budget_s)
    prev = oracle.set_threads(1)
    try:
        fps1, desc1, _, _, _ = oracle_sample(w, steps=single_steps)
    finally:
        oracle.set_threads(prev)
    return dict(value=round(fps, 5), unit="frames/s", cores=threads, kind="oracle", sample=desc,
                cpu_model=cpu_model(), single_thread=dict(value=round(fps1, 5), unit="frames/s", cores=1,
                                                          sample=desc1))


def coc_reach(w, gbs, prm):
    """Largest CoC radius (full-resolution px) the workload's frames reach: the thin-lens
    radius at the nearest depth of the G-buffers (Eq. 6 closed form), and the same after
    the max_coc_px clamp the passes apply."""
    import torch
    f, N, d, ws = (w.intr[k] for k in ("f_m", "f_number", "focus_m", "sensor_w_m"))
    k_coc = (f / N) * f * w.W / (ws * (d - f))
    zmin = min(float(torch.nan_to_num(g["depth"], posinf=1e30).min()) for g in gbs)
    r = abs(k_coc * (zmin - d) / zmin) / 2.0
    return dict(nearest_depth_m=round(zmin, 4), physical=round(r, 2),
                clamped=round(min(r, float(prm["max_coc_px"])), 2), clamp=float(prm["max_coc_px"]))


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def gbuffer_producers(dof, ctx, scene, w, prm, reps=10):
    """Device time of the two G-buffer producers on the workload's first camera (outputs
    preallocated, 3 warm-up calls each), and whether their outputs agree bit for bit."""
    import torch
    cam = w.camera(0)
    outs, ms = {}, {}
    for raster in (False, True):
        o = dof.gbuffer(ctx, scene, cam, prm, w.W, w.H, raster=raster)
        for _ in range(2):
            dof.gbuffer(ctx, scene, cam, prm, w.W, w.H, out=o, raster=raster)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            dof.gbuffer(ctx, scene, cam, prm, w.W, w.H, out=o, raster=raster)
        e1.record()
        torch.cuda.synchronize()
        ms["raster" if raster else "ray_cast"] = round(e0.elapsed_time(e1) / reps, 4)
        outs[raster] = o
    same = all(torch.equal(outs[False][k].view(torch.int32), outs[True][k].view(torch.int32))
               for k in ("color", "depth", "normal", "prim"))
    return dict(ms=ms, bitwise_equal=bool(same))


def run_ours(args, rank, world):
    import numpy as np
    import torch
    from paper_2210_06158_gb300 import _build, dof, tune
    from synth import make_workload

    _build.build()
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.size:
        sw, sh = (int(v) for v in args.size.lower().split("x"))
        w = make_workload(args.config, W=sw, H=sh, session=rank)
    else:
        w = make_workload(args.config, session=rank)
    prm = dict(w.params)
    if args.taa:
        w.jitter = True
        prm["taa_alpha"] = 0.1
    if args.image_storage == "f16":
        prm["image_storage"] = 1
    spp = int(prm["spp"])
    ctx = dof.Context(local)
    stream = torch.cuda.current_stream()
    # the packet tracer's visit counters only in the instrumented pass below
    ctx.set_trace(stats=False)

    t0 = time.perf_counter()
    scene = dof.Scene(ctx, w.scene)
    bvh_ms = (time.perf_counter() - t0) * 1e3
    info = scene.info()

    # G-buffers of the dolly (A0, on the device)
    gbs = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for k in range(CYCLE):
        gbs.append(dof.gbuffer(ctx, scene, w.camera(k % w.n_frames), prm, w.W, w.H))
    ev1.record()
    torch.cuda.synchronize()
    gbuf_ms = ev0.elapsed_time(ev1) / CYCLE
    gbuf_cmp = gbuffer_producers(dof, ctx, scene, w, prm)
    reach = coc_reach(w, gbs, prm)
    for g in gbs:
        del g["prim"]
    pstruct = dof.params_struct(prm)

    def cam_for(step):
        c = w.camera(step % CYCLE % w.n_frames)
        c.frame_index = step
        return dof.camera_struct(c)

    cams = [cam_for(s) for s in range(args.warmup + args.steps)]
    out = torch.empty((w.H, w.W, 4), dtype=torch.float32, device=dev)
    hist = dof.History(ctx, w.W, w.H, max_rays=spp, taa=args.taa)

    def step(s, h, g=None):
        gb = g if g is not None else gbs[s % CYCLE]
        dof.frame(ctx, scene, gb, None, None, h, out, cam_struct=cams[s], params_s=pstruct)

    # session start (untimed): the autotuners pick the BVH build (PLOC radius), the
    # tree the rays traverse and the tracer's launch shape -- or --settings pins them
    t0 = time.perf_counter()
    pinned = parse_settings(args.settings)
    if pinned:
        ctx.set_ploc_radius(pinned["ploc_radius"])
        scene.close()
        scene = dof.Scene(ctx, w.scene)
        info = scene.info()
        tuned = {k: pinned[k] for k in tune.DEFAULT}
        ctx.set_trace(**tuned)
        tuned = dict(tuned, ploc_radius=pinned["ploc_radius"], pinned=True)
        gsel = dict(gather_block=pinned["main_filter_block"], main_form=pinned["main_filter_form"],
                    recon_block=pinned["recon_block"])
        ctx.set_gather(block=gsel["gather_block"], main_form=gsel["main_form"], recon_block=gsel["recon_block"])
    else:
        # the tracer first (on the default tree), then the tree under that tracer (the
        # trees' quality differs between radii, and by traversal), then the tracer again
        # on the chosen tree
        fixed_width = (args.bvh_width,) if args.bvh_width else None
        first, _ = tune.tune_trace(ctx, lambda k: step(k % len(cams), hist), frames=4, widths=fixed_width)
        widths = (args.bvh_width,) if args.bvh_width else ((2,) if first.get("packets") else (4, 2))
        scene.close()
        scene, tuned_bvh, _ = tune.tune_scene(
            ctx, w.scene, lambda sc, k: dof.frame(ctx, sc, gbs[k % CYCLE], None, None, hist, out,
                                                  cam_struct=cams[k % len(cams)], params_s=pstruct), widths=widths)
        info = scene.info()
        tuned, _ = tune.tune_trace(ctx, lambda k: step(k % len(cams), hist), frames=4, rounds=1,
                                   widths=fixed_width or ((2,) if first.get("packets") else None), start=first)
        tuned = dict(tuned, ploc_radius=tuned_bvh["ploc_radius"])
        # the 81-tap gathers' block shape and the main filter's form
        gsel, _ = tune.tune_gathers(ctx, lambda k: step(k % len(cams), hist), frames=4)
    gathers = dict(main_filter_block=list(gsel["gather_block"]), main_filter_form=gsel["main_form"],
                   recon_block=list(gsel["recon_block"]))
    tune_s = time.perf_counter() - t0
    hist.reset()

    dist = world > 1
    if dist:
        import torch.distributed as tdist
    for s in range(args.warmup):
        step(s, hist)
    torch.cuda.synchronize()
    if dist:
        tdist.barrier()
    # ---- timed region (device events on the launching stream)
    e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed")      # profilers select the timed frames by this range
        launches0 = dof.launch_count()           # the library's own tally of enqueued kernels
        e_start.record(stream)
        for s in range(args.warmup, args.warmup + args.steps):
            step(s, hist)
        e_end.record(stream)
        launches = dof.launch_count() - launches0
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    if dist:
        tdist.barrier()
    ms = max_over_ranks(e_start.elapsed_time(e_end))
    st = hist.stats()
    ms_per_step = ms / args.steps
    value = job_value(args.steps, ms, world)

    # ---- the FP16-storage variant over the same steps (another session history), with
    # the gathers' launch settings tuned for it (its texels are smaller)
    p16 = dof.params_struct(dict(prm, image_storage=1))
    h16 = dof.History(ctx, w.W, w.H, max_rays=spp, taa=args.taa)
    if pinned:
        gsel16 = gsel
    else:
        gsel16, _ = tune.tune_gathers(ctx, lambda k: dof.frame(ctx, scene, gbs[k % CYCLE], None, None, h16, out,
                                                              cam_struct=cams[k % len(cams)], params_s=p16), frames=4)
        h16.reset()
    for s in range(args.warmup):
        dof.frame(ctx, scene, gbs[s % CYCLE], None, None, h16, out, cam_struct=cams[s], params_s=p16)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for s in range(args.warmup, args.warmup + args.steps):
        dof.frame(ctx, scene, gbs[s % CYCLE], None, None, h16, out, cam_struct=cams[s], params_s=p16)
    f1.record(stream)
    torch.cuda.synchronize()
    ms16 = max_over_ranks(f0.elapsed_time(f1))
    fp16 = {"ms_per_step": round(ms16 / args.steps, 4), "value": round(job_value(args.steps, ms16, world), 2),
            "unit": "frames/s", "storage": "colour image buffers FP16, FP32 arithmetic/depth/CoC/history",
            "gathers": dict(main_filter_block=list(gsel16["gather_block"]), main_filter_form=gsel16["main_form"],
                            recon_block=list(gsel16["recon_block"]))}
    del h16
    # the FP32 session's gather settings again for the instrumented pass
    ctx.set_gather(block=gsel["gather_block"], main_form=gsel["main_form"], recon_block=gsel["recon_block"])

    # ---- instrumented pass: per-kernel device times and the tracer's node visits and
    # triangle tests over the same kind of steps
    ctx.set_trace(stats=True)
    htime = dof.History(ctx, w.W, w.H, max_rays=spp, timing=True, taa=args.taa)
    for s in range(args.warmup):
        step(s, htime)
    htime.kernel_times()
    ktot = {k: 0.0 for k in dof.KERNELS}
    nk = 0
    rays = masked = visits = tests = 0
    s = args.warmup
    while s < args.warmup + args.steps:
        for _ in range(min(32, args.warmup + args.steps - s)):
            step(s, htime)
            s += 1
        km, n = htime.kernel_times()
        for k, v in km.items():
            ktot[k] += v
        nk += n
        fs = htime.stats()
        rays += fs.rays
        masked += fs.masked_pixels
        visits += fs.node_visits
        tests += fs.tri_tests
    kavg = {k: v / nk for k, v in ktot.items()}
    if not args.taa:
        kavg["k_taa"] = 0.0             # no TAA launch: its timing slot only brackets nothing
    if int(prm["ray_mode"]) != 1:
        kavg["k_edges"] = 0.0
    for k in ("k_var_blur", "k_mips", "k_tile_dilate"):
        kavg[k] = 0.0                    # fused into other kernels: their slots bracket nothing
    n_samples = math.ceil(args.steps / 32)
    rays_per_frame = rays / n_samples
    masked_per_frame = masked / n_samples

    # ---- end to end through the C ABI with host buffers
    ctx.set_trace(stats=False)
    pin = []
    for g in gbs:
        pin.append(dict(color=g["color"].cpu().pin_memory(), depth=g["depth"].cpu().pin_memory()))
        if int(prm["ray_mode"]) == 1:
            pin[-1]["normal"] = g["normal"].cpu().pin_memory()
    hout = torch.empty((w.H, w.W, 4), dtype=torch.float32).pin_memory()
    he = dof.History(ctx, w.W, w.H, max_rays=spp, taa=args.taa)
    h2d = sum(t.numel() * 4 for t in pin[0].values())
    d2h = hout.numel() * 4

    # through dof_frame_host: each frame's G-buffer is copied in from pinned host memory
    # and its image copied out to pinned host memory, on the library's copy streams, so
    # the copies of one frame overlap the passes of its neighbours
    def e2e_step(s):
        dof.frame_host(ctx, scene, pin[s % CYCLE], None, None, he, hout, cam_struct=cams[s], params_s=pstruct)

    for s in range(args.warmup):
        e2e_step(s)
    dof.frame_host_join(he)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s in range(args.warmup, args.warmup + args.steps):
        e2e_step(s)
    dof.frame_host_join(he, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks(e0.elapsed_time(e1))
    e2e = {"value": job_value(args.steps, ms_e2e, world), "unit": "frames/s", "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(d2h)}

    # ---- roofline of the dominant kernel
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    N = (w.W // 2) * (w.H // 2)
    units = {"N": N, "M": masked_per_frame, "R": rays_per_frame, "P": w.W * w.H}
    dom = max(kavg, key=lambda k: kavg[k])
    kern = {}
    for k, v in kavg.items():
        if v <= 0:
            continue
        e = {"ms": round(v, 5), "share": round(v / sum(kavg.values()), 4)}
        if k in BYTES:
            e["gbs"] = round(algo_bytes(k, units) / (v * 1e-3) / 1e9, 1)
        kern[k] = e
    clocks = clk.summary()
    sm_mhz = clocks.get("sm_mhz") or float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    fp32_peak = 2.0 * FP32_LANES_PER_SM * n_sm * sm_mhz * 1e6 / 1e12      # TFLOP/s, FMA = 2
    # warp packets always traverse the binary tree
    wide = tuned["bvh_width"] == 4 and not tuned.get("packets")
    trace_flop = (visits * FLOP_PER_NODE[4 if wide else 2] + tests * FLOP_PER_TRI) / n_samples
    tracer_key = "k_trace_packets" if tuned.get("packets") else f"k_trace_rays<{1 if wide else 0}>"
    dom_key = tracer_key if dom == "k_trace_rays" else dom
    traffic = PROFILED_TRAFFIC.get(args.config, {}).get(dom_key) if not args.size else None
    if dom == "k_trace_rays" and kavg[dom] > 0:
        achieved = trace_flop / (kavg[dom] * 1e-3) / 1e12
        roof = {"kernel": dom_key, "bound": "alu", "achieved": round(achieved, 3), "peak": round(fp32_peak, 2),
                "unit": "TFLOP/s", "frac": round(achieved / fp32_peak, 4), "traffic": traffic,
                "peak_source": f"derived: 2 x {FP32_LANES_PER_SM} FP32 lanes x {n_sm} SMs x {sm_mhz:.0f} MHz",
                "algorithmic_flop": int(trace_flop), "node_visits_per_ray": round(visits / max(1, rays), 2),
                "tri_tests_per_ray": round(tests / max(1, rays), 2)}
    elif dom in FLOP_PER_GATHER and kavg[dom] > 0:
        unit, per = FLOP_PER_GATHER[dom]
        flop = per * units[unit]
        achieved = flop / (kavg[dom] * 1e-3) / 1e12
        roof = {"kernel": dom, "bound": "alu", "achieved": round(achieved, 3), "peak": round(fp32_peak, 2),
                "unit": "TFLOP/s", "frac": round(achieved / fp32_peak, 4), "traffic": traffic,
                "peak_source": f"derived: 2 x {FP32_LANES_PER_SM} FP32 lanes x {n_sm} SMs x {sm_mhz:.0f} MHz",
                "algorithmic_flop": int(flop),
                "note": "81-tap gather, bound by issue slots and L1 together: FP32 operations counted per tap"}
    elif dom in BYTES:
        algo = algo_bytes(dom, units)
        achieved = algo / (kavg[dom] * 1e-3) / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(achieved / hbm_peak, 4), "traffic": traffic, "peak_source": peak_src,
                "algorithmic_bytes": int(algo)}
    else:
        roof = {"kernel": dom, "bound": "alu", "achieved": None, "peak": None, "unit": None, "frac": None,
                "traffic": None}
    # image passes vs HBM: the streaming passes (HBM-bound by design) together, and the
    # gather passes (81-tap filters: L1/issue-bound by nature, reported apart)
    def agg(names):
        names = [k for k in names if kavg.get(k, 0) > 0]
        b = sum(algo_bytes(k, units) for k in names)
        t = sum(kavg[k] for k in names)
        return b, t
    img_bytes, img_ms = agg(STREAMING)
    gat_bytes, gat_ms = agg(GATHERS)
    ray_bytes, ray_ms = agg(RAY_LIST)
    res = dict(metric=METRIC, value=round(value, 2), unit="frames/s", n_gpus=world, steps=args.steps,
               warmup=args.warmup, ms_per_step=round(ms_per_step, 4), higher_is_better=True, scaling="weak",
               vs_baseline=None, dtype="f32", data="synthetic",
               config=dict(workload=f"{w.name}: {w.W}x{w.H}, {info.n_tris} triangles (lawn + box field), "
                                    f"{w.intr['f_m'] * 1000:.0f} mm f/{w.intr['f_number']:g} focus "
                                    f"{w.intr['focus_m']:g} m, CoC radius <= {prm['max_coc_px']:g} px, {spp} spp, "
                                    f"16-frame dolly" + (", camera jitter + final TAA (blend 0.1)" if args.taa else "")
                                    + (", FP16 image storage" if args.image_storage == "f16" else ""),
                           resolution=[w.W, w.H], triangles=info.n_tris, spp=spp, bvh_depth=info.depth,
                           tracer=dict(tuned, tune_s=round(tune_s, 2)), gathers=gathers,
                           parallelism="replicas" if world > 1 else "single-gpu",
                           l2=f"inputs larger than L2: {CYCLE} distinct G-buffers cycled "
                              f"({CYCLE} x {w.W * w.H * 20 / 1e6:.0f} MB)"),
               roofline=roof, e2e=e2e, fp16_storage=fp16,
               # counted by the library over the timed steps: per frame the downscale (with the
               # counter reset), prefilter (with the tile dilation), main filter, median, mask,
               # trace, shade, accumulation, the fused RT resolve (variance blur, median, mip
               # pyramid), recon, composite (+ 2 edge kernels in adaptive mode, + the final TAA)
               gpu_launches=int(launches),
               clocks=clocks, kernel_ms=kern,
               image_passes={"streaming": {"kernels": STREAMING, "ms": round(img_ms, 4),
                                           "gbs": round(img_bytes / (img_ms * 1e-3) / 1e9, 1),
                                           "frac_of_hbm": round(img_bytes / (img_ms * 1e-3) / 1e9 / hbm_peak, 4)},
                             "gathers": {"kernels": GATHERS, "ms": round(gat_ms, 4),
                                         "gbs": round(gat_bytes / (gat_ms * 1e-3) / 1e9, 1),
                                         "bound": "L1 / issue (81-tap taps), see profiles/"},
                             "ray_list": {"kernels": RAY_LIST, "ms": round(ray_ms, 4),
                                          "gbs": round(ray_bytes / (ray_ms * 1e-3) / 1e9, 1) if ray_ms > 0 else None,
                                          "lens_grid": tuned.get("ray_grid"),
                                          "bound": "HBM in pixel order; one Philox lens sample per ray "
                                                   "when grouped by lens cell"}},
               mrays_per_s=round(rays_per_frame / (kavg.get("k_trace_rays", 0) * 1e-3) / 1e6, 1)
               if kavg.get("k_trace_rays", 0) > 0 else None,
               rays_per_frame=int(rays_per_frame), mask_fraction=round(masked_per_frame / N, 4),
               bvh_build_ms=round(bvh_ms, 2), gbuffer_ms=round(gbuf_ms, 3), gbuffer_producers=gbuf_cmp,
               coc_radius_px=reach, device_status=int(st.device_status))
    return res, w


# ---------------------------------------------------------------------------
# batched and served workloads
# ---------------------------------------------------------------------------

RES = [(1280, 720), (1920, 1080), (2560, 1440)]


def batch_sessions(n, res_cycle, tri_lo, tri_hi, seed, frames=8):
    """n sessions, each its own seeded lawn scene with log-uniform triangle count in
    [tri_lo, tri_hi] and the 35 mm lens of the 1080p workload."""
    import numpy as np
    from synth import make_workload
    from synth.scenes import scene_grass_field
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        W, H = res_cycle[k % len(res_cycle)]
        w = make_workload("c2", W=W, H=H, n_frames=frames, session=k)
        tris = float(np.exp(rng.uniform(np.log(tri_lo), np.log(tri_hi))))
        dens = tris / 495_802.0
        sd = 2000 + 100 * k
        w.scene_fn = (lambda sd=sd, dens=dens: scene_grass_field(sd, dens, near=(1.2, 4.7)))
        w._scene = None
        w.params = dict(w.params, seed=sd, albedo_seed=sd, session=k, max_coc_px=32.0 * W / 1920.0)
        out.append(w)
    return out


def run_batch(args):
    import torch
    from paper_2210_06158_gb300 import _build, dof, tune
    _build.build()
    dev = torch.device("cuda", 0)
    ctx = dof.Context(0)
    ctx.set_trace(stats=False)          # no node-visit counters in these timings
    ws = batch_sessions(32, RES, 200_000, 1_000_000, seed=4)
    S = []
    for w in ws:
        sc = dof.Scene(ctx, w.scene)
        gbs = []
        for f in range(w.n_frames):
            g = dof.gbuffer(ctx, sc, w.camera(f), w.params, w.W, w.H)
            del g["prim"]
            gbs.append(g)
        S.append(dict(w=w, sc=sc, gbs=gbs, hb=dof.History(ctx, w.W, w.H), hs=dof.History(ctx, w.W, w.H),
                      h16=dof.History(ctx, w.W, w.H), hgr=dof.History(ctx, w.W, w.H),
                      out=torch.empty((w.H, w.W, 4), device=dev),
                      p=dof.params_struct(w.params), p16=dof.params_struct(dict(w.params, image_storage=1)),
                      cams=[dof.camera_struct(w.camera(f)) for f in range(w.n_frames)]))
    tris = sum(s["sc"].info().n_tris for s in S)
    px = sum(s["w"].W * s["w"].H for s in S)
    torch.cuda.synchronize()

    def batched(step):
        f = step % 8
        dof.batch_frame(ctx, [dict(scene=s["sc"], gbuf=s["gbs"][f], cam=s["cams"][f], params=s["p"], hist=s["hb"],
                                   out=s["out"]) for s in S])

    def batched16(step):
        f = step % 8
        dof.batch_frame(ctx, [dict(scene=s["sc"], gbuf=s["gbs"][f], cam=s["cams"][f], params=s["p16"],
                                   hist=s["h16"], out=s["out"]) for s in S])

    def single(step):
        f = step % 8
        for s in S:
            dof.frame(ctx, s["sc"], s["gbs"][f], None, None, s["hs"], s["out"], cam_struct=s["cams"][f],
                      params_s=s["p"])

    # the autotuners pick the tracer's tree and launch shape and the gathers' launch
    # settings on the batch, and the gathers' again for the FP16-storage batch (untimed)
    t0 = time.perf_counter()
    tuned, _ = tune.tune_trace(ctx, batched, frames=2)
    gsel16, _ = tune.tune_gathers(ctx, batched16, frames=2)
    gsel, _ = tune.tune_gathers(ctx, batched, frames=2)
    tune_s = time.perf_counter() - t0
    for s in S:
        s["hb"].reset()
        s["h16"].reset()

    def gathers(g):
        return dict(main_filter_block=list(g["gather_block"]), main_filter_form=g["main_form"],
                    recon_block=list(g["recon_block"]))

    def graph_items(step):
        f = step % 8
        return [dict(scene=s["sc"], gbuf=s["gbs"][f], cam=s["cams"][f], params=s["p"], hist=s["hgr"], out=s["out"])
                for s in S]

    graph = dof.Graph(ctx, graph_items(0))     # captured once, after tuning

    def batched_graph(step):
        graph.launch(graph_items(step))

    res = {}
    for name, fn in (("batched", batched), ("batched_graph", batched_graph), ("per_frame", single),
                     ("batched_fp16", batched16)):
        if name == "batched_fp16":
            ctx.set_gather(block=gsel16["gather_block"], main_form=gsel16["main_form"],
                           recon_block=gsel16["recon_block"])
        for k in range(args.warmup):
            fn(k)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(0) as clk:
            l0 = dof.launch_count()
            e0.record()
            for k in range(args.warmup, args.warmup + args.steps):
                fn(k)
            e1.record()
            torch.cuda.synchronize()
            nl = dof.launch_count() - l0
        ms = e0.elapsed_time(e1)
        res[name] = dict(ms_per_step=ms / args.steps, frames_per_s=len(S) * args.steps / (ms / 1e3),
                         clocks=clk.summary(), launches=int(nl))
    line = dict(metric=METRIC, value=round(res["batched"]["frames_per_s"], 2), unit="frames/s", n_gpus=1,
                steps=args.steps, warmup=args.warmup, ms_per_step=round(res["batched"]["ms_per_step"], 3),
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32", data="synthetic",
                config=dict(workload=f"batched: 32 sessions, own lawn scenes 200k-1M triangles ({tris} total), "
                                     f"1280x720/1920x1080/2560x1440 cycled ({px / 1e6:.1f} Mpx per step), 8-frame dollies, "
                                     "one dof_batch_frame (one launch per pass) per step",
                            l2="inputs larger than L2: 256 distinct G-buffers",
                            tracer=dict(tuned, tune_s=round(tune_s, 2)), gathers=gathers(gsel)),
                per_frame_form=dict(frames_per_s=round(res["per_frame"]["frames_per_s"], 2),
                                    ms_per_step=round(res["per_frame"]["ms_per_step"], 3),
                                    note="plain FP32, one dof_frame per session"),
                batched_graph_form=dict(frames_per_s=round(res["batched_graph"]["frames_per_s"], 2),
                                        ms_per_step=round(res["batched_graph"]["ms_per_step"], 3),
                                        note="the same step captured once as a CUDA graph and replayed"),
                batched_fp16_form=dict(frames_per_s=round(res["batched_fp16"]["frames_per_s"], 2),
                                       ms_per_step=round(res["batched_fp16"]["ms_per_step"], 3),
                                       note="FP16 storage of the colour image buffers, FP32 arithmetic",
                                       gathers=gathers(gsel16)),
                gpu_launches=res["batched"]["launches"], clocks=res["batched"]["clocks"])
    return line


def run_budget(args):
    """Adaptive ray count (Eq. 4) on the 1080p workload with the ray cap m swept over
    1, 10, 30, 50 (the paper varies m the same way): rays, tracer and frame time per m
    and the least-squares slope of frame time over m.  The BVH is tuned once (at m = 10)
    and the tracer's settings at every m (untimed), as a session would."""
    import numpy as np
    import torch
    from paper_2210_06158_gb300 import _build, dof, tune
    from synth import make_workload
    _build.build()
    dev = torch.device("cuda", 0)
    w = make_workload("c2")
    ctx = dof.Context(0)
    ctx.set_trace(stats=False)          # no node-visit counters in these timings
    scene = dof.Scene(ctx, w.scene)
    gbs = []
    for k in range(CYCLE):
        g = dof.gbuffer(ctx, scene, w.camera(k % w.n_frames), w.params, w.W, w.H)
        del g["prim"]
        gbs.append(g)
    out = torch.empty((w.H, w.W, 4), dtype=torch.float32, device=dev)
    rows = []
    clk_all = None
    cams = [dof.camera_struct(w.camera(s % CYCLE % w.n_frames)) for s in range(args.warmup + args.steps)]
    p10 = dof.params_struct(dict(w.params, ray_mode=1, m=10))
    h10 = dof.History(ctx, w.W, w.H, max_rays=10)
    scene, tuned_bvh, _ = tune.tune_scene(
        ctx, w.scene, lambda sc, k: dof.frame(ctx, sc, gbs[k % CYCLE], None, None, h10, out, cam_struct=cams[k],
                                              params_s=p10))
    del h10
    for m in (1, 10, 30, 50):
        prm = dict(w.params, ray_mode=1, m=m)
        ps = dof.params_struct(prm)
        h = dof.History(ctx, w.W, w.H, max_rays=m)
        ht = dof.History(ctx, w.W, w.H, max_rays=m, timing=True)
        tuned, _ = tune.tune_trace(ctx, lambda k: dof.frame(ctx, scene, gbs[k % CYCLE], None, None, h, out,
                                                             cam_struct=cams[k % len(cams)], params_s=ps), frames=3)
        h.reset()
        for s in range(args.warmup):
            dof.frame(ctx, scene, gbs[s % CYCLE], None, None, h, out, cam_struct=cams[s], params_s=ps)
            dof.frame(ctx, scene, gbs[s % CYCLE], None, None, ht, out, cam_struct=cams[s], params_s=ps)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(0) as clk:
            e0.record()
            for s in range(args.warmup, args.warmup + args.steps):
                dof.frame(ctx, scene, gbs[s % CYCLE], None, None, h, out, cam_struct=cams[s], params_s=ps)
            e1.record()
            torch.cuda.synchronize()
        clk_all = clk.summary()
        ms = e0.elapsed_time(e1) / args.steps
        ht.kernel_times()
        rays = 0
        for s in range(args.warmup, args.warmup + args.steps):
            dof.frame(ctx, scene, gbs[s % CYCLE], None, None, ht, out, cam_struct=cams[s], params_s=ps)
            rays += ht.stats().rays
        km, n = ht.kernel_times()
        rows.append(dict(m=m, frame_ms=round(ms, 4), trace_ms=round(km["k_trace_rays"] / n, 4),
                         shade_ms=round(km["k_shade"] / n, 4), rays_per_frame=int(rays / args.steps),
                         rays_per_masked_pixel=round(rays / args.steps / max(1, ht.stats().masked_pixels), 3),
                         status=int(ht.stats().device_status), tracer=tuned))
        del h, ht
    mm = np.array([r["m"] for r in rows], float)
    fm = np.array([r["frame_ms"] for r in rows], float)
    slope = float(np.polyfit(mm, fm, 1)[0])
    r10 = next(r for r in rows if r["m"] == 10)
    return dict(metric=METRIC, value=round(1e3 / r10["frame_ms"], 2), unit="frames/s", n_gpus=1, steps=args.steps,
                warmup=args.warmup, ms_per_step=r10["frame_ms"], higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f32", data="synthetic",
                config=dict(workload="budget: the 1080p lawn workload in adaptive mode (Eq. 4), ray cap m in "
                                     "{1, 10, 30, 50}; value = frames/s at m = 10",
                            l2=f"inputs larger than L2: {CYCLE} distinct G-buffers cycled"),
                budget=rows, slope_ms_per_m=round(slope, 5), clocks=clk_all, bvh=tuned_bvh,
                paper_context="0.04-0.07 ms per unit m for the ray-trace pass on an RTX 2080 Ti (Table 2)")


SERVE_LOADS = (0.25, 0.5, 0.75, 1.0, 1.5)      # offered load as a fraction of the batched FP32 capacity


def run_serve(args):
    from paper_2210_06158_gb300 import _build
    from paper_2210_06158_gb300.serve import GpuExecutor, Server, SessionSpec, poisson_arrivals
    import torch
    _build.build()
    res = [(1280, 720), (1920, 1080), (2560, 1440), (3840, 2160)]
    ws = batch_sessions(64, res, 100_000, 2_000_000, seed=5, frames=4)
    duration = float(os.environ.get("DOF_SERVE_SECONDS", "1.5"))
    ex = GpuExecutor(budget_bytes=40 << 30, gbuf_ring=2)
    srv = Server(ex, max_batch=32)
    specs = {}
    t0 = time.time()
    for k, w in enumerate(ws):
        specs[k] = SessionSpec(f"s{k}", w.W, w.H, 30.0 if k % 2 == 0 else 60.0, scene=w.scene, params=w.params,
                               poses=w.poses, intr=w.intr)
        srv.admit(k, specs[k])
    setup_s = time.time() - t0
    # start-up: the tracer's and the gathers' settings tuned on batched steps of the
    # admitted sessions (the gathers' once per image storage)
    t1 = time.time()
    tracer = ex.tune()
    tracer = dict(tracer, tune_s=round(time.time() - t1, 2))
    gathers = dict(ex.gathers)

    def gather_rec(g):
        return dict(main_filter_block=list(g["gather_block"]), main_filter_form=g["main_form"],
                    recon_block=list(g["recon_block"]))
    admitted = {k: v for k, v in specs.items() if k in srv.specs}
    nominal = {k: v.fps for k, v in admitted.items()}
    offered_nominal = sum(nominal.values())

    def serve_at(scale, seed):
        """Poisson requests at `scale` x the nominal 30/60 fps of every session."""
        for k, v in admitted.items():
            v.fps = nominal[k] * scale
        arr = poisson_arrivals(seed, admitted, duration_s=duration)
        st = srv.run(arr)
        torch.cuda.synchronize()
        return st, len(arr)

    def point(st, n_req, offered):
        return dict(offered_frames_per_s=round(offered, 1), frames_per_s=round(st["frames_per_s"], 2),
                    p50_ms=round(st["p50_ms"], 3), p99_ms=round(st["p99_ms"], 3), frames=st["frames"],
                    requests=n_req, superseded=round(st["dropped"] / max(1, n_req), 4),
                    mean_batch=round(st["mean_batch"], 2))

    forms = [("batched_fp32", False, False), ("batched_fp16", False, True), ("per_frame_fp32", True, False)]
    out = {}
    capacity = None
    with ClockSampler(0) as clk:
        for name, per_frame, fp16 in forms:
            ex.set_form(per_frame=per_frame, fp16=fp16)
            # capacity: the nominal 30/60 fps offer far more frames than one GPU renders
            st, n_req = serve_at(1.0, 6)
            cap = st["frames_per_s"]
            if capacity is None:
                capacity = cap           # the batched FP32 capacity sets the sweep's offered loads
            sweep = []
            for f in SERVE_LOADS:
                scale = f * capacity / offered_nominal
                st_f, n_f = serve_at(scale, 7 + int(100 * f))
                sweep.append(dict(point(st_f, n_f, scale * offered_nominal), load=f))
            out[name] = dict(capacity_frames_per_s=round(cap, 2), overload=point(st, n_req, offered_nominal),
                             sweep=sweep)
    n_rejected = len(srv.rejected)
    for k in list(srv.specs):
        srv.release(k)
    del ex, srv
    torch.cuda.synchronize()
    # admission under a budget that binds: 8 GB admits only part of the 64 sessions
    ex8 = GpuExecutor(budget_bytes=8 << 30, gbuf_ring=2)
    ex8.ctx.set_trace(**{k: v for k, v in tracer.items() if k != "tune_s"})
    ex8.gathers = gathers
    ex8.set_form(per_frame=False, fp16=False)
    srv8 = Server(ex8, max_batch=32)
    specs8 = {k: SessionSpec(f"s{k}", w.W, w.H, 30.0 if k % 2 == 0 else 60.0, scene=w.scene, params=w.params,
                             poses=w.poses, intr=w.intr) for k, w in enumerate(ws)}
    for k in specs8:
        srv8.admit(k, specs8[k])
    adm8 = {k: v for k, v in specs8.items() if k in srv8.specs}
    st8 = srv8.run(poisson_arrivals(9, adm8, duration_s=duration))
    budget8 = dict(budget_gb=8, admitted=len(adm8), rejected=len(srv8.rejected),
                   bytes_in_use=int(ex8.ctx.bytes_in_use), frames_per_s=round(st8["frames_per_s"], 2),
                   p50_ms=round(st8["p50_ms"], 3), p99_ms=round(st8["p99_ms"], 3))
    for k in list(srv8.specs):
        srv8.release(k)
    b = out["batched_fp32"]
    half = next(p for p in b["sweep"] if p["load"] == 0.5)
    line = dict(metric=METRIC, value=b["capacity_frames_per_s"], unit="frames/s", n_gpus=1,
                steps=b["overload"]["frames"], warmup=0, ms_per_step=None, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f32", data="synthetic",
                config=dict(workload="serving: 64 sessions, Poisson frame requests (nominal 30/60 fps), "
                                     f"{duration:g} s per point, 1280x720..3840x2160, lawn scenes 100k-2M "
                                     "triangles, 40 GB device budget, continuous batching (<= 32 per launch, "
                                     "2 streams)", tracer=tracer,
                            gathers={"fp32": gather_rec(gathers[False]), "fp16": gather_rec(gathers[True])}),
                served=dict(p50_ms_at_half_load=half["p50_ms"], p99_ms_at_half_load=half["p99_ms"],
                            admitted=len(admitted), rejected=n_rejected),
                forms=out, budget_8gb=budget8, setup_s=round(setup_s, 1), clocks=clk.summary(),
                note="value = batched FP32 capacity (served frames/s when every session always has a "
                     "request); sweep loads are fractions of it, the same offered loads for every form")
    return line


def parse_settings(text):
    """--settings "key=value,...": the tracer's and gathers' settings as the autotuners
    report them (config.tracer, config.gathers), the rest at their defaults; blocks as
    WxH.  None when not given."""
    if not text:
        return None
    from paper_2210_06158_gb300 import tune
    out = dict(tune.DEFAULT, ploc_radius=48, main_filter_block=(32, 8), main_filter_form=0, recon_block=(32, 8))
    for item in text.split(","):
        k, v = (s.strip() for s in item.split("="))
        if k not in out:
            raise SystemExit(f"--settings: unknown key {k!r} (keys: {', '.join(sorted(out))})")
        out[k] = tuple(int(x) for x in v.lower().split("x")) if k.endswith("_block") else int(v)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=64)
    ap.add_argument("--warmup", type=int, default=8)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c2", choices=["c1", "c2", "c3", "batch", "serve", "budget"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-c3", action="store_true",
                    help="skip the 4K sub-record of the default (c2) run")
    ap.add_argument("--taa", action="store_true",
                    help="camera jitter (Halton 2, 3) and the final TAA pass with blend 0.1")
    ap.add_argument("--size", default=None,
                    help="WxH: the workload's scene, lens and camera path at another resolution (profiler captures)")
    ap.add_argument("--image-storage", default="f32", choices=["f32", "f16"],
                    help="colour image buffers of the timed session (f16: the FP16-storage form; profiler captures)")
    ap.add_argument("--bvh-width", type=int, default=None, choices=[2, 4],
                    help="traverse this tree width instead of the autotuner's choice (profiler captures)")
    ap.add_argument("--settings", default=None,
                    help="pin the tracer and gather settings instead of autotuning them, e.g. "
                         "ploc_radius=16,bvh_width=2,ray_grid=1,packets=1,main_filter_block=64x4 "
                         "(keys as in config.tracer / config.gathers; reproduces a tuned run under a profiler); "
                         "the main workload only, the 4K sub-record is still autotuned")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world = int(os.environ.get("WORLD_SIZE", 1))
    rank = int(os.environ.get("RANK", 0))

    if args.impl == "reference":
        if rank != 0:
            return 0
        from synth import make_workload
        # the batched, served and budget modes run the 1080p workload's frames
        w = make_workload(args.config if args.config in ("c1", "c2", "c3") else "c2")
        fps, desc, threads, times, frac = oracle_sample(w, steps=args.warmup + args.steps if args.steps <= 16 else None)
        timed = times[min(len(times) - 1, args.warmup):] or times
        ms = statistics.median(timed) / frac * 1e3
        line = dict(metric=METRIC, value=round(1e3 / ms, 5), unit="frames/s", n_gpus=world, steps=len(timed),
                    warmup=min(args.warmup, len(times) - len(timed)), ms_per_step=round(ms, 2),
                    higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                    impl="reference",
                    config=dict(workload=f"{w.name}: {w.W}x{w.H} (FP64 oracle on the host cores)"),
                    cpu_baseline=dict(value=round(1e3 / ms, 5), unit="frames/s", cores=threads, kind="oracle",
                                      sample=desc),
                    e2e=dict(value=round(1e3 / ms, 5), unit="frames/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
        print(json.dumps(line), flush=True)
        return 0

    if args.config in ("batch", "serve", "budget"):
        if rank == 0:
            line = {"batch": run_batch, "serve": run_serve, "budget": run_budget}[args.config](args)
            print(json.dumps(line), flush=True)
        return 0
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("gloo")
    res, w = run_ours(args, rank, world)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(w)
    if args.config == "c2" and not args.size and not args.no_c3:
        # the 4K workload (3840x2160, 4 spp) with the same timing method: its own frames/s,
        # kernel times, image-pass rooflines, end-to-end figure and clocks
        import copy
        a3 = copy.copy(args)
        a3.config, a3.steps = "c3", min(args.steps, C3_STEPS)
        a3.settings = None          # --settings pins the run's main workload only
        r3, w3 = run_ours(a3, rank, world)
        keep = ("value", "unit", "steps", "warmup", "ms_per_step", "config", "roofline", "e2e", "fp16_storage",
                "gpu_launches", "clocks", "kernel_ms", "image_passes", "mrays_per_s", "rays_per_frame",
                "mask_fraction", "coc_radius_px", "device_status")
        res["c3"] = {k: r3[k] for k in keep}
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            res["c3"]["cpu_baseline"] = cpu_baseline(w3, budget_s=10.0, single_steps=1)
    if world > 1:
        import torch.distributed as tdist
        tdist.barrier()
        tdist.destroy_process_group()
    if rank == 0:
        print(json.dumps(res), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
