"""Autotuners of the ray tracer -- the BVH build (PLOC search radius), the persistent
tracer's tree width, work order, launch shape and scheduling -- and of the 81-tap
gathers' launch shape and main-filter form.

The knobs (the tree the rays traverse: binary or 4-wide; the order the tracer takes
a block's rays in: grouped by lens cell on a g x g grid, or pixel by pixel; the
traversal stack depth, which the launch raises to what the tree needs; 128-thread
blocks per SM, idle lanes that trigger a refill, traversal steps between refill
checks; warp packets over the binary tree instead of one ray per lane) change only
the speed of dof_frame, never its result (the closest hit does not depend on the
tree's shape).
`tune_trace` times a few frames of the caller's own session for each candidate
(coordinate descent from the defaults, CUDA events on the session's stream) and
leaves the fastest setting on the context.  Every candidate is timed on the same
frames (run_frame(0) .. run_frame(frames - 1), after one warm-up run_frame(0)), so a
moving camera does not favour the settings that happened to get the cheaper frames;
a candidate that beats the incumbent by more than 1% replaces it only if a second
timing of both confirms it.
"""

from __future__ import annotations

SPACE = {
    "bvh_width": [4, 2],
    "ray_grid": [4, 1, 2, 8, 12, 16],
    "stack": [96, 64, 32],
    "blocks_per_sm": [4, 6, 8, 12, 16],
    "refill_idle": [4, 8, 12, 16, 24],
    "steps": [8, 16, 32, 64],
    "packets": [0, 1],
}
DEFAULT = {"bvh_width": 4, "ray_grid": 4, "stack": 96, "blocks_per_sm": 8, "refill_idle": 16, "steps": 64,
           "packets": 0}


def _warm(run_frame, frames, st):
    """Frames 0 .. frames - 1 untimed, so that the session's history is in its steady
    state before any candidate is timed (in the adaptive mode of Eq. 4 the first frames
    of a fresh history trace fewer rays)."""
    for f in range(frames):
        run_frame(f)
    sync = getattr(st, "synchronize", None)
    if sync is not None:
        sync()


def _time_frames(run_frame, frames, st):
    """Warm-up frame 0, then the CUDA-event time of frames 0 .. frames - 1 (ms per frame)."""
    import torch
    run_frame(0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for f in range(frames):
        run_frame(f)
    e1.record(st)
    e1.synchronize()
    return e0.elapsed_time(e1) / frames


def tune_trace(ctx, run_frame, frames=6, rounds=2, stream=None, widths=None, start=None):
    """run_frame(k) enqueues frame k of a representative session on `stream` (or the
    current stream); `widths` restricts the tree widths searched (default: all); `start`
    is the search's starting point (default: DEFAULT).  Returns (best settings,
    {settings tuple: ms per frame})."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    space = dict(SPACE, bvh_width=list(widths)) if widths else SPACE
    best = dict(start or DEFAULT)
    best = {k: best[k] for k in DEFAULT}
    if best["bvh_width"] not in space["bvh_width"]:
        best["bvh_width"] = space["bvh_width"][0]
    seen = {}

    def canon(cfg):
        # warp packets traverse the binary tree whatever the width says
        return dict(cfg, bvh_width=2) if cfg.get("packets") and 2 in space["bvh_width"] else cfg

    def measure(cfg, fresh=False):
        key = tuple(sorted(cfg.items()))
        if key in seen and not fresh:
            return seen[key]
        ctx.set_trace(**cfg)
        seen[key] = _time_frames(run_frame, frames, st)
        return seen[key]

    _warm(run_frame, frames, st)
    best_ms = measure(best)
    for _ in range(rounds):
        improved = False
        for name, values in space.items():
            for v in values:
                cand = canon(dict(best, **{name: v}))
                ms = measure(cand)
                if ms < best_ms * 0.99:
                    ms2, inc2 = measure(cand, fresh=True), measure(best, fresh=True)
                    if ms2 < inc2 * 0.99:
                        best, best_ms, improved = cand, ms2, True
                    else:
                        best_ms = inc2
        if not improved:
            break
    ctx.set_trace(**best)
    return best, seen


GATHER_SPACE = {
    "gather_block": [(32, 8), (16, 16), (64, 4), (32, 4), (16, 8), (32, 16), (64, 8)],
    "main_form": [0, 1, 2, 3],
    "recon_block": [(32, 8), (16, 16), (64, 4), (32, 4), (16, 8), (32, 16), (64, 8)],
}
GATHER_DEFAULT = {"gather_block": (32, 8), "main_form": 0, "recon_block": (32, 8)}


def tune_gathers(ctx, run_frame, frames=4, rounds=2, stream=None):
    """The 81-tap gathers' launch shapes (block of the main filter, block of the
    reconstruction) and the main filter's form (halo tile in shared memory up to 64 KB,
    through L1, halo tile up to the SM's opt-in shared memory, or columns of four pixels
    through L1): coordinate descent
    over GATHER_SPACE from GATHER_DEFAULT with the same timing rules as tune_trace.
    Returns (best settings, {settings tuple: ms per frame}); the context keeps the best."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    best = dict(GATHER_DEFAULT)
    seen = {}

    def apply(cfg):
        ctx.set_gather(block=cfg["gather_block"], main_form=cfg["main_form"], recon_block=cfg["recon_block"])

    def measure(cfg, fresh=False):
        key = tuple(sorted(cfg.items()))
        if key in seen and not fresh:
            return seen[key]
        apply(cfg)
        seen[key] = _time_frames(run_frame, frames, st)
        return seen[key]

    _warm(run_frame, frames, st)
    best_ms = measure(best)
    for _ in range(rounds):
        improved = False
        for name, values in GATHER_SPACE.items():
            for v in values:
                cand = dict(best, **{name: v})
                ms = measure(cand)
                if ms < best_ms * 0.99:
                    ms2, inc2 = measure(cand, fresh=True), measure(best, fresh=True)
                    if ms2 < inc2 * 0.99:
                        best, best_ms, improved = cand, ms2, True
                    else:
                        best_ms = inc2
        if not improved:
            break
    apply(best)
    return best, seen


# PLOC search radii tried per scene: on the grass workloads the tree quality does not
# follow the radius (node tests per ray vary by up to a third between neighbouring
# radii), so several are built and the fastest kept
SCENE_RADII = [8, 12, 16, 24, 32, 40, 48, 56, 64, 96, 128, 192]


def tune_scene(ctx, host_scene, run_frame, radii=None, widths=(4, 2), frames=4, stream=None):
    """Build the scene's BVH with each PLOC search radius and time `frames` frames with
    each tree width; keep the fastest.  run_frame(scene, k) enqueues frame k of a
    representative session with the given device scene (the hits, hence the images,
    do not depend on the tree).  Returns (device scene, {"ploc_radius", "bvh_width"},
    {(radius, width): ms per frame}); the context keeps the chosen width."""
    import torch
    from . import dof
    st = stream if stream is not None else torch.cuda.current_stream()
    best, best_ms, best_scene = None, float("inf"), None
    seen = {}
    for r in (radii or SCENE_RADII):
        ctx.set_ploc_radius(r)
        sc = dof.Scene(ctx, host_scene)
        if not seen:
            _warm(lambda f: run_frame(sc, f), frames, st)
        for wdt in widths:
            ctx.set_bvh_width(wdt)
            ms = _time_frames(lambda f: run_frame(sc, f), frames, st)
            seen[(r, wdt)] = ms
            if ms < best_ms:
                best_ms, best = ms, {"ploc_radius": r, "bvh_width": wdt}
        if best_scene is None or best["ploc_radius"] == r:
            if best_scene is not None and best_scene is not sc:
                best_scene.close()
            best_scene = sc
        else:
            sc.close()
    ctx.set_ploc_radius(best["ploc_radius"])
    ctx.set_bvh_width(best["bvh_width"])
    return best_scene, best, seen
