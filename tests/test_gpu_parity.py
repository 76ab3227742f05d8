"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same seeded
inputs: every intermediate of the frame, hit ids, and the final image."""

import math

import numpy as np
import pytest

import oracle
from synth import make_workload, plane_scene, tiny_scene, Camera, camera_pose
from synth.scenes import Workload, default_params

from parity import (GpuRunner, classify_hits, dilate, mask_ties, full_res, max_abs, max_hdr, oracle_inputs, psnr,
                    taint_radius, threshold_ties, weight_ties)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2210_06158_gb300 import _build
    _build.build()
    oracle.build()


def run_sequence(w, n_frames=1, params=None, report=None, tol_img=2e-3, gbuf_f16=False, ctx=None):
    """Frames 0..n-1 of workload w on both sides; asserts parity frame by frame.
    gbuf_f16: the kernels take colour and normal as half planes (DOF_FMT_F16) and the
    oracle the same values widened to float.  ctx: a context with its options set
    (default: a fresh one)."""
    params = dict(params or w.params)
    w.params = params
    osc = oracle.Scene(w.scene)
    gpu = GpuRunner(w, params, ctx=ctx)
    ohist = oracle.History(w.W, w.H)
    H2, W2 = w.H // 2, w.W // 2
    rt_r = taint_radius(params)
    taint_h = np.zeros((H2, W2), bool)
    stats = []
    # per-pixel blurred-variance error of the previous frame: Eq. 4 reads that variance
    e_var_prev_px = np.zeros((H2, W2))
    adaptive = int(params["ray_mode"]) == 1
    m_rays = float(params["m"])
    for k in range(n_frames):
        cam = w.camera(k)
        gb = oracle.gbuffer_f32(oracle.gbuffer(osc, cam, params, w.W, w.H))
        gb_dev = gb
        if gbuf_f16:
            gb_dev = dict(gb, color=gb["color"].astype(np.float16), normal=gb["normal"].astype(np.float16))
            gb = dict(gb, color=gb_dev["color"].astype(np.float32), normal=gb_dev["normal"].astype(np.float32))
        hist0 = ohist.copy()
        ref = oracle.frame(osc, cam, params, w.W, w.H, gb, ohist)
        got = gpu.frame(cam, gb_dev)
        # ---- ray counts.  The mask may differ only on tiles whose dilated near radius
        # lies within rounding of the threshold.  In adaptive mode each side's count is
        # clamp(ceil(x_f), 1, m) of its own x_f (Eq. 4); x_f may differ per pixel by what
        # the errors of its inputs explain -- the edge measure x_n and the previous
        # frame's blurred variance times var_w_mask, both scaled by m -- plus the FP32
        # rounding of x_f itself.  A count then differs only where an integer lies
        # between the two x_f values, i.e. where the count is decided on a rounding tie.
        mask_g, mask_o = got["nrays"] > 0, ref["nrays"] > 0
        tile_ties = mask_ties(ref, params)
        assert not (mask_g != mask_o)[~tile_ties].any()
        both = mask_g & mask_o
        if adaptive:
            xg = got["xf"].astype(np.float64)
            assert np.array_equal(got["nrays"][mask_g], np.clip(np.ceil(xg), 1, m_rays).astype(np.int32)[mask_g])
            d_xn = np.abs(got["xn"].astype(np.float64) - ref["xn"])
            xf_band = m_rays * (d_xn + float(params["var_w_mask"]) * e_var_prev_px) + 4e-7 * m_rays
            d_xf = np.abs(xg - ref["xf"])
            over = both & ~taint_h & (d_xf > xf_band)
            assert not over.any(), (int(over.sum()), float(d_xf[over].max()))
        else:
            assert np.array_equal(got["nrays"][both], ref["nrays"][both])
        n_forced = int((got["nrays"] != ref["nrays"]).sum())
        n_masked = int(mask_o.sum())
        # rounding ties of the count are rare: at most 1e-3 of the masked pixels
        assert n_forced <= max(2, 1e-3 * n_masked), (n_forced, n_masked)
        force = None
        if n_forced:
            # either count is valid there: the oracle reruns the frame with the kernel's
            # counts at those pixels, so everything downstream is compared in full
            force = np.where(got["nrays"] != ref["nrays"], got["nrays"], -1).astype(np.int32)
            ohist = hist0.copy()
            ref = oracle.frame(osc, cam, params, w.W, w.H, gb, ohist, nrays_force=force)
            assert np.array_equal(got["nrays"], ref["nrays"])
        # ---- hit ids: equal except where rounding can explain the difference (the
        # oracle's hit_check: the kernel's triangle is hit within rounding and no clean
        # hit lies certainly in front of it); such near ties are at most 1e-4 of the
        # rays (a floor of 2 for the small crops); the oracle then reruns the frame
        # with the kernel's hits for those rays
        n_rays, n_mis, n_bad, mism = classify_hits(osc, w, params, cam, got, ref)
        assert n_bad == 0, f"{n_bad} hit-id mismatches are not FP near ties"
        assert n_mis <= max(2, 1e-4 * n_rays), (n_mis, n_rays)
        if n_mis:
            mr_o = ref["ray_prim"].shape[2]
            valid = np.arange(mr_o)[None, None, :] < ref["nrays"][..., None]
            gp = got["ray_prim"][..., :mr_o]
            hforce = np.where(valid & (gp != ref["ray_prim"]), gp, -2).astype(np.int32)
            ohist = hist0.copy()
            ref = oracle.frame(osc, cam, params, w.W, w.H, gb, ohist, nrays_force=force, hit_force=hforce)
            valid_g = np.arange(gp.shape[2])[None, None, :] < ref["nrays"][..., None]
            assert np.array_equal(np.where(valid_g, gp, 0), np.where(valid_g, ref["ray_prim"], 0))
        # ---- post-process: same FP32 inputs on both sides
        assert np.array_equal(got["z_h"], ref["z_h"].astype(np.float32))
        assert max_hdr(got["pp_in"][..., :3], ref["pp_in"][..., :3]) < 1e-6
        assert max_abs(got["pp_in"][..., 3], ref["pp_in"][..., 3]) < 2e-5
        assert max_abs(got["tile_raw"], ref["tile_raw"]) < 2e-5
        assert max_abs(got["tile_dil"], ref["tile_dil"]) < 2e-5
        e_pre = max_hdr(got["pre"], ref["pre"])
        e_main = max_hdr(got["main_out"], ref["main_out"])
        e_med = max_hdr(got["pp_med"], ref["pp_med"])
        assert e_pre < 1e-4 and e_main < 5e-4 and e_med < 5e-4, (e_pre, e_main, e_med)
        # ---- mask
        ties = weight_ties(ref)
        e_xf = 0.0
        if adaptive:
            e_xn = max_abs(got["xn"], ref["xn"])
            e_xf = max_abs(got["xf"][~taint_h], ref["xf"][~taint_h])
            assert e_xn < 1e-4, e_xn
        st = got["stats"]
        assert st.device_status == 0
        assert st.rays == int(got["nrays"].sum())
        # ---- taint cone of the far-weight ties, carried through the history
        seed = ties
        taint_h = dilate(dilate(taint_h, 2) | seed, rt_r)
        ok = ~taint_h
        # a pixel's ray sums depend on its own rays only
        m = (ref["nrays"] > 0) & ~ties
        # h and the field colours absolute, the field CoC radii (up to rmax) relative
        e_rt = max_hdr(got["rt"][..., 1:8][m], ref["rt"][..., 1:8][m]) if m.any() else 0.0
        e_rb = (max_abs(got["rt"][..., 8:10][m], ref["rt"][..., 8:10][m]) /
                max(1.0, float(np.abs(ref["rt"][..., 8:10]).max()))) if m.any() else 0.0
        both_far = m & (got["rt"][..., 13] > 0) & (ref["rt"][..., 13] > 0)
        e_pf = (max_abs(got["rt"][..., 10:13][both_far], ref["rt"][..., 10:13][both_far]) /
                max(1.0, float(np.abs(ref["rt"][..., 10:13][both_far]).max()))) if both_far.any() else 0.0
        assert e_rt < 1e-4 and e_rb < 1e-4 and e_pf < 1e-4, (e_rt, e_rb, e_pf)
        e_crt = max_hdr(got["crt"][ok], ref["crt"][ok])
        e_ct = max_abs(got["ct"][ok], ref["ct"][ok])
        e_hist = max_abs(got["hist"][ok], ref["hist"][ok])
        e_var = max_abs(got["var_blur"][ok], ref["var_blur"][ok])
        e_rtm = max_hdr(got["rt_med"][ok], ref["rt_med"][ok])
        e_rec = max_hdr(got["recon"][ok], ref["recon"][ok])
        e_hist = max_hdr(got["hist"][..., [0, 1, 2, 3, 4, 5, 6, 7, 10, 11]][ok],
                         ref["hist"][..., [0, 1, 2, 3, 4, 5, 6, 7, 10, 11]][ok])
        rmax = 0.5 * float(params["max_coc_px"])
        e_ct = max(e_ct, max_abs(got["hist"][..., 8:10][ok], ref["hist"][..., 8:10][ok])) / max(1.0, rmax)
        assert e_crt < 5e-4 and e_hist < 5e-4 and e_rtm < 5e-4 and e_rec < 1e-3, (e_crt, e_hist, e_rtm, e_rec)
        # FP32 reprojection of a moving camera is accurate to ~1e-5 px, which mixes that
        # share of a (noisy) neighbour's history in; a static camera is exact.  The
        # luminance variance scales with the square of the radiance (emitters reach 8),
        # so the bound is relative to its magnitude where that exceeds 1
        var_scale = max(1.0, float(np.abs(ref["var_blur"][ok]).max())) if ok.any() else 1.0
        # c_t (relative to rmax): a moving camera reprojects in FP32, where pixel positions
        # carry the spacing of FP32 at the image size (1.2e-4 px at 1920 half-resolution
        # columns); times a CoC step of up to rmax between neighbouring pixels, that is
        # the reprojected c_t's error (4 spacings cover the projection's rounding steps)
        ct_tol = max(1e-4, 4.0 * float(np.spacing(np.float32(max(W2, H2))))) if cam_moved(cam) else 1e-4
        assert e_ct < ct_tol and e_var < (2e-5 if cam_moved(cam) else 1e-6) * var_scale, (e_ct, ct_tol, e_var,
                                                                                          var_scale)
        e_var_prev_px = np.where(ok, np.abs(got["var_blur"].astype(np.float64) - ref["var_blur"]), 0.0)
        # ---- final image (linear RGB)
        taint_f = full_res(taint_h, w.W, w.H)
        if "out_taa" in ref:
            # composite before the final TAA, then the resolved image (its history carries
            # the taint of earlier frames, dilated by the 3x3 clamp and the reprojection)
            e_comp = max_hdr(got["composite"][..., :3][~taint_f], ref["out"][..., :3][~taint_f])
            assert e_comp <= tol_img, e_comp
            taint_taa = taint_f if k == 0 else dilate(taint_taa | taint_f, 3)
            e_out = max_hdr(got["out"][..., :3][~taint_taa], ref["out_taa"][..., :3][~taint_taa])
            p = psnr(got["out"][..., :3], ref["out_taa"][..., :3])
        else:
            e_out = max_hdr(got["out"][..., :3][~taint_f], ref["out"][..., :3][~taint_f])
            p = psnr(got["out"][..., :3], ref["out"][..., :3])
        assert e_out <= tol_img, e_out
        assert p >= 50.0, p
        s = dict(frame=k, rays=n_rays, mismatches=n_mis, forced=n_forced, masked=n_masked, xf=e_xf,
                 tainted=float(taint_f.mean()), max_out=e_out, psnr=p,
                 pre=e_pre, main=e_main, rt=e_rt, crt=e_crt, recon=e_rec)
        stats.append(s)
        if report is not None:
            report.append(s)
    return stats


def cam_moved(cam):
    return any(not np.array_equal(np.asarray(getattr(cam, a), np.float32), np.asarray(getattr(cam, "prev_" + a), np.float32))
               for a in ("pos", "right", "up", "fwd"))


def _print(stats, name):
    for s in stats:
        print(f"[{name}] " + " ".join(f"{k}={v:.3g}" if isinstance(v, float) else f"{k}={v}" for k, v in s.items()))


def test_gbuffer_matches_oracle():
    from paper_2210_06158_gb300 import dof
    import torch
    for name, W, H in [("c1", 256, 144), ("c2", 322, 182)]:
        w = make_workload(name, W=W, H=H)
        cam = w.camera(0)
        osc = oracle.Scene(w.scene)
        ref = oracle.gbuffer(osc, cam, w.params, W, H)
        ctx = dof.Context(0)
        sc = dof.Scene(ctx, w.scene)
        got = dof.gbuffer(ctx, sc, cam, w.params, W, H)
        torch.cuda.synchronize()
        prim = got["prim"].cpu().numpy()
        bad = np.argwhere(prim != ref["prim"])
        for (j, i) in bad:
            d = oracle.pixel_dir(cam, W, H, i + 0.5, j + 0.5)
            assert osc.near_tie(np.asarray(cam.pos, np.float64), d, int(prim[j, i]), int(ref["prim"][j, i]))
        assert len(bad) <= max(2, 1e-4 * W * H)
        ok = prim == ref["prim"]
        hit = ok & (prim >= 0)
        col = got["color"].cpu().numpy()[..., :3]
        assert max_abs(col[ok], ref["color"][ok]) < 1e-5
        dep = got["depth"].cpu().numpy()
        rel = np.abs(dep[hit] - ref["depth"][hit]) / ref["depth"][hit]
        assert rel.max() < 2e-5
        assert np.all(np.isinf(dep[ok & (prim < 0)]))
        assert max_abs(got["normal"].cpu().numpy()[..., :3][ok], ref["normal"][ok]) < 1e-5


@pytest.mark.parametrize("builder,width", [("ploc", 4), ("ploc", 2), ("lbvh", 4)])
def test_gpu_hits_equal_brute_force_on_tiny_scenes(builder, width):
    """G-buffer ids against the oracle's all-triangle loop (no BVH on either side
    decides the answer), incl. shared-edge and coplanar ties; 0, 1 and 2 triangles;
    every tree builder and traversal width."""
    from paper_2210_06158_gb300 import dof
    import torch
    ctx = dof.Context(0)
    ctx.set_bvh_builder(builder)
    ctx.set_bvh_width(width)
    pose = camera_pose((0.0, 0.0, 0.0), pitch_deg=0.0)
    cam = Camera.from_poses(dict(f_m=0.05, f_number=2.0, focus_m=3.0, sensor_w_m=0.036), pose)
    W, H = 96, 64
    for n in [0, 1, 2, 7, 64, 200]:
        s = tiny_scene(500 + n, n, ties=n >= 8)
        osc = oracle.Scene(s)
        sc = dof.Scene(ctx, s)
        got = dof.gbuffer(ctx, sc, cam, default_params(), W, H)
        torch.cuda.synchronize()
        prim = got["prim"].cpu().numpy()
        n_bad = 0
        for j in range(H):
            for i in range(W):
                d = oracle.pixel_dir(cam, W, H, i + 0.5, j + 0.5)
                o = np.zeros(3)
                want, _ = osc.closest(o, d, brute=True)
                if prim[j, i] != want and not osc.near_tie(o, d, int(prim[j, i]), want):
                    n_bad += 1
        assert n_bad == 0, (n, n_bad)


def test_frame_parity_c1():
    stats = run_sequence(make_workload("c1"))
    _print(stats, "c1")


def test_frame_parity_bright_bokeh():
    """Emissive spheres out of focus in front of and behind the focus plane (the bright
    path of the main filter and the composite), 85 mm f/1.2, 4 spp, 3 frames of a dolly."""
    w = make_workload("bokeh", n_frames=3)
    osc = oracle.Scene(w.scene)
    cam = w.camera(0)
    gb = oracle.gbuffer_f32(oracle.gbuffer(osc, cam, w.params, w.W, w.H))
    fr = oracle.frame(osc, cam, w.params, w.W, w.H, gb)
    assert fr["main_out"][..., 3].max() > 0.5          # bright taps reach the gather
    stats = run_sequence(w, 3)
    _print(stats, "bokeh")


@pytest.mark.parametrize("blades,name,W,H", [(6, "c3", 384, 216), (5, "bokeh", None, None)])
def test_frame_parity_polygonal_aperture(blades, name, W, H):
    """A regular n-gon aperture (a hexagon, and the odd pentagon on the bright-bokeh
    scene): lens samples uniform over it, the 81-tap kernels of the main filter and the
    reconstruction on it, sampleAlpha over its area; two frames against the oracle."""
    w = make_workload(name, n_frames=2) if W is None else make_workload(name, W=W, H=H, n_frames=2)
    prm = dict(w.params, aperture_blades=blades)
    # the shape changes what the oracle computes, so the comparison below is not vacuous
    osc = oracle.Scene(w.scene)
    cam = w.camera(0)
    gb = oracle.gbuffer_f32(oracle.gbuffer(osc, cam, prm, w.W, w.H))
    circ = oracle.frame(osc, cam, w.params, w.W, w.H, gb)
    poly = oracle.frame(osc, cam, prm, w.W, w.H, gb)
    assert np.abs(poly["main_out"] - circ["main_out"]).max() > 1e-2
    assert np.abs(poly["out"] - circ["out"]).max() > 1e-2
    stats = run_sequence(w, 2, prm)
    _print(stats, f"{name}-{blades}-gon")


@pytest.mark.parametrize("mode", [0, 1])
def test_frame_parity_half_gbuffer(mode):
    """A G-buffer whose colour and normal planes are half precision (DOF_FMT_F16), in the
    fixed and the adaptive ray mode (which reads the normals), 3 frames of the dolly."""
    w = make_workload("c2", W=256, H=144, n_frames=3)
    stats = run_sequence(w, 3, dict(w.params, ray_mode=mode, m=6), gbuf_f16=True)
    _print(stats, f"c2-f16-gbuffer-mode{mode}")


def test_frame_parity_ragged_dolly_with_history():
    """The lawn scene at 250x142 (125x71 hpx: ragged 8x8 tiles in both directions),
    4 frames of the dolly: camera motion, reprojection, history."""
    w = make_workload("c2", W=250, H=142, n_frames=4)
    stats = run_sequence(w, 4)
    _print(stats, "c2-250x142")


@pytest.mark.parametrize("moving", [True, False])
def test_frame_parity_jitter_and_taa(moving):
    """Camera jitter (Section 3.1.2) and the final TAA (Section 3.4): jittered pixel rays
    and G-buffer, reprojection minus the previous jitter, TAA history clamped to the
    current neighbourhood; a moving dolly and a static pose with only the jitter moving."""
    w = make_workload("c2", W=256, H=144, n_frames=4)
    if not moving:
        w.poses = [w.poses[0]] * 4
    w.jitter = True
    prm = dict(w.params, taa_alpha=0.1)
    stats = run_sequence(w, 4, prm)
    _print(stats, "c2-taa" + ("" if moving else "-static"))


def test_frame_parity_static_accumulation():
    """Static camera over 4 frames (the EMA at 0.95 with new lens samples per frame)."""
    w = make_workload("c1", W=160, H=90)
    w.poses = [w.poses[0]] * 4
    stats = run_sequence(w, 4)
    _print(stats, "c1-static")


def test_frame_parity_4spp_c3_lens():
    w = make_workload("c3", W=384, H=216, n_frames=2)
    stats = run_sequence(w, 2)
    _print(stats, "c3-384x216")


@pytest.mark.parametrize("m,name,W,H,moving", [(6, "c1", 192, 108, False), (30, "c2", 256, 144, True)])
def test_frame_parity_adaptive_ray_count(m, name, W, H, moving):
    """Eq. 4 adaptive mode: Sobel edge measure and the previous frame's variance; a
    static camera and a moving one, small and large ray caps m."""
    w = make_workload(name, W=W, H=H, n_frames=3)
    if not moving or w.n_frames < 3:
        w.poses = [w.poses[0]] * 3
    prm = dict(w.params, ray_mode=1, m=m)
    stats = run_sequence(w, 3, prm)
    _print(stats, f"{name}-adaptive-m{m}")


def test_edge_cases_tiny_empty_single():
    # 2x2 image (one half-resolution pixel), 4x2, an empty scene, a one-triangle scene
    for W, H, scene in [(2, 2, None), (4, 2, None), (64, 36, "empty"), (64, 36, "one")]:
        w = make_workload("c1", W=W, H=H)
        if scene == "empty":
            sc = tiny_scene(1, 0, ties=False)
            w._scene = sc
        elif scene == "one":
            w._scene = plane_scene([(2.0, "right", 0.0, 0)])
        prm = dict(w.params, mask_near_hpx=0.0)
        run_sequence(w, 1, prm)


def test_max_spp_and_history_reset():
    from paper_2210_06158_gb300 import dof
    w = make_workload("c1", W=64, H=36)
    prm = dict(w.params, spp=64, mask_near_hpx=0.0)
    run_sequence(w, 1, prm)
    # reset: the next frame equals a first frame
    osc, cam, gb = oracle_inputs(w, 0)
    g = GpuRunner(w, w.params)
    a = g.frame(cam, gb)["out"]
    g.frame(cam, gb)
    g.hist.reset()
    b = g.frame(cam, gb)["out"]
    assert np.array_equal(a, b)


def test_checkpoint_resume_bit_identical():
    """export after frame 1, import into a fresh history: frame 2 is bit-identical to the
    uninterrupted session (history + counter-based lens samples are the whole state)."""
    from paper_2210_06158_gb300 import dof
    w = make_workload("c2", W=320, H=180, n_frames=3)
    osc = oracle.Scene(w.scene)
    gbs = [oracle.gbuffer_f32(oracle.gbuffer(osc, w.camera(k), w.params, w.W, w.H)) for k in range(3)]
    a = GpuRunner(w, w.params)
    for k in range(2):
        a.frame(w.camera(k), gbs[k], read=False)
    ck = a.hist.export()
    b = GpuRunner(w, w.params, ctx=a.ctx)
    b.hist.load(ck)
    out_a = a.frame(w.camera(2), gbs[2])
    out_b = b.frame(w.camera(2), gbs[2])
    assert np.array_equal(out_a["out"], out_b["out"])
    assert np.array_equal(out_a["hist"], out_b["hist"])
    other = dof.History(a.ctx, 322, 180)
    with pytest.raises(dof.DofError) as e:
        other.load(ck)
    assert e.value.code == -7


@pytest.mark.parametrize("name,W,H", [("c3", 384, 216), ("c2", 322, 182)])
def test_scheduling_knobs_do_not_change_results(name, W, H):
    """The autotuned knobs change only speed: the tracer's work order (lens-cell grid 1
    = pixel order, 2 .. 16), its traversal stack, the tree's width, warp packets
    instead of one ray per lane, the gathers' block shapes and the main filter's form (shared-memory halo tile,
    L1, or columns of four pixels through L1) give bit-identical hit ids, intermediates
    and images over two frames of a moving camera (the c3 crop with its 64 px clamp
    takes the halo tile only in the opt-in form)."""
    from paper_2210_06158_gb300 import dof
    import torch
    dev = torch.device("cuda", 0)
    w = make_workload(name, W=W, H=H, n_frames=2)
    prm = dict(w.params)
    osc = oracle.Scene(w.scene)
    gbs = []
    for f in range(2):
        gb = oracle.gbuffer_f32(oracle.gbuffer(osc, w.camera(f), prm, w.W, w.H))
        gbs.append({k: torch.from_numpy(np.ascontiguousarray(v)).to(dev) for k, v in gb.items()})
    ctx = dof.Context(0)
    sc = dof.Scene(ctx, w.scene)
    variants = [dict(ray_grid=1), dict(ray_grid=2), dict(ray_grid=4), dict(ray_grid=8), dict(ray_grid=12),
                dict(ray_grid=16), dict(ray_grid=8, stack=32), dict(ray_grid=8, stack=64),
                dict(ray_grid=1, packets=1), dict(ray_grid=4, packets=1), dict(ray_grid=8, packets=1, stack=32),
                dict(ray_grid=4, packets=1, stats=0),
                dict(ray_grid=1, width=2), dict(ray_grid=8, width=2, stack=32),
                dict(block=(16, 16), main_form=0, recon=(16, 16)), dict(block=(64, 4), main_form=1, recon=(64, 8)),
                dict(block=(32, 16), main_form=2, recon=(32, 16)), dict(block=(64, 8), main_form=2, recon=(64, 4)),
                dict(block=(32, 8), main_form=1, recon=(8, 32)), dict(block=(32, 8), main_form=3),
                dict(block=(64, 4), main_form=3, recon=(16, 16)), dict(block=(16, 8), main_form=3)]
    results = []
    for v in variants:
        ctx.set_trace(ray_grid=v.get("ray_grid", 4), stack=v.get("stack", 96), packets=v.get("packets", 0),
                      bvh_width=v.get("width", 4), stats=v.get("stats", 1))
        ctx.set_gather(block=v.get("block", (32, 8)), main_form=v.get("main_form", 0),
                       recon_block=v.get("recon", (32, 8)))
        h = dof.History(ctx, w.W, w.H, max_rays=oracle.max_rays(prm), record_rays=True)
        outs = [dof.frame(ctx, sc, gbs[f], w.camera(f), prm, h).cpu().numpy() for f in range(2)]
        torch.cuda.synchronize()
        st = h.stats()
        assert st.device_status == 0
        # the packet tracer's counters only when asked for (the rays are counted either way)
        assert (st.node_visits > 0) == (v.get("stats", 1) == 1) and st.rays > 0
        results.append((v, outs, h.read("RAY_PRIM", np.int32), h.read("MAIN", np.float32),
                        h.read("RECON", np.float32)))
        h.close()
    r0 = results[0]
    for r in results[1:]:
        for f in range(2):
            assert np.array_equal(r0[1][f], r[1][f]), (r[0], f)
        for k in (2, 3, 4):
            assert np.array_equal(r0[k], r[k]), (r[0], k)


def test_tree_shape_does_not_change_hits():
    """The closest hit is a property of the triangles, not of the tree: PLOC or LBVH,
    with or without tree rotations, binary or 4-wide traversal give bit-identical hit
    ids and images."""
    from paper_2210_06158_gb300 import dof
    import torch
    dev = torch.device("cuda", 0)
    w = make_workload("c2", W=322, H=182, n_frames=2, session=3)
    prm = dict(w.params)
    osc = oracle.Scene(w.scene)
    gbs = []
    for f in range(2):
        gb = oracle.gbuffer_f32(oracle.gbuffer(osc, w.camera(f), prm, w.W, w.H))
        gbs.append({k: torch.from_numpy(np.ascontiguousarray(v)).to(dev) for k, v in gb.items()})
    results = []
    for builder, rot in (("ploc", 0), ("lbvh", 0), ("ploc", 4), ("lbvh", 2)):
        ctx = dof.Context(0)
        ctx.set_bvh_builder(builder)
        ctx.set_bvh_rotations(rot)
        sc = dof.Scene(ctx, w.scene)
        info = sc.info()
        assert info.n_nodes4 > 0 and 0 < info.depth4 <= info.depth
        assert info.n_nodes4 <= info.n_nodes
        for width in (2, 4):
            ctx.set_bvh_width(width)
            h = dof.History(ctx, w.W, w.H, max_rays=oracle.max_rays(prm), record_rays=True)
            outs = []
            for f in range(2):
                outs.append(dof.frame(ctx, sc, gbs[f], w.camera(f), prm, h).cpu().numpy())
            torch.cuda.synchronize()
            assert h.stats().device_status == 0
            results.append((f"{builder}/rot{rot}", width, outs, h.read("RAY_PRIM", np.int32), h.stats().node_visits))
            h.close()
        sc.close()
    b0 = results[0]
    for b in results[1:]:
        for f in range(2):
            assert np.array_equal(b0[2][f], b[2][f]), (b[0], b[1], f)
        assert np.array_equal(b0[3], b[3]), (b[0], b[1])
    # the 4-wide tree visits fewer nodes than the binary one
    assert results[0][1] == 2 and results[1][1] == 4
    assert results[1][4] < results[0][4]


@pytest.mark.parametrize("packets", [0, 1])
def test_batch_equals_alone(packets):
    """dof_batch_frame over sessions of different sizes, scenes, lenses, ray modes and
    aperture shapes gives, for every session, exactly what dof_frame gives for it alone
    (alone: one ray per lane; batched: the same, or warp packets, whose warps straddle
    the sessions' ray lists at their boundaries)."""
    from paper_2210_06158_gb300 import dof
    import torch
    dev = torch.device("cuda", 0)
    specs = [("c1", 256, 144, {}), ("c2", 322, 182, dict(aperture_blades=6)), ("c3", 192, 108, {}),
             ("c1", 130, 74, dict(ray_mode=1, m=4, aperture_blades=5))]
    ctx = dof.Context(0)
    sess = []
    for k, (name, W, H, over) in enumerate(specs):
        w = make_workload(name, W=W, H=H, n_frames=2, session=k)
        if w.n_frames < 2:
            w.poses = [w.poses[0]] * 2            # a static camera for the one-pose workload
        prm = dict(w.params, **over)
        osc = oracle.Scene(w.scene)
        gbs = []
        for f in range(2):
            gb = oracle.gbuffer_f32(oracle.gbuffer(osc, w.camera(f), prm, W, H))
            gbs.append({kk: torch.from_numpy(np.ascontiguousarray(v)).to(dev) for kk, v in gb.items()})
        sc = dof.Scene(ctx, w.scene)
        mr = oracle.max_rays(prm)
        sess.append(dict(w=w, prm=prm, gbs=gbs, sc=sc, alone=dof.History(ctx, W, H, mr),
                         mixed=dof.History(ctx, W, H, mr)))
    for f in range(2):
        ctx.set_trace(packets=0)
        alone = [dof.frame(ctx, s["sc"], s["gbs"][f], s["w"].camera(f), s["prm"], s["alone"]).clone() for s in sess]
        ctx.set_trace(packets=packets)
        mixed = dof.batch_frame(ctx, [dict(scene=s["sc"], gbuf=s["gbs"][f], cam=s["w"].camera(f), params=s["prm"],
                                           hist=s["mixed"]) for s in sess])
        torch.cuda.synchronize()
        for k in range(len(sess)):
            assert torch.equal(alone[k], mixed[k]), (f, k)
    with pytest.raises(dof.DofError):
        s = sess[0]
        dof.batch_frame(ctx, [dict(scene=s["sc"], gbuf=s["gbs"][0], cam=s["w"].camera(0), params=s["prm"],
                                   hist=s["mixed"])] * 2)


@pytest.mark.parametrize("packets", [0, 1])
def test_graph_equals_batch(packets):
    """A captured step (CUDA graph) replayed with new cameras and G-buffers gives, frame
    after frame, exactly what dof_batch_frame gives, with either tracer (one ray per lane
    or warp packets); launches that need other histories, launch shapes or the other
    tracer are refused."""
    from paper_2210_06158_gb300 import dof
    import torch
    dev = torch.device("cuda", 0)
    specs = [("c1", 256, 144, {}), ("c2", 322, 182, {}), ("c1", 130, 74, dict(ray_mode=1, m=4))]
    ctx = dof.Context(0)
    ctx.set_trace(packets=packets)
    sess = []
    nf = 3
    for k, (name, W, H, over) in enumerate(specs):
        w = make_workload(name, W=W, H=H, n_frames=nf, session=k)
        if w.n_frames < nf:
            w.poses = [w.poses[0]] * nf
        prm = dict(w.params, **over)
        osc = oracle.Scene(w.scene)
        gbs = []
        for f in range(nf):
            gb = oracle.gbuffer_f32(oracle.gbuffer(osc, w.camera(f), prm, W, H))
            gbs.append({kk: torch.from_numpy(np.ascontiguousarray(v)).to(dev) for kk, v in gb.items()})
        sc = dof.Scene(ctx, w.scene)
        mr = oracle.max_rays(prm)
        sess.append(dict(w=w, prm=prm, gbs=gbs, sc=sc, hb=dof.History(ctx, W, H, mr), hg=dof.History(ctx, W, H, mr)))

    def items(f, key):
        return [dict(scene=s["sc"], gbuf=s["gbs"][f], cam=s["w"].camera(f), params=s["prm"], hist=s[key]) for s in sess]

    graph = dof.Graph(ctx, items(0, "hg"))
    for f in range(nf):
        a = [t.clone() for t in dof.batch_frame(ctx, items(f, "hb"))]
        b = graph.launch(items(f, "hg"))
        torch.cuda.synchronize()
        for k in range(len(sess)):
            assert torch.equal(a[k], b[k]), (f, k)
    assert sess[0]["hg"].stats().device_status == 0
    with pytest.raises(dof.DofError):
        graph.launch(items(0, "hb"))                    # not the captured histories
    with pytest.raises(dof.DofError):
        graph.launch(items(0, "hg")[:2])                # fewer sessions
    wider = items(0, "hg")
    for it in wider:
        it["params"] = dict(it["params"], max_coc_px=2.0 * float(it["params"]["max_coc_px"]))
    with pytest.raises(dof.DofError):
        graph.launch(wider)                             # another main-filter tile (halo follows max_coc_px)
    ctx.set_trace(packets=1 - packets)
    with pytest.raises(dof.DofError):
        graph.launch(items(0, "hg"))                    # captured with the other tracer
    graph.close()


# Bounds of the added error against the FP64 oracle, per output, for the plain FP32
# form and the FP16-storage form (colour image planes stored as half, FP32 arithmetic,
# FP32 depth, CoC, ray sums and history).  Half rounding is 2^-11 relative per stored
# value; the filters' weighted sums keep it there.
OUTPUT_TOL = {"fp32": dict(pp_med=5e-4, crt=5e-4, rt_med=5e-4, recon=1e-3, hist=5e-4, out=2e-3),
              "fp16": dict(pp_med=2e-3, crt=2e-3, rt_med=2e-3, recon=2e-3, hist=5e-4, out=2e-3)}


@pytest.mark.parametrize("name,W,H,nf", [("c3", 384, 216, 2), ("c2", 322, 182, 3)])
def test_fp16_storage_error_vs_oracle(name, W, H, nf):
    """Added error against the FP64 oracle per output -- post-process median (PP), ray
    colour and its median (RT), reconstruction, history, final image -- for the plain
    FP32 form and the FP16-storage form; each within its bound (OUTPUT_TOL), and the
    final image within the FP32 tolerances (max |d| <= 2e-3, PSNR >= 50 dB)."""
    w = make_workload(name, W=W, H=H, n_frames=nf)
    prm32 = dict(w.params)
    prm16 = dict(prm32, image_storage=1)
    osc = oracle.Scene(w.scene)
    runs = {"fp32": GpuRunner(w, prm32), "fp16": GpuRunner(w, prm16)}
    ohist = oracle.History(w.W, w.H)
    taint = np.zeros((H // 2, W // 2), bool)
    for k in range(nf):
        cam = w.camera(k)
        gb = oracle.gbuffer_f32(oracle.gbuffer(osc, cam, prm32, W, H))
        hist0 = ohist.copy()
        ref = oracle.frame(osc, cam, prm32, W, H, gb, ohist)
        got = {form: g.frame(cam, gb) for form, g in runs.items()}
        assert np.array_equal(got["fp16"]["ray_prim"], got["fp32"]["ray_prim"])
        assert np.array_equal(got["fp16"]["nrays"], got["fp32"]["nrays"])
        # counts may differ only on mask ties (fixed mode); the oracle then takes the kernel's
        diff_n = got["fp32"]["nrays"] != ref["nrays"]
        assert not diff_n[~mask_ties(ref, prm32)].any()
        force = np.where(diff_n, got["fp32"]["nrays"], -1).astype(np.int32) if diff_n.any() else None
        if force is not None:
            ohist = hist0.copy()
            ref = oracle.frame(osc, cam, prm32, W, H, gb, ohist, nrays_force=force)
        n_rays, n_mis, n_bad, _ = classify_hits(osc, w, prm32, cam, got["fp32"], ref)
        assert n_bad == 0 and n_mis <= max(2, 1e-4 * n_rays)
        if n_mis:
            # either hit is valid: the oracle takes the kernels' (both forms trace the same rays)
            mr_o = ref["ray_prim"].shape[2]
            valid = np.arange(mr_o)[None, None, :] < ref["nrays"][..., None]
            gp = got["fp32"]["ray_prim"][..., :mr_o]
            hforce = np.where(valid & (gp != ref["ray_prim"]), gp, -2).astype(np.int32)
            ohist = hist0.copy()
            ref = oracle.frame(osc, cam, prm32, W, H, gb, ohist, nrays_force=force, hit_force=hforce)
        taint = dilate(dilate(taint, 2) | weight_ties(ref), taint_radius(prm32))
        tf = full_res(taint, W, H)
        ok = ~taint
        hist_ch = [0, 1, 2, 3, 4, 5, 6, 7, 10, 11]
        for form, g in got.items():
            err = dict(pp_med=max_hdr(g["pp_med"], ref["pp_med"]),
                       crt=max_hdr(g["crt"][ok], ref["crt"][ok]),
                       rt_med=max_hdr(g["rt_med"][ok], ref["rt_med"][ok]),
                       recon=max_hdr(g["recon"][ok], ref["recon"][ok]),
                       hist=max_hdr(g["hist"][..., hist_ch][ok], ref["hist"][..., hist_ch][ok]),
                       out=max_hdr(g["out"][..., :3][~tf], ref["out"][..., :3][~tf]))
            p_out = psnr(g["out"][..., :3], ref["out"][..., :3])
            print(f"[precision {name} {form}] frame={k} " + " ".join(f"{o}={e:.3g}" for o, e in err.items())
                  + f" psnr_out={p_out:.1f} tainted={tf.mean():.3g}")
            for o, e in err.items():
                assert e <= OUTPUT_TOL[form][o], (form, o, e)
            assert p_out >= 50.0, (form, p_out)


def test_determinism_bit_identical():
    w = make_workload("c2", W=320, H=180, n_frames=2)
    osc = oracle.Scene(w.scene)
    outs = []
    for _ in range(2):
        g = GpuRunner(w, w.params)
        seq = []
        for k in range(2):
            cam = w.camera(k)
            gb = oracle.gbuffer_f32(oracle.gbuffer(osc, cam, w.params, w.W, w.H))
            seq.append(g.frame(cam, gb, read=False)["out"])
        outs.append(seq)
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_host_validation_errors():
    from paper_2210_06158_gb300 import dof
    import torch
    ctx = dof.Context(0)
    w = make_workload("c1", W=64, H=36)
    sc = dof.Scene(ctx, w.scene)
    h = dof.History(ctx, 64, 36, max_rays=1)
    dev = torch.device("cuda", 0)
    gb = dict(color=torch.zeros((36, 64, 4), device=dev), depth=torch.ones((36, 64), device=dev))
    cam = w.camera(0)
    with pytest.raises(dof.DofError) as e:
        dof.frame(ctx, sc, gb, cam, dict(w.params, spp=2), h)
    assert e.value.code == -1
    bad = w.camera(0)
    bad.focus_m = 0.01
    with pytest.raises(dof.DofError) as e:
        dof.frame(ctx, sc, gb, bad, w.params, h)
    assert e.value.code == -1
    for blades in (1, 2, 9):                         # aperture: 0 (circle) or 3..8 blades
        with pytest.raises(dof.DofError) as e:
            dof.frame(ctx, sc, gb, cam, dict(w.params, aperture_blades=blades), h)
        assert e.value.code == -1
    gb2 = dict(color=torch.zeros((38, 64, 4), device=dev), depth=torch.ones((38, 64), device=dev))
    with pytest.raises(dof.DofError) as e:
        dof.frame(ctx, sc, gb2, cam, w.params, h)
    assert e.value.code == -7
    with pytest.raises(dof.DofError) as e:
        dof.History(ctx, 63, 36)
    assert e.value.code == -1
    # handles may be released in any order (the context outlives its scene and history)
    c2 = dof.Context(0)
    sc2 = dof.Scene(c2, w.scene)
    h2 = dof.History(c2, 64, 36)
    used = c2.bytes_in_use
    assert used > 0
    c2.close()
    h2.close()
    sc2.close()
    small = dof.Context(0, mem_budget_bytes=1 << 16)
    with pytest.raises(dof.DofError) as e:
        dof.History(small, 640, 360)
    assert e.value.code == -3
    assert small.bytes_in_use == 0


def _bench_context(ploc_radius, **trace):
    """A context with the tracer settings the benchmark's autotuner picks for a workload
    on GB300 (the results do not depend on them; the launches do)."""
    from paper_2210_06158_gb300 import dof
    ctx = dof.Context(0)
    ctx.set_ploc_radius(ploc_radius)
    ctx.set_trace(**trace)
    return ctx


@pytest.mark.slow
def test_full_size_c2_two_frames():
    """1920x1080, 495,802 triangles, 1 spp, frames 0 and 1 of the dolly, in the launch
    configuration the benchmark times (binary tree from PLOC radius 16, pixel order,
    warp packets)."""
    w = make_workload("c2", n_frames=2)
    stats = run_sequence(w, 2, ctx=_bench_context(16, bvh_width=2, ray_grid=1, packets=1))
    _print(stats, "c2-full")
    tot = sum(s["rays"] for s in stats)
    mis = sum(s["mismatches"] for s in stats)
    assert mis <= max(2, 1e-4 * tot), (mis, tot)


def test_full_size_c3_two_frames():
    """3840x2160, 1,980,930 triangles, 85 mm f/1.2, CoC radius clamp 64 px, 4 spp, frames
    0 and 1 of the dolly at full size, in the launch configuration the benchmark times
    (the main filter's halo and the tracer's batch as at 4K; binary tree from PLOC radius
    48, rays grouped on an 8 x 8 lens grid, one ray per lane)."""
    w = make_workload("c3", n_frames=2)
    stats = run_sequence(w, 2, ctx=_bench_context(48, bvh_width=2, ray_grid=8, packets=0))
    _print(stats, "c3-full")
    tot = sum(s["rays"] for s in stats)
    mis = sum(s["mismatches"] for s in stats)
    assert mis <= max(2, 1e-4 * tot), (mis, tot)


def test_host_frames_equal_device_frames():
    """dof_frame_host (G-buffer in and image out through host memory, two device slots,
    copies on the library's own streams, three frames in flight before the join) gives
    the images dof_frame gives from device buffers, bit for bit; in the adaptive mode the
    normal plane travels too."""
    from paper_2210_06158_gb300 import dof
    import torch
    for mode in (0, 1):
        w = make_workload("c1", n_frames=5)
        prm = dict(w.params, ray_mode=mode, m=6)
        ctx = dof.Context(0)
        sc = dof.Scene(ctx, w.scene)
        gbs = [dof.gbuffer(ctx, sc, w.camera(k), prm, w.W, w.H) for k in range(w.n_frames)]
        mr = oracle.max_rays(prm)
        ha = dof.History(ctx, w.W, w.H, max_rays=mr)
        hb = dof.History(ctx, w.W, w.H, max_rays=mr)
        want = []
        for k in range(w.n_frames):
            want.append(dof.frame(ctx, sc, gbs[k], w.camera(k), prm, ha).cpu())
        keys = ("color", "depth", "normal") if mode == 1 else ("color", "depth")
        hosts = [{key: gbs[k][key].cpu().pin_memory() for key in keys} for k in range(w.n_frames)]
        outs = [torch.empty((w.H, w.W, 4), dtype=torch.float32).pin_memory() for _ in range(w.n_frames)]
        for k in range(w.n_frames):
            dof.frame_host(ctx, sc, hosts[k], w.camera(k), prm, hb, outs[k])
        dof.frame_host_join(hb)
        torch.cuda.synchronize()
        for k in range(w.n_frames):
            assert torch.equal(outs[k].view(torch.int32), want[k].view(torch.int32)), (mode, k)


def test_launch_count_per_frame():
    """The library's own launch tally (dof_launch_count): 11 kernels per frame, +2 for the
    edge measure in the adaptive mode, +1 for the final TAA; a replayed graph counts the
    kernels it holds."""
    from paper_2210_06158_gb300 import dof
    import torch
    w = make_workload("c1", W=128, H=72)
    ctx = dof.Context(0)
    sc = dof.Scene(ctx, w.scene)
    g = dof.gbuffer(ctx, sc, w.camera(0), w.params, w.W, w.H)
    for over, taa, want in ((dict(ray_mode=0), False, 11), (dict(ray_mode=1, m=4), False, 13),
                            (dict(ray_mode=0, taa_alpha=0.1), True, 12)):
        prm = dict(w.params, **over)
        h = dof.History(ctx, w.W, w.H, max_rays=oracle.max_rays(prm), taa=taa)
        dof.frame(ctx, sc, g, w.camera(0), prm, h)
        n0 = dof.launch_count()
        for _ in range(3):
            dof.frame(ctx, sc, g, w.camera(0), prm, h)
        assert dof.launch_count() - n0 == 3 * want, (over, dof.launch_count() - n0)
    h = dof.History(ctx, w.W, w.H, max_rays=1)
    items = [dict(scene=sc, gbuf=g, cam=w.camera(0), params=w.params, hist=h)]
    n0 = dof.launch_count()
    graph = dof.Graph(ctx, items)
    assert dof.launch_count() == n0                 # capturing runs nothing
    graph.launch(items)
    graph.launch(items)
    torch.cuda.synchronize()
    assert dof.launch_count() - n0 == 2 * 11
    graph.close()


@pytest.mark.parametrize("grid", [1, 8])
def test_packets_in_adaptive_mode_equal_one_ray_per_lane(grid):
    """In the adaptive mode of Eq. 4 (up to m rays per pixel, as many as the edge measure
    and the history's variance ask for) warp packets give, over three frames of a moving
    camera, the hit ids, ray counts and images of the per-ray tracer bit for bit."""
    from paper_2210_06158_gb300 import dof
    import torch
    dev = torch.device("cuda", 0)
    w = make_workload("c2", W=322, H=182, n_frames=3)
    prm = dict(w.params, ray_mode=1, m=12)
    osc = oracle.Scene(w.scene)
    gbs = []
    for f in range(3):
        gb = oracle.gbuffer_f32(oracle.gbuffer(osc, w.camera(f), prm, w.W, w.H))
        gbs.append({k: torch.from_numpy(np.ascontiguousarray(v)).to(dev) for k, v in gb.items()})
    ctx = dof.Context(0)
    sc = dof.Scene(ctx, w.scene)
    results = []
    for packets in (0, 1):
        ctx.set_trace(bvh_width=2, ray_grid=grid, packets=packets)
        h = dof.History(ctx, w.W, w.H, max_rays=12, record_rays=True)
        outs = [dof.frame(ctx, sc, gbs[f], w.camera(f), prm, h).cpu().numpy() for f in range(3)]
        torch.cuda.synchronize()
        st = h.stats()
        assert st.device_status == 0 and st.rays > st.masked_pixels     # several rays per pixel
        results.append((outs, h.read("RAY_PRIM", np.int32), h.read("NRAYS", np.int32)))
        h.close()
    for f in range(3):
        assert np.array_equal(results[0][0][f], results[1][0][f]), f
    assert np.array_equal(results[0][1], results[1][1])
    assert np.array_equal(results[0][2], results[1][2])


def test_packets_on_tiny_trees_equal_one_ray_per_lane():
    """Warp packets on the smallest trees -- no triangle, one (the root is a leaf), two,
    seven, and 64 and 200 with shared-edge and coplanar ties -- give the per-ray tracer's
    hit ids and images bit for bit with the device status clear.  The packet loop has no
    per-step guard: it relies on the structure check each tree passes at upload."""
    from paper_2210_06158_gb300 import dof
    import torch
    ctx = dof.Context(0)
    pose = camera_pose((0.0, 0.0, 0.0), pitch_deg=0.0)
    cam = Camera.from_poses(dict(f_m=0.085, f_number=1.2, focus_m=30.0, sensor_w_m=0.036), pose)
    W, H = 128, 72
    prm = default_params(spp=4, mask_near_hpx=0.0, max_coc_px=16.0)
    for n in [0, 1, 2, 7, 64, 200]:
        sc = dof.Scene(ctx, tiny_scene(700 + n, n, ties=n >= 8))
        gb = dof.gbuffer(ctx, sc, cam, prm, W, H)
        del gb["prim"]
        results = []
        for packets in (0, 1):
            ctx.set_trace(bvh_width=2, ray_grid=4, packets=packets)
            h = dof.History(ctx, W, H, max_rays=4, record_rays=True)
            out = dof.frame(ctx, sc, gb, cam, prm, h).cpu().numpy()
            torch.cuda.synchronize()
            st = h.stats()
            assert st.device_status == 0, (n, packets)
            assert n == 0 or st.rays > 0, n
            results.append((out, h.read("RAY_PRIM", np.int32)))
            h.close()
        assert np.array_equal(results[0][0], results[1][0]), n
        assert np.array_equal(results[0][1], results[1][1]), n
        sc.close()
