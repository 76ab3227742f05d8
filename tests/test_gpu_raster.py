"""The object-order G-buffer producer (dof_gbuffer_raster) against the ray-cast one
(dof_gbuffer): both run the same watertight ray/triangle test on the same primary
ray per pixel and keep the closest hit by (distance, triangle id), so every output
must agree bit for bit.  The ray-cast producer is itself checked against the
oracle (test_gpu_parity.py); here the cases are the ones a rasteriser's setup can
get wrong: triangles across the camera plane or behind it, seen edge-on, through
the lens centre, degenerate, larger than the image, far and tiny, shared edges and
exact depth ties, jittered and rotated cameras, and the workload scenes."""
import math

import numpy as np
import pytest

from synth.scenes import (Camera, _Builder, camera_pose, default_params, make_workload, plane_scene,
                          tiny_scene, SplitMix64)

pytestmark = pytest.mark.gpu


def _run(ctx, sc, cam, prm, W, H):
    from paper_2210_06158_gb300 import dof
    import torch
    a = dof.gbuffer(ctx, sc, cam, prm, W, H)
    b = dof.gbuffer(ctx, sc, cam, prm, W, H, raster=True)
    torch.cuda.synchronize()
    return ({k: v.cpu().numpy() for k, v in a.items()}, {k: v.cpu().numpy() for k, v in b.items()})


def _assert_same(a, b, tag):
    bad = np.argwhere(a["prim"] != b["prim"])
    assert len(bad) == 0, (tag, len(bad), bad[:5].tolist(),
                           [(int(a["prim"][j, i]), int(b["prim"][j, i])) for j, i in bad[:5]])
    for k in ("color", "depth", "normal"):
        x, y = a[k].view(np.uint32), b[k].view(np.uint32)
        nd = int(np.count_nonzero(x != y))
        assert nd == 0, (tag, k, nd)


def edge_case_scene(seed=11) -> "Scene":
    """Triangles that stress a rasteriser's setup, around a camera at the origin looking
    along +z."""
    b = _Builder(seed)
    # ground plane reaching behind the camera (crosses the camera plane)
    b.add("ground", [[-500.0, -1.0, -500.0], [500.0, -1.0, -500.0], [0.0, -1.0, 800.0]], [(0, 1, 2)])
    # one vertex behind the camera, two in front
    b.add("straddle", [[-1.2, 0.0, -1.0], [-0.5, 0.1, 2.0], [-0.6, -0.3, 1.5]], [(0, 1, 2)])
    b.add("straddle2", [[0.8, 0.3, -0.5], [0.3, 0.35, 3.0], [0.5, 0.15, 2.5]], [(0, 1, 2)])
    # wholly behind the camera
    b.add("behind", [[-1.0, -1.0, -2.0], [1.0, -1.0, -2.0], [0.0, 1.0, -2.0]], [(0, 1, 2)])
    # in a plane through the lens centre (seen edge-on)
    b.add("edge_on", [[0.0, 0.1, 2.0], [0.0, 0.5, 3.0], [0.0, -0.3, 4.0]], [(0, 1, 2)])
    # collinear vertices, a single point, a vertex at the lens centre
    b.add("collinear", [[0.2, 0.2, 2.0], [0.4, 0.4, 2.0], [0.6, 0.6, 2.0]], [(0, 1, 2)])
    b.add("point", [[-0.2, 0.1, 2.0], [-0.2, 0.1, 2.0], [-0.2, 0.1, 2.0]], [(0, 1, 2)])
    b.add("at_lens", [[0.0, 0.0, 0.0], [0.4, 0.1, 3.0], [0.1, 0.5, 3.0]], [(0, 1, 2)])
    # thin slivers, far tiny triangles, near large ones
    b.add("sliver", [[-0.8, -0.6, 3.0], [0.8, 0.61, 3.0], [0.8, 0.6, 3.0001]], [(0, 1, 2)])
    rng = SplitMix64(seed)
    n = 300
    c = np.stack([rng.uniform(n, -250, 250), rng.uniform(n, -60, 120), rng.uniform(n, 500, 900)], -1)
    v = c[:, None, :] + rng.uniform(9 * n, -3.0, 3.0).reshape(n, 3, 3)
    b.add("far_tiny", v.reshape(-1, 3), np.arange(3 * n).reshape(n, 3))
    m = 12
    c = np.stack([rng.uniform(m, -0.5, 0.5), rng.uniform(m, -0.3, 0.3), rng.uniform(m, 0.3, 0.8)], -1)
    v = c[:, None, :] + rng.uniform(9 * m, -0.04, 0.04).reshape(m, 3, 3)
    b.add("near_large", v.reshape(-1, 3), np.arange(3 * m).reshape(m, 3))
    # a fan of triangles sharing one vertex, and a quad split along its diagonal
    k = 24
    ang = np.linspace(0.0, 2 * math.pi, k + 1)
    fan = np.concatenate([[[0.6, -0.2, 2.5]], np.stack([0.6 + 0.3 * np.cos(ang), -0.2 + 0.3 * np.sin(ang),
                                                          np.full(k + 1, 2.5)], -1)])
    b.add("fan", fan, [(0, 1 + i, 2 + i) for i in range(k)])
    return b.build()


def _cam(pos=(0.0, 0.0, 0.0), pitch=0.0, yaw=0.0, jitter=(0.0, 0.0), f_m=0.05):
    pose = camera_pose(pos, pitch_deg=pitch, yaw_deg=yaw)
    cam = Camera.from_poses(dict(f_m=f_m, f_number=2.0, focus_m=3.0, sensor_w_m=0.036), pose)
    cam.jitter = jitter
    return cam


def test_raster_equals_ray_cast_on_edge_cases():
    from paper_2210_06158_gb300 import dof
    ctx = dof.Context(0)
    prm = default_params()
    sc = dof.Scene(ctx, edge_case_scene())
    for W, H in [(96, 64), (320, 180), (2, 2)]:
        for pos, pitch, yaw, jit in [((0, 0, 0), 0.0, 0.0, (0.0, 0.0)), ((0, 0, 0), 7.0, 13.0, (0.31, -0.27)),
                                     ((0.05, 0.02, 0.01), -4.0, -25.0, (-0.5, 0.5)),
                                     ((0, 0, 0), 0.0, 180.0, (0.0, 0.0))]:
            cam = _cam(pos, pitch, yaw, jit)
            a, b = _run(ctx, sc, cam, prm, W, H)
            _assert_same(a, b, (W, H, pos, pitch, yaw))
    # the straddling and edge-on triangles really are in view (the case is not vacuous)
    a, _ = _run(ctx, sc, _cam(), prm, 320, 180)
    assert len(np.unique(a["prim"])) > 20


def test_raster_equals_ray_cast_on_tiny_and_plane_scenes():
    from paper_2210_06158_gb300 import dof
    ctx = dof.Context(0)
    prm = default_params()
    cam = _cam()
    for n in [0, 1, 2, 7, 64, 200, 2000]:
        sc = dof.Scene(ctx, tiny_scene(900 + n, n, ties=n >= 8))
        a, b = _run(ctx, sc, cam, prm, 96, 64)
        _assert_same(a, b, ("tiny", n))
    # fronto-parallel planes with half-plane edges exactly on pixel-centre columns
    W, H = 64, 32
    f_px = 0.05 / 0.036 * W
    xe = 3.0 * (W / 2 - 20.5) / f_px
    sc = dof.Scene(ctx, plane_scene([(5.0, "full", 0.0, 0), (3.0, "right", xe, 0), (3.0, "left", xe, 1)]))
    a, b = _run(ctx, sc, cam, prm, W, H)
    _assert_same(a, b, "planes")


@pytest.mark.parametrize("name,W,H", [("c1", 256, 144), ("c2", 640, 360), ("c3", 960, 540)])
def test_raster_equals_ray_cast_on_workload_scenes(name, W, H):
    from paper_2210_06158_gb300 import dof
    w = make_workload(name, W=W, H=H)
    ctx = dof.Context(0)
    sc = dof.Scene(ctx, w.scene)
    for f in (0, w.n_frames - 1):
        cam = w.camera(f)
        cam.jitter = (0.375, -0.2) if f else (0.0, 0.0)
        a, b = _run(ctx, sc, cam, w.params, W, H)
        _assert_same(a, b, (name, f))


def test_raster_equals_ray_cast_at_full_size():
    """The 1920x1080 frame of the 0.5 M-triangle scene (every output pixel)."""
    from paper_2210_06158_gb300 import dof
    w = make_workload("c2")
    ctx = dof.Context(0)
    sc = dof.Scene(ctx, w.scene)
    a, b = _run(ctx, sc, w.camera(0), w.params, w.W, w.H)
    _assert_same(a, b, "c2 full")


@pytest.mark.parametrize("name,W,H", [("c1", 256, 144), ("c2", 322, 182), ("edge", 96, 64)])
def test_raster_matches_oracle_gbuffer(name, W, H):
    """The object-order producer against the FP64 oracle's G-buffer directly (not only
    against the ray-cast producer): ids equal except where the oracle's hit_check accepts
    the kernel's triangle as a rounding tie (on the workload scenes at most 1e-4 of the
    pixels, a floor of 2), colour and normal within 1e-5, depth within 2e-5 relative,
    misses at +inf."""
    import oracle
    from paper_2210_06158_gb300 import dof
    import torch
    if name == "edge":
        scene = edge_case_scene()
        cam = Camera.from_poses(dict(f_m=0.05, f_number=2.0, focus_m=3.0, sensor_w_m=0.036),
                                camera_pose((0.0, 0.0, 0.0), pitch_deg=0.0))
        prm = default_params()
    else:
        w = make_workload(name, W=W, H=H)
        scene, cam, prm = w.scene, w.camera(0), w.params
    osc = oracle.Scene(scene)
    ref = oracle.gbuffer(osc, cam, prm, W, H)
    ctx = dof.Context(0)
    sc = dof.Scene(ctx, scene)
    got = dof.gbuffer(ctx, sc, cam, prm, W, H, raster=True)
    torch.cuda.synchronize()
    prim = got["prim"].cpu().numpy()
    bad = np.argwhere(prim != ref["prim"])
    for (j, i) in bad:
        d = oracle.pixel_dir(cam, W, H, i + 0.5, j + 0.5)
        code = osc.hit_check(np.asarray(cam.pos, np.float64), d, int(prim[j, i]), int(ref["prim"][j, i]))
        assert code >= 0, (name, i, j, int(prim[j, i]), int(ref["prim"][j, i]), code)
    if name != "edge":          # the stress scene's edge-on triangles tie along whole lines
        assert len(bad) <= max(2, 1e-4 * W * H), (name, len(bad))
    ok = prim == ref["prim"]
    hit = ok & (prim >= 0)
    col = got["color"].cpu().numpy()[..., :3]
    assert np.abs(col[ok].astype(np.float64) - ref["color"][ok]).max() < 1e-5
    dep = got["depth"].cpu().numpy()
    assert (np.abs(dep[hit] - ref["depth"][hit]) / ref["depth"][hit]).max() < 2e-5
    assert np.all(np.isinf(dep[ok & (prim < 0)]))
    nrm = got["normal"].cpu().numpy()[..., :3]
    assert np.abs(nrm[ok].astype(np.float64) - ref["normal"][ok]).max() < 1e-5
