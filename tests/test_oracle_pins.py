"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here calls the CUDA library: each test checks the oracle against a closed
form, an independent library routine (numpy's Philox, scipy's filters, numpy's
median), brute force, or an invariant that the paper's method must satisfy.
"""

import ctypes as C
import json
import math
import os

import numpy as np
import pytest
import scipy.ndimage as ndi

import oracle
from synth import make_workload, plane_scene, tiny_scene, Camera, camera_pose
from synth.scenes import default_params

SQRT2 = math.sqrt(2.0)
HERE = os.path.dirname(os.path.abspath(__file__))


def axis_camera(f=0.05, N=1.4, d=10.0, ws=0.036, pos=(0.0, 0.0, 0.0), prev_pos=None, frame=0):
    pose = camera_pose(pos, pitch_deg=0.0)
    prev = camera_pose(prev_pos, pitch_deg=0.0) if prev_pos is not None else None
    return Camera.from_poses(dict(f_m=f, f_number=N, focus_m=d, sensor_w_m=ws), pose, prev, frame)


def f32(x):
    return float(np.float32(x))


def seg_fraction(tau):
    """Share of a unit disk on the far side of the chord at signed offset tau."""
    if tau >= 1.0:
        return 0.0
    if tau <= -1.0:
        return 1.0
    return (math.acos(tau) - tau * math.sqrt(1.0 - tau * tau)) / math.pi


# ---------------------------------------------------------------------------
# Section 3.3, Eq. 6 and the thin-lens CoC
# ---------------------------------------------------------------------------

LENSES = [(0.05, 1.4, 15.0, 256), (0.035, 2.0, 20.0, 1920), (0.085, 1.2, 20.0, 3840)]


@pytest.mark.parametrize("f,N,d,W", LENSES)
def test_coc_zero_at_focus_and_eq6_bounds(f, N, d, W):
    cam = axis_camera(f, N, d)
    assert oracle.coc(cam, W, f32(d)) == 0.0
    zn, zf = oracle.zof_bounds(cam, W)
    assert zn < f32(d)
    assert abs(abs(oracle.coc(cam, W, zn)) - SQRT2) <= 1e-12 * SQRT2
    assert oracle.coc(cam, W, zn) < 0.0
    if math.isfinite(zf):
        assert abs(oracle.coc(cam, W, zf) - SQRT2) <= 1e-12 * SQRT2
    else:
        assert oracle.coc(cam, W, 1e300) <= SQRT2
    # inside the zone |c| < sqrt2, outside larger
    assert abs(oracle.coc(cam, W, 0.5 * (zn + f32(d)))) < SQRT2
    assert abs(oracle.coc(cam, W, 0.9 * zn)) > SQRT2


@pytest.mark.parametrize("f,N,d,W", LENSES)
def test_coc_matches_lens_equation(f, N, d, W):
    """Independent derivation: the image of depth z focuses at v_z = f z / (z - f);
    the sensor sits at v = f d / (d - f); the blur spot on the sensor has diameter
    a (v - v_z) / v_z by similar triangles (negative when v_z > v, i.e. near)."""
    cam = axis_camera(f, N, d)
    f, N, d, ws = f32(f), f32(N), f32(d), 0.036
    ws = f32(ws)
    a = f / N
    v = f * d / (d - f)
    for z in [0.3, 0.5, 1.0, 2.7, 9.9, d, 33.0, 1e3, 1e5]:
        vz = f * z / (z - f)
        ref = a * (v - vz) / vz * W / ws
        got = oracle.coc(cam, W, z)
        assert abs(got - ref) <= 1e-10 * max(1.0, abs(ref)), (z, got, ref)
    # limit at infinity: a f / (d - f) in sensor units
    cinf = a * f / (d - f) * W / ws
    assert abs(oracle.coc(cam, W, 1e14) - cinf) <= 1e-9 * cinf


# ---------------------------------------------------------------------------
# Philox4x64-10 against numpy's independent implementation
# ---------------------------------------------------------------------------

def test_philox_matches_numpy():
    rng = np.random.default_rng(5)
    for _ in range(200):
        ctr = [int(x) for x in rng.integers(1, 2 ** 63, size=4, dtype=np.int64)]
        key = [int(x) for x in rng.integers(0, 2 ** 63, size=2, dtype=np.int64)]
        mine = oracle.philox4x64(ctr, key)
        # numpy's Philox increments its counter before each block
        c = list(ctr)
        c[0] -= 1
        ref = np.random.Philox(counter=c, key=key).random_raw(4)
        assert list(mine) == list(ref)


def test_philox_lens_uniforms_chi2():
    n = 40000
    u = np.empty(n)
    for i in range(n):
        x = oracle.philox4x64([i, 3, 7, 0], [1001, 0])
        u[i] = (int(x[0]) >> 40) * 2.0 ** -24
    hist, _ = np.histogram(u, bins=64, range=(0, 1))
    e = n / 64
    chi2 = ((hist - e) ** 2 / e).sum()
    assert chi2 < 120.0          # 63 dof: p ~ 1e-5 at 120


# ---------------------------------------------------------------------------
# closest hit: BVH vs all triangles
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 5, 17, 64, 200])
def test_bvh_equals_brute_force(n):
    sc = tiny_scene(100 + n, n)
    os_ = oracle.Scene(sc)
    rng = np.random.default_rng(n)
    tv = sc.tri_vertices().astype(np.float64)
    targets = list(rng.uniform([-1.5, -1.5, 1.5], [1.5, 1.5, 4.5], size=(400, 3)))
    # aim exactly at vertices and edge midpoints (shared-edge and coplanar ties)
    for t in tv[-4:]:
        targets += [t[0], t[1], t[2], 0.5 * (t[0] + t[1]), 0.5 * (t[0] + t[2]), t.mean(0)]
    for T in targets:
        o = rng.uniform(-0.3, 0.3, 3)
        o[2] = 0.0
        d = np.asarray(T) - o
        d /= np.linalg.norm(d)
        assert os_.closest(o, d) == os_.closest(o, d, brute=True)


def test_bvh_equals_brute_force_c1_scene():
    w = make_workload("c1")
    os_ = oracle.Scene(w.scene)
    cam = w.camera(0)
    rng = np.random.default_rng(1)
    hits = 0
    for _ in range(1500):
        x, y = rng.uniform(0, w.W), rng.uniform(0, w.H)
        d = oracle.pixel_dir(cam, w.W, w.H, x, y)
        o = np.asarray(cam.pos, dtype=np.float64) + rng.uniform(-0.02, 0.02, 3)
        a = os_.closest(o, d)
        assert a == os_.closest(o, d, brute=True)
        hits += a[0] >= 0
    assert hits > 1000


def _tri_scene(tris):
    """A scene of the given triangles (each 3 corners), float32 corners."""
    from synth.scenes import Scene
    v = np.asarray(tris, dtype=np.float64).reshape(-1, 3)
    return Scene(verts=v.astype(np.float32), tris=np.arange(len(v), dtype=np.uint32).reshape(-1, 3),
                 mat=np.zeros(len(tris), np.uint32), seed=1)


def test_hit_check_classifier_tiny_ties():
    sc = tiny_scene(3, 4, ties=True)          # exactly the shared-edge quad and the coplanar pair
    os_ = oracle.Scene(sc)
    o = np.zeros(3)
    # the quad (z = 3) is split along its diagonal (-0.5,-0.5)-(0.5,0.5): aim at the diagonal
    # beside the coplanar pair (z = 2.5, which covers the diagonal's middle)
    d = np.array([0.4, 0.4, 3.0]); d /= np.linalg.norm(d)
    assert os_.closest(o, d)[0] in (0, 1)
    assert os_.hit_check(o, d, 0, 1) >= 1 and os_.hit_check(o, d, 1, 0) >= 1
    # nearer the quad's centre the coplanar pair lies in front: the quad is no valid answer
    d = np.array([0.1, 0.1, 3.0]); d /= np.linalg.norm(d)
    assert os_.closest(o, d)[0] in (2, 3)
    assert os_.hit_check(o, d, 0, 2) == -2
    # well inside triangle 0 (below the diagonal): triangle 1 is missed, a miss is wrong
    d = np.array([0.4, -0.45, 3.0]); d /= np.linalg.norm(d)
    prim, _ = os_.closest(o, d)
    assert prim == 0
    assert os_.hit_check(o, d, 1, 0) == -1
    assert os_.hit_check(o, d, -1, 0) == -2
    # the FP64 answer is itself a miss while the kernel reports a clean hit: inconsistent
    assert os_.hit_check(o, d, 0, -1) == -3
    # on the quad's outer edge (x = 0.5), the only hit is grazed: a miss is valid
    d = np.array([0.5, 0.0, 3.0]); d /= np.linalg.norm(d)
    assert os_.hit_check(o, d, -1, 0) == 4
    assert os_.hit_check(o, d, 0, -1) == 3
    # coplanar overlapping triangles at equal distance: a depth tie
    d = np.array([0.0, 0.0, 2.5]); d /= np.linalg.norm(d)
    assert os_.hit_check(o, d, 2, 3) == 1 and os_.hit_check(o, d, 3, 2) == 1


def test_hit_check_rejects_what_rounding_cannot_explain():
    """Each case is a plausible tracer bug that an edge-line or either-side graze test
    would let through."""
    z = np.array([0.0, 0.0, 1.0])
    o = np.zeros(3)
    near = [(-1, -1, 1), (1, -1, 1), (0, 1, 1)]                 # 0: clean near hit at t = 1
    line_only = [(0.5, 0, 3), (1.5, 0, 3), (1, 1, 3)]           # 1: its edge's LINE meets the ray at (0,0,3)
    grazed_far = [(0, -1, 3), (1, -1, 3), (0, 1, 3)]            # 2: an edge segment through (0,0,3)
    behind = [(-1, -1, -2), (1, -1, -2), (0, 1, -2)]            # 3: on the ray's line, behind the origin
    os_ = oracle.Scene(_tri_scene([near, line_only, grazed_far, behind]))
    assert os_.closest(o, z)[0] == 0
    # a far triangle whose extended edge line passes the ray, against a clean nearer hit
    assert os_.hit_check(o, z, 1, 0) == -1
    # a grazed far triangle hiding a clean near one
    assert os_.hit_check(o, z, 2, 0) == -2
    # a triangle behind the origin
    assert os_.hit_check(o, z, 3, 0) == -1
    # an id out of range
    assert os_.hit_check(o, z, 4, 0) == -1


def test_hit_check_grazed_near_and_depth_ties():
    o = np.zeros(3)
    z = np.array([0.0, 0.0, 1.0])
    dlt = float(np.float32(5e-7))     # inside the 1e-6 (|o| + s) band at s = 1
    far = float(np.float32(5e-6))     # outside it
    T = [[(0, -1, 1), (1, -1, 1), (0, 1, 1)],                   # 0: near, edge through the ray (grazed hit)
         [(-2, -2, 2), (2, -2, 2), (0, 2, 2)],                  # 1: clean at t = 2
         [(dlt, -1, 1), (1, 0, 1), (dlt, 1, 1)],                # 2: near, the ray passes 5e-7 outside its edge
         [(far, -1, 1), (1, 0, 1), (far, 1, 1)],                # 3: near, 5e-6 outside its edge
         [(-2, -2, 1.5), (2, -2, 1.5), (0, 2, 1.5)],            # 4: clean at t = 1.5
         [(-2, -2, 2.0000005), (2, -2, 2.0000005), (0, 2, 2.0000005)],   # 5: clean, 2.4e-7 behind 1
         [(-2, -2, 2.001), (2, -2, 2.001), (0, 2, 2.001)]]      # 6: clean, 5e-4 behind 1
    os_ = oracle.Scene(_tri_scene(T))
    # the FP64 hit is grazed: the kernel may miss it and see the clean hit behind
    sub = oracle.Scene(_tri_scene([T[0], T[1]]))
    assert sub.closest(o, z)[0] == 0
    assert sub.hit_check(o, z, 1, 0) == 2
    # ... but not past a clean hit in between
    sub = oracle.Scene(_tri_scene([T[0], T[1], T[4]]))
    assert sub.hit_check(o, z, 1, 0) == -2 and sub.hit_check(o, z, 2, 0) == 2
    # a near triangle missed by 5e-7 may be hit in lower precision; by 5e-6 it may not
    sub = oracle.Scene(_tri_scene([T[1], T[2], T[3]]))
    assert sub.closest(o, z)[0] == 0
    assert sub.hit_check(o, z, 1, 0) == 3
    assert sub.hit_check(o, z, 2, 0) == -1
    # depth ties: 2.4e-7 relative is within rounding, 5e-4 is not
    sub = oracle.Scene(_tri_scene([T[1], T[5], T[6]]))
    assert sub.closest(o, z)[0] == 0
    assert sub.hit_check(o, z, 1, 0) == 1
    assert sub.hit_check(o, z, 2, 0) == -2
    assert os_.hit_check(o, z, 0, 0) == 0


def test_hit_check_accepts_rounding_and_rejects_wrong_ids():
    """Completeness and soundness on random scenes: the FP64 closest hit of the same ray
    perturbed at rounding scale (1e-9, far below the 1e-6 band) is always accepted; an
    id the ray does not meet at all is always rejected."""
    rng = np.random.default_rng(5)
    n_alt = n_rej = 0
    for seed in range(4):
        sc = tiny_scene(40 + seed, 200, ties=True)
        os_ = oracle.Scene(sc)
        V = sc.tri_vertices().astype(np.float64)
        for _ in range(600):
            o = rng.uniform(-0.05, 0.05, 3)
            # aim at a random triangle's edge or vertex half the time, else anywhere
            k = rng.integers(sc.n_tris)
            if rng.uniform() < 0.5:
                a, b = rng.choice(3, 2, replace=False)
                tgt = V[k, a] + rng.uniform() * (V[k, b] - V[k, a])
            else:
                tgt = np.array([rng.uniform(-1.5, 1.5), rng.uniform(-1.5, 1.5), 3.0])
            d = tgt - o
            d /= np.linalg.norm(d)
            want, _ = os_.closest(o, d, brute=True)
            d2 = d * (1.0 + 1e-9 * rng.standard_normal(3))
            o2 = o + 1e-9 * rng.standard_normal(3)
            alt, _ = os_.closest(o2, d2, brute=True)
            if alt != want:
                n_alt += 1
            assert os_.hit_check(o, d, alt, want) >= 0, (seed, want, alt)
            # a triangle whose corners all lie more than 1e-3 from the ray's line: missed
            other = int(rng.integers(sc.n_tris))
            P = V[other] - o
            dist = np.linalg.norm(P - (P @ d)[:, None] * d[None, :], axis=1)
            cen = V[other].mean(0) - o
            ray_dist_c = np.linalg.norm(cen - (cen @ d) * d)
            if other != want and dist.min() > 1e-3 and ray_dist_c > 1.0 and os_.closest(o, d)[0] != other:
                assert os_.hit_check(o, d, other, want) < 0
                n_rej += 1
    assert n_alt >= 5 and n_rej >= 100, (n_alt, n_rej)


# ---------------------------------------------------------------------------
# G-buffer producer
# ---------------------------------------------------------------------------

def test_gbuffer_fronto_parallel_plane():
    sc = oracle.Scene(plane_scene([(5.0, "full", 0.0, 0)]))
    cam = axis_camera()
    prm = default_params()
    gb = oracle.gbuffer(sc, cam, prm, 32, 16)
    assert np.all(gb["prim"] == 0)
    assert np.allclose(gb["depth"], 5.0, rtol=0, atol=1e-12)
    assert np.allclose(gb["normal"], [0, 0, -1], atol=1e-15)
    alb = np.zeros(3)
    oracle.lib().or_albedo(prm["albedo_seed"], 0, alb.ctypes.data_as(C.c_void_p))
    assert np.all((alb >= 0.1) & (alb <= 0.9))
    l = np.asarray(prm["light_dir"], dtype=np.float32).astype(np.float64)
    l /= np.linalg.norm(l)
    lam = max(0.0, -np.dot([0, 0, -1], l))
    want = alb * (f32(prm["k_a"]) + f32(prm["k_d"]) * lam)
    assert np.allclose(gb["color"], want, atol=1e-12)


def test_gbuffer_ground_plane_depth_closed_form():
    """Camera at height h, pitched down: a ray with direction dir meets y = 0 at
    t = h / -dir_y; its depth along the optical axis is t (dir . fwd)."""
    sc = oracle.Scene(_ground_only())
    pose = camera_pose((0.0, 1.5, 0.0), pitch_deg=20.0)
    cam = Camera.from_poses(dict(f_m=0.05, f_number=2.0, focus_m=10.0, sensor_w_m=0.036), pose)
    W, H = 40, 30
    gb = oracle.gbuffer(sc, cam, default_params(), W, H)
    fwd = np.asarray(cam.fwd, dtype=np.float64)
    n_hit = 0
    for j in range(H):
        for i in range(W):
            d = oracle.pixel_dir(cam, W, H, i + 0.5, j + 0.5)
            if d[1] < -1e-3:
                t = f32(1.5) / -d[1]
                assert abs(gb["depth"][j, i] - t * np.dot(d, fwd)) <= 1e-9 * t
                n_hit += 1
            else:
                assert gb["prim"][j, i] < 0 and np.isinf(gb["depth"][j, i])
    assert n_hit > 100


def _ground_only():
    from synth.scenes import _Builder, ground
    b = _Builder(3)
    b.add("ground", *ground())
    return b.build()


# ---------------------------------------------------------------------------
# ray-traced layer: aperture -> 0 is a pinhole render
# ---------------------------------------------------------------------------

def test_aperture_zero_is_pinhole():
    w = make_workload("c1")
    sc = oracle.Scene(w.scene)
    cam = w.camera(0)
    cam.f_number = 1e30                     # a = f / N -> 0
    prm = dict(w.params, mask_near_hpx=0.0, spp=1)
    gb = oracle.gbuffer(sc, cam, prm, w.W, w.H)
    g32 = oracle.gbuffer_f32(gb)
    fr = oracle.frame(sc, cam, prm, w.W, w.H, g32)
    assert np.all(fr["nrays"] == 1)
    # the half-resolution pinhole render shoots through the same sensor points
    half = oracle.gbuffer(sc, cam, prm, w.W // 2, w.H // 2)
    prim = fr["ray_prim"][..., 0]
    mism = np.argwhere(prim != half["prim"])
    for (j, i) in mism:
        o, d = oracle.lens_ray(cam, prm, w.W, w.H, i, j, 0)
        assert sc.near_tie(o, d, prim[j, i], half["prim"][j, i])
    assert len(mism) <= 2
    ok = prim == half["prim"]
    col = fr["rt"][..., 2:5] + fr["rt"][..., 5:8]
    assert np.abs(col[ok] - half["color"][ok]).max() < 1e-12
    assert np.abs(fr["rt"][..., 1]).max() < 1e-20          # nothing is out of focus
    # zero aperture: the composite is the sharp image (Eq. 6 holds everywhere)
    assert np.abs(fr["out"][..., :3] - g32["color"][..., :3]).max() < 1e-12


# ---------------------------------------------------------------------------
# ray-traced layer: partial occlusion and the thin-lens integral (closed forms)
# ---------------------------------------------------------------------------

def _lens_geometry(W, f=0.05, N=1.4, d=10.0, ws=0.036):
    f, N, d, ws = f32(f), f32(N), f32(d), f32(ws)
    v = f * d / (d - f)
    return dict(A=0.5 * f / N, F=W * v / ws, d=d)


def test_partial_occlusion_circular_segment():
    """A foreground half-plane x > 0 at z1 = 1 m in front of a background plane at
    20 m, focus at 10 m.  The ray from lens point L towards the focus point P_f
    crosses z1 at x = L_x (1 - s) + P_fx s with s = z1 / d, so it is blocked iff
    L_x > -P_fx s / (1 - s): a circular segment of the lens disk."""
    W, H, spp = 512, 4, 4096
    sc = oracle.Scene(plane_scene([(1.0, "right", 0.0, 0), (20.0, "full", 0.0, 0)]))
    cam = axis_camera()
    prm = default_params(spp=spp, mask_near_hpx=0.0, max_coc_px=64.0)
    gb = oracle.gbuffer(sc, cam, prm, W, H)
    col_fg, col_bg = gb["color"][0, -1], gb["color"][0, 0]
    assert gb["prim"][0, -1] == 0 and gb["prim"][0, 0] == 1
    fr = oracle.frame(sc, cam, prm, W, H, oracle.gbuffer_f32(gb))
    g = _lens_geometry(W)
    s = 1.0 / g["d"]
    checked = 0
    for i in range(W // 2 // 2 - 12, W // 2 // 2 + 12):
        Pfx = g["d"] * ((2 * i + 1) - W / 2) / g["F"]
        tau = (-Pfx * s / (1 - s)) / g["A"]
        p = seg_fraction(tau)
        sig = math.sqrt(p * (1 - p) / spp)
        for j in range(H // 2):
            h = fr["rt"][j, i, 1]
            assert abs(h - p) <= 4.5 * sig + 1e-3, (i, tau, h, p)
            colr = fr["rt"][j, i, 2:5] + fr["rt"][j, i, 5:8]
            assert np.allclose(colr, h * col_fg + (1 - h) * col_bg, atol=1e-12)
            assert np.allclose(fr["rt"][j, i, 2:5], h * col_fg, atol=1e-12)
            checked += 1
    assert checked == 48


def _polygon_share_right_of(n, tau):
    """Share of the regular n-gon (circumradius 1, a vertex at angle 0) with x > tau,
    by clipping its vertex list against the half-plane and the shoelace formula."""
    ang = 2 * np.pi * np.arange(n) / n
    pts = list(zip(np.cos(ang), np.sin(ang)))
    out = []
    for k in range(n):
        a, b = pts[k], pts[(k + 1) % n]
        if a[0] > tau:
            out.append(a)
        if (a[0] > tau) != (b[0] > tau):
            t = (tau - a[0]) / (b[0] - a[0])
            out.append((tau, a[1] + t * (b[1] - a[1])))
    if len(out) < 3:
        return 0.0
    x, y = np.array(out).T
    area = 0.5 * abs(np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y))
    return min(1.0, area / (0.5 * n * np.sin(2 * np.pi / n)))


@pytest.mark.parametrize("n", [5, 6])
def test_partial_occlusion_polygonal_aperture(n):
    """The partial-occlusion scene above with an n-blade aperture: a ray is blocked iff
    its lens point has L_x > -P_fx s / (1 - s), so the blocked share is the part of the
    n-gon right of that line (the pentagon is not symmetric about x = 0, so this also
    fixes the aperture's orientation along the camera's right axis)."""
    W, H, spp = 512, 4, 4096
    sc = oracle.Scene(plane_scene([(1.0, "right", 0.0, 0), (20.0, "full", 0.0, 0)]))
    cam = axis_camera()
    prm = default_params(spp=spp, mask_near_hpx=0.0, max_coc_px=64.0, aperture_blades=n)
    gb = oracle.gbuffer(sc, cam, prm, W, H)
    fr = oracle.frame(sc, cam, prm, W, H, oracle.gbuffer_f32(gb))
    g = _lens_geometry(W)
    s = 1.0 / g["d"]
    shares = []
    for i in range(W // 2 // 2 - 12, W // 2 // 2 + 12):
        Pfx = g["d"] * ((2 * i + 1) - W / 2) / g["F"]
        tau = (-Pfx * s / (1 - s)) / g["A"]
        p = _polygon_share_right_of(n, tau)
        shares.append(p)
        sig = math.sqrt(p * (1 - p) / spp)
        for j in range(H // 2):
            h = fr["rt"][j, i, 1]
            assert abs(h - p) <= 4.5 * sig + 1e-3, (i, tau, h, p)
    # the polygon's shares differ from the disk's where the line crosses it
    disk = [seg_fraction(-Pfx * s / (1 - s) / g["A"]) for Pfx in
            [g["d"] * ((2 * i + 1) - W / 2) / g["F"] for i in range(W // 4 - 12, W // 4 + 12)]]
    assert max(abs(a - b) for a, b in zip(shares, disk)) > 0.02


def test_thin_lens_step_edge_behind_focus():
    """A coplanar colour step at z = 30 m (behind the 10 m focus plane): the ray
    lands at x = L_x (1 - s) + P_fx s, s = 3, so it lands right of the edge iff
    L_x < 1.5 P_fx -- the step is blurred by the disk of the thin-lens integral."""
    W, H, spp = 512, 4, 4096
    sc = oracle.Scene(plane_scene([(30.0, "left", 0.0, 0), (30.0, "right", 0.0, 0)]))
    cam = axis_camera()
    prm = default_params(spp=spp, mask_near_hpx=0.0, max_coc_px=64.0)
    gb = oracle.gbuffer(sc, cam, prm, W, H)
    fr = oracle.frame(sc, cam, prm, W, H, oracle.gbuffer_f32(gb))
    g = _lens_geometry(W)
    s = 30.0 / g["d"]
    for i in range(W // 4 - 16, W // 4 + 16):
        Pfx = g["d"] * ((2 * i + 1) - W / 2) / g["F"]
        tau0 = Pfx * s / (s - 1.0)
        p_right = 1.0 - seg_fraction(tau0 / g["A"])
        sig = math.sqrt(p_right * (1 - p_right) / spp)
        for j in range(H // 2):
            rays = fr["ray_prim"][j, i]
            got = np.mean(rays == 1)
            assert np.all((rays == 0) | (rays == 1))
            assert abs(got - p_right) <= 4.5 * sig + 1e-3, (i, got, p_right)
            assert fr["rt"][j, i, 1] == 0.0             # far field only


# ---------------------------------------------------------------------------
# post-process invariants and library cross-checks
# ---------------------------------------------------------------------------

def _run_stage_frame(name="c2", W=200, H=112, **over):
    w = make_workload(name, W=W, H=H)
    sc = oracle.Scene(w.scene)
    cam = w.camera(0)
    prm = dict(w.params, **over)
    gb = oracle.gbuffer(sc, cam, prm, W, H)
    g32 = oracle.gbuffer_f32(gb)
    return w, sc, cam, prm, g32, oracle.frame(sc, cam, prm, W, H, g32)


def test_uniform_colour_is_fixed_point_of_post_process():
    w, sc, cam, prm, g32, _ = _run_stage_frame()
    g = dict(g32)
    g["color"] = np.empty_like(g32["color"])
    g["color"][...] = np.float32([0.3, 0.55, 0.7, 1.0])
    fr = oracle.frame(sc, cam, prm, w.W, w.H, g)
    want = np.float32([0.3, 0.55, 0.7]).astype(np.float64)
    for k in ("pp_in", "pre", "main_out", "pp_med"):
        assert np.abs(fr[k][..., :3] - want).max() < 1e-12, k
    assert np.abs(fr["main_out"][..., 3]).max() == 0.0         # no bright samples
    # a uniform emitter colour (luminance 6 > bright_lum + bright_ramp): every tap is
    # bright, so the bright fraction is 1 and the colour is still a fixed point
    bright = np.float32([5.0, 6.0, 7.0])
    g["color"][...] = np.append(bright, np.float32(1.0))
    assert float(bright.astype(np.float64) @ [0.2126, 0.7152, 0.0722]) > prm["bright_lum"] + prm["bright_ramp"]
    fr = oracle.frame(sc, cam, prm, w.W, w.H, g)
    for k in ("pp_in", "pre", "main_out", "pp_med"):
        assert np.abs(fr[k][..., :3] - bright.astype(np.float64)).max() < 1e-12, k
    assert np.abs(fr["main_out"][..., 3] - 1.0).max() < 1e-12


def test_downscale_and_tiles_by_definition():
    w, sc, cam, prm, g32, fr = _run_stage_frame(W=202, H=114)
    H2, W2 = w.H // 2, w.W // 2
    col = g32["color"][..., :3].astype(np.float64).reshape(H2, 2, W2, 2, 3).mean(axis=(1, 3))
    assert np.abs(fr["pp_in"][..., :3] - col).max() < 1e-12
    z = np.minimum(g32["depth"].astype(np.float64), prm["z_far_m"]).reshape(H2, 2, W2, 2)
    assert np.array_equal(fr["z_h"], z.min(axis=(1, 3)))
    rmax = prm["max_coc_px"] / 2
    for (j, i) in [(0, 0), (H2 - 1, W2 - 1), (17, 33), (40, 90)]:
        want = np.clip(oracle.coc(cam, w.W, fr["z_h"][j, i]) / 4.0, -rmax, rmax)
        assert abs(fr["pp_in"][j, i, 3] - want) < 1e-12
    # tile max (ragged: 101 x 57 hpx in 8 x 8 tiles) and dilation vs scipy
    T = prm["tile"]
    rho = fr["pp_in"][..., 3]
    TH, TW = fr["tile_raw"].shape[:2]
    pad = np.full((TH * T, TW * T), np.nan)
    pad[:H2, :W2] = rho
    blocks = pad.reshape(TH, T, TW, T)
    assert np.array_equal(fr["tile_raw"][..., 0], np.nanmax(np.maximum(0, -blocks), axis=(1, 3)))
    assert np.array_equal(fr["tile_raw"][..., 1], np.nanmax(np.abs(blocks), axis=(1, 3)))
    K = math.ceil(rmax / T)
    for c in range(2):
        ref = ndi.maximum_filter(fr["tile_raw"][..., c], size=2 * K + 1, mode="constant", cval=0.0)
        assert np.array_equal(fr["tile_dil"][..., c], ref)


def test_median_is_exact_selection():
    rng = np.random.default_rng(0)
    L = oracle.lib()
    for k in range(1, 10):
        for _ in range(50):
            v = rng.normal(size=9)
            out = np.zeros(1)
            L.or_median9(v.ctypes.data_as(C.c_void_p), k, out.ctypes.data_as(C.c_void_p))
            if k % 2:
                assert out[0] == np.median(v[:k])
            else:
                assert out[0] == np.sort(v[:k])[(k - 1) // 2]
    # the PP median postfilter equals scipy's 3x3 median with edge replication
    w, sc, cam, prm, g32, fr = _run_stage_frame(W=98, H=66)
    for c in range(4):
        ref = ndi.median_filter(fr["main_out"][..., c], size=3, mode="nearest")
        assert np.array_equal(fr["pp_med"][..., c], ref)


def test_binomial_and_sobel_vs_scipy_and_ramp():
    L = oracle.lib()
    rng = np.random.default_rng(2)
    img = rng.normal(size=(23, 31))
    out = np.zeros_like(img)
    L.or_binomial5(img.ctypes.data_as(C.c_void_p), 31, 23, 1, out.ctypes.data_as(C.c_void_p))
    b = np.array([1, 4, 6, 4, 1.0]) / 16
    assert np.allclose(out, ndi.correlate(img, np.outer(b, b), mode="nearest"), atol=1e-13)
    gx, gy = np.zeros_like(img), np.zeros_like(img)
    L.or_sobel5(img.ctypes.data_as(C.c_void_p), 31, 23, 1, 0, gx.ctypes.data_as(C.c_void_p),
                gy.ctypes.data_as(C.c_void_p))
    sm = np.array([1, 4, 6, 4, 1.0])
    dv = np.array([-1, -2, 0, 2, 1.0])
    assert np.allclose(gx, ndi.correlate(img, np.outer(sm, dv) / 128, mode="nearest"), atol=1e-13)
    assert np.allclose(gy, ndi.correlate(img, np.outer(dv, sm) / 128, mode="nearest"), atol=1e-13)
    # a linear ramp of slope 0.37 per pixel (away from the clamped border)
    jj, ii = np.mgrid[0:23, 0:31]
    ramp = 0.37 * ii - 1.1 * jj + 4.0
    L.or_sobel5(ramp.ctypes.data_as(C.c_void_p), 31, 23, 1, 0, gx.ctypes.data_as(C.c_void_p),
                gy.ctypes.data_as(C.c_void_p))
    assert np.allclose(gx[2:-2, 2:-2], 0.37, atol=1e-13)
    assert np.allclose(gy[2:-2, 2:-2], -1.1, atol=1e-13)


def test_mask_counts():
    w, sc, cam, prm, g32, fr = _run_stage_frame()
    T = prm["tile"]
    near = np.repeat(np.repeat(fr["tile_dil"][..., 0], T, 0), T, 1)[:w.H // 2, :w.W // 2]
    assert np.array_equal(fr["nrays"] > 0, near >= f32(prm["mask_near_hpx"]))
    assert set(np.unique(fr["nrays"])) <= {0, prm["spp"]}
    # a fronto-parallel plane has no edges: x_n = 0 away from the border
    sc2 = oracle.Scene(plane_scene([(5.0, "full", 0.0, 0)]))
    cam2 = axis_camera()
    prm2 = default_params(ray_mode=1, m=10)
    gb = oracle.gbuffer(sc2, cam2, prm2, 64, 48)
    fr2 = oracle.frame(sc2, cam2, prm2, 64, 48, oracle.gbuffer_f32(gb))
    assert np.abs(fr2["xn"]).max() < 1e-12
    # adaptive mode: 1 <= n <= m, n = ceil(x_f) where masked
    w, sc, cam, prm, g32, fr = _run_stage_frame(ray_mode=1, m=10)
    msk = fr["nrays"] > 0
    assert fr["nrays"].max() <= 10
    assert np.array_equal(fr["nrays"][msk], np.clip(np.ceil(fr["xf"][msk]), 1, 10).astype(np.int32))
    # Eq. 3 / Eq. 4 ranges
    assert fr["xn"].min() >= 0 and fr["xn"].max() <= 1
    assert fr["xf"].max() <= 10


# ---------------------------------------------------------------------------
# temporal accumulation
# ---------------------------------------------------------------------------

def _accumulate(cam, prm, W, H, z_h, rt, nrays, hist_in, has):
    L = oracle.lib()
    H2, W2 = H // 2, W // 2
    N = W2 * H2
    hist_out, crt, ct, var = np.zeros(12 * N), np.zeros((H2, W2, 4)), np.zeros((H2, W2)), np.zeros((H2, W2))
    c, p = oracle.camera(cam), oracle.params(prm)
    vp = lambda a: a.ctypes.data_as(C.c_void_p)
    L.or_accumulate(C.byref(c), C.byref(p), W, H, vp(z_h), vp(rt), vp(nrays), vp(hist_in), int(has),
                    vp(hist_out), vp(crt), vp(ct), vp(var))
    return hist_out, crt, ct, var


def _rt_field(H2, W2, colour, h, cn=2.0, cf=3.0):
    rt = np.zeros((H2, W2, 14))
    rt[..., 0] = 1
    rt[..., 1] = h
    rt[..., 2:5] = h * np.asarray(colour)
    rt[..., 5:8] = (1 - h) * np.asarray(colour)
    rt[..., 8] = h * cn
    rt[..., 9] = (1 - h) * cf
    return rt


def test_ema_closed_form_static_camera():
    W, H = 48, 32
    H2, W2 = H // 2, W // 2
    cam = axis_camera()
    prm = default_params()
    alpha = f32(prm["alpha"])
    z_h = np.full((H2, W2), 5.0)
    nr = np.ones((H2, W2), dtype=np.int32)
    A, B = np.array([0.9, 0.2, 0.4]), np.array([0.1, 0.6, 0.3])
    hist, crt, ct, var = _accumulate(cam, prm, W, H, z_h, _rt_field(H2, W2, A, 0.25), nr, np.zeros(12 * W2 * H2), 0)
    assert np.allclose(crt[..., :3], A, atol=1e-15)
    assert np.all(var == 0.0)
    for k in range(1, 9):
        hist, crt, ct, var = _accumulate(cam, prm, W, H, z_h, _rt_field(H2, W2, B, 0.25), nr, hist, 1)
        want = alpha ** k * A + (1 - alpha ** k) * B
        assert np.abs(crt[..., :3] - want).max() < 1e-12, k
        assert np.abs(crt[..., 3] - 0.25).max() < 1e-12
        assert np.abs(ct - (0.25 * 2 + 0.75 * 3)).max() < 1e-12
    # luminance moments of a sequence (lum A, then lum B k times)
    la = 0.2126 * A[0] + 0.7152 * A[1] + 0.0722 * A[2]
    lb = 0.2126 * B[0] + 0.7152 * B[1] + 0.0722 * B[2]
    wa = alpha ** 8
    m1, m2 = wa * la + (1 - wa) * lb, wa * la * la + (1 - wa) * lb * lb
    assert np.abs(var - (m2 - m1 * m1)).max() < 1e-12


def test_reprojection_integer_shift():
    """Move the camera sideways so that a plane at 5 m shifts by one half-resolution
    pixel: every pixel's history comes from its right-hand neighbour."""
    W, H = 64, 32
    H2, W2 = H // 2, W // 2
    g = _lens_geometry(W)
    delta = f32(2.0 * 5.0 / g["F"])              # 2 full-res px at depth 5 m
    cam = axis_camera(pos=(delta, 0.0, 0.0), prev_pos=(0.0, 0.0, 0.0))
    prm = default_params()
    am = f32(prm["alpha_motion"])
    z_h = np.full((H2, W2), 5.0)
    nr = np.ones((H2, W2), dtype=np.int32)
    hist = np.zeros((H2, W2, 12))
    ii = np.arange(W2)[None, :] + 0 * np.arange(H2)[:, None]
    hist[..., 0] = ii * 0.01 + 0.1                # An red varies with x
    hist[..., 6] = 1.0                           # h = 1, g = 0 (valid)
    cur = _rt_field(H2, W2, [0.5, 0.5, 0.5], 1.0)
    hout, crt, ct, var = _accumulate(cam, prm, W, H, z_h, cur, nr, hist.reshape(-1), 1)
    hout = hout.reshape(H2, W2, 12)
    want = am * hist[:, 1:, 0] + (1 - am) * 0.5
    assert np.abs(hout[:, :-1, 0] - want).max() < 1e-6
    # the last column reprojects outside the image: no history, the current value
    assert np.abs(hout[:, -1, 0] - 0.5).max() < 1e-6


# ---------------------------------------------------------------------------
# reconstruction and composite
# ---------------------------------------------------------------------------

def test_recon_blend_limits():
    L = oracle.lib()
    W2, H2 = 40, 24
    rng = np.random.default_rng(4)
    med = np.concatenate([rng.uniform(0, 1, (H2, W2, 3)), rng.uniform(0, 1, (H2, W2, 1))], -1)
    ct = rng.uniform(0, 8, (H2, W2))
    nr = np.ones((H2, W2), dtype=np.int32)
    nr[:, :5] = 0
    med[:, :5] = 0
    prm = oracle.params(default_params())
    vp = lambda a: a.ctypes.data_as(C.c_void_p)
    out = np.zeros_like(med)
    L.or_recon(C.byref(prm), W2, H2, vp(med), vp(ct), vp(np.zeros((H2, W2))), vp(nr), vp(out))
    assert np.array_equal(out, med)                     # b = 0 (Eq. 5) keeps the pixel
    uni = np.zeros_like(med)
    uni[:, 5:] = [0.2, 0.4, 0.6, 0.3]
    L.or_recon(C.byref(prm), W2, H2, vp(uni), vp(ct), vp(np.full((H2, W2), 1.0)), vp(nr), vp(out))
    assert np.abs(out[:, 5:] - [0.2, 0.4, 0.6, 0.3]).max() < 1e-12   # normalised filter
    assert np.all(out[:, :5] == 0)


def test_composite_special_cases():
    L = oracle.lib()
    W, H = 512, 8            # at this width c(0.3 m) ~ -83 px and c(1e4 m) ~ +2.5 px
    W2, H2 = W // 2, H // 2
    cam = axis_camera()
    prm = default_params()
    P, S, R = np.array([0.2, 0.3, 0.4]), np.array([0.9, 0.8, 0.7]), np.array([0.5, 0.1, 0.6])
    color4 = np.zeros((H, W, 4), dtype=np.float32)
    color4[..., :3] = S
    vp = lambda a: a.ctypes.data_as(C.c_void_p)

    def run(z, bright, h, rays):
        depth = np.full((H, W), z, dtype=np.float32)
        pp = np.zeros((H2, W2, 4)); pp[..., :3] = P; pp[..., 3] = bright
        rc = np.zeros((H2, W2, 4)); rc[..., :3] = R; rc[..., 3] = h
        nr = np.full((H2, W2), rays, dtype=np.int32)
        out = np.zeros((H, W, 4))
        L.or_composite(C.byref(oracle.camera(cam)), C.byref(oracle.params(prm)), W, H, vp(color4),
                       vp(depth), vp(pp), vp(rc), vp(nr), vp(out))
        return out[..., :3].astype(np.float32).astype(np.float64)

    S32, P32, R32 = (np.float32(x).astype(np.float64) for x in (S, P, R))
    tol = 1e-6
    assert np.abs(run(10.0, 0.5, 0.5, 1) - S32).max() < tol             # in focus: sharp
    assert np.abs(run(0.3, 0.0, 0.5, 0) - P32).max() < tol              # no rays: PP
    assert np.abs(run(0.3, 0.0, 0.5, 1) - R32).max() < tol              # near, not bright: RT
    assert np.abs(run(0.3, 1.0, 0.5, 1) - P32).max() < tol              # near, bright: PP
    assert np.abs(run(1e4, 0.0, 0.0, 1) - R32).max() < tol              # far, h = 0: RT
    assert np.abs(run(1e4, 0.0, 0.3, 1) - P32).max() < tol              # far, h >= 0.3: PP
    mid = run(1e4, 0.0, 0.15, 1)                                        # smoothstep(0.5) = 0.5
    assert np.abs(mid - 0.5 * (R32 + P32)).max() < tol


def test_default_params_are_the_papers():
    with open(os.path.join(HERE, "golden", "paper_constants.json")) as fh:
        g = json.load(fh)
    p = default_params()
    for k in ("s", "var_w_mask", "alpha", "var_w_recon", "b_max", "h_edge", "lod_scale",
              "lod_max", "depth_range_m"):
        assert p[k] == g[k]["value"], k


def test_forced_ray_counts_are_taken_and_neutral():
    """The test hook for count ties: forcing the mask's own counts reproduces the frame
    bit for bit; a forced count is the one traced."""
    import oracle
    from synth import make_workload
    w = make_workload("c1", W=64, H=36)
    prm = dict(w.params)
    osc = oracle.Scene(w.scene)
    cam = w.camera(0)
    gb = oracle.gbuffer_f32(oracle.gbuffer(osc, cam, prm, w.W, w.H))
    a = oracle.frame(osc, cam, prm, w.W, w.H, gb, oracle.History(w.W, w.H))
    b = oracle.frame(osc, cam, prm, w.W, w.H, gb, oracle.History(w.W, w.H), nrays_force=a["nrays"])
    for k in ("nrays", "rt", "out", "hist_out"):
        assert np.array_equal(a[k], b[k]), k
    force = np.full(a["nrays"].shape, -1, np.int32)
    masked = np.argwhere(a["nrays"] > 0)
    assert len(masked) > 0
    j, i = masked[0]
    force[j, i] = 0
    c = oracle.frame(osc, cam, prm, w.W, w.H, gb, oracle.History(w.W, w.H), nrays_force=force)
    assert c["nrays"][j, i] == 0 and c["rt"][j, i, 0] == 0.0
    other = np.ones(a["nrays"].shape, bool)
    other[j, i] = False
    assert np.array_equal(c["nrays"][other], a["nrays"][other])


def test_forced_hits_are_taken():
    """The test hook for near-tie hits: forcing the closest hits reproduces the frame
    (the forced hit's distance is its plane's, equal to the hit distance up to
    rounding); a forced miss makes that ray see the sky and changes only its pixel."""
    import oracle
    from synth import make_workload
    w = make_workload("c1", W=64, H=36)
    prm = dict(w.params)
    osc = oracle.Scene(w.scene)
    cam = w.camera(0)
    gb = oracle.gbuffer_f32(oracle.gbuffer(osc, cam, prm, w.W, w.H))
    a = oracle.frame(osc, cam, prm, w.W, w.H, gb, oracle.History(w.W, w.H))
    b = oracle.frame(osc, cam, prm, w.W, w.H, gb, oracle.History(w.W, w.H), hit_force=a["ray_prim"])
    assert np.array_equal(a["ray_prim"], b["ray_prim"])
    assert np.allclose(a["rt"], b["rt"], rtol=1e-10, atol=1e-10)
    hits = np.argwhere((a["ray_prim"][..., 0] >= 0) & (a["nrays"] > 0))
    j, i = hits[0]
    force = np.full(a["ray_prim"].shape, -2, np.int32)
    force[j, i, 0] = -1
    c = oracle.frame(osc, cam, prm, w.W, w.H, gb, oracle.History(w.W, w.H), hit_force=force)
    assert c["ray_prim"][j, i, 0] == -1
    other = np.ones(a["nrays"].shape, bool)
    other[j, i] = False
    assert np.array_equal(c["rt"][other], a["rt"][other])
    assert not np.array_equal(c["rt"][j, i], a["rt"][j, i])


def _taa_cam(pos=(0.0, 1.0, 0.0), prev=None, jitter=(0.0, 0.0), prev_jitter=(0.0, 0.0)):
    intr = dict(f_m=0.035, f_number=2.0, focus_m=20.0, sensor_w_m=0.036)
    cam = Camera.from_poses(intr, camera_pose(pos, pitch_deg=0.0), camera_pose(prev or pos, pitch_deg=0.0))
    cam.jitter, cam.prev_jitter = jitter, prev_jitter
    return cam


def _bilinear_clamped(img, u, v):
    """img (H, W, C) sampled at texel coordinates (u, v) (centres at integers), clamp to edge."""
    H, W = img.shape[:2]
    x0, y0 = np.floor(u).astype(int), np.floor(v).astype(int)
    fx, fy = u - x0, v - y0
    out = np.zeros(u.shape + img.shape[2:])
    for dy in (0, 1):
        for dx in (0, 1):
            xi, yi = np.clip(x0 + dx, 0, W - 1), np.clip(y0 + dy, 0, H - 1)
            w = (fx if dx else 1 - fx) * (fy if dy else 1 - fy)
            out += w[..., None] * img[yi, xi]
    return out


def _taa_expected(cur, hist_sampled, alpha):
    lo = ndi.minimum_filter(cur[..., :3], size=(3, 3, 1), mode="nearest")
    hi = ndi.maximum_filter(cur[..., :3], size=(3, 3, 1), mode="nearest")
    hc = np.minimum(np.maximum(hist_sampled[..., :3], lo), hi)
    return hc + alpha * (cur[..., :3] - hc)


@pytest.mark.parametrize("case", ["static", "jitter", "pan"])
def test_taa_matches_reprojection_closed_forms(case):
    """Final TAA (Section 3.4, Karis 2014): history reprojected onto the newest frame,
    clamped to the current 3x3 neighbourhood, blended with alpha.  On a fronto-parallel
    wall at distance Z: a static camera reprojects every pixel to itself; jitter alone
    shifts the history by (j - j_prev); a sideways move by dx shifts it by F dx / Z
    (F the focal length in pixels) -- checked against numpy shifts with bilinear taps."""
    W, H, Z, alpha = 48, 32, 7.0, 0.1
    rng = np.random.default_rng(3)
    cur = rng.uniform(0, 1, (H, W, 4))
    hist = rng.uniform(0, 1, (H, W, 4))
    depth = np.full((H, W), Z, np.float32)
    F = W * (0.035 * 20.0 / (20.0 - 0.035)) / 0.036
    ys, xs = np.mgrid[0:H, 0:W].astype(float)
    if case == "static":
        cam, su, sv = _taa_cam(), xs, ys
    elif case == "jitter":
        j, pj = (0.25, -0.125), (-0.375, 0.0625)
        cam = _taa_cam(jitter=j, prev_jitter=pj)
        su, sv = xs + j[0] - pj[0], ys + j[1] - pj[1]
    else:
        dx = 0.02
        cam = _taa_cam(pos=(dx, 1.0, 0.0), prev=(0.0, 1.0, 0.0))
        su, sv = xs + F * dx / Z, ys
    prm = default_params(taa_alpha=alpha)
    got = oracle.taa(cam, prm, W, H, depth, cur, hist)
    want = _taa_expected(cur, _bilinear_clamped(hist, su, sv), alpha)
    assert np.allclose(got[..., :3], want, atol=1e-9), np.abs(got[..., :3] - want).max()
    assert np.all(got[..., 3] == 1.0)
    # no previous frame: the current image
    first = oracle.taa(cam, prm, W, H, depth, cur, None)
    assert np.array_equal(first[..., :3], cur[..., :3])


# ---- polygonal aperture (Section 1.1: bokeh takes the aperture's shape, polygonal for
# an n-blade diaphragm; Section 2.2: the kernel's shape can be changed to produce it) ----

def _support_norm(n, x, y):
    """Polygon norm of (x, y) for the regular n-gon of circumradius 1 with a vertex at
    angle 0, from its edge normals (angles (2k + 1) pi / n) and apothem cos(pi / n):
    1 exactly on the boundary.  Independent of the oracle's radial formula."""
    ang = (2 * np.arange(n) + 1) * np.pi / n
    return np.max(np.cos(ang) * x + np.sin(ang) * y) / np.cos(np.pi / n)


@pytest.mark.parametrize("n", [3, 4, 5, 6, 7, 8])
def test_polygon_boundary_and_area_against_geometry(n):
    """The boundary radius agrees with the support-function norm of the n-gon, its
    vertices sit on the unit circle, and the area equals the shoelace area."""
    for th in np.linspace(-3.0, 9.0, 997):
        r = oracle.poly_rho(n, th)
        assert _support_norm(n, r * np.cos(th), r * np.sin(th)) == pytest.approx(1.0, abs=1e-12)
    for k in range(n):
        assert oracle.poly_rho(n, 2 * np.pi * k / n) == pytest.approx(1.0, abs=1e-12)
    vx = np.cos(2 * np.pi * np.arange(n) / n)
    vy = np.sin(2 * np.pi * np.arange(n) / n)
    shoelace = 0.5 * abs(np.sum(vx * np.roll(vy, -1) - np.roll(vx, -1) * vy))
    assert oracle.poly_area(n) == pytest.approx(shoelace, rel=1e-13)
    assert oracle.poly_rho(0, 1.234) == 1.0 and oracle.poly_area(0) == pytest.approx(np.pi, rel=1e-15)


@pytest.mark.parametrize("n", [0, 3, 5, 6, 8])
def test_aperture_point_is_uniform_over_the_aperture(n):
    """Lens points from a midpoint grid of the two uniforms: all inside the aperture,
    centred, with the second moment of the uniform n-gon, (2 + cos(2 pi / n)) / 6
    (1/2 for the disk), and a quarter of them inside the aperture scaled by 1/2."""
    g = (np.arange(240) + 0.5) / 240
    pts = np.array([oracle.aperture_point(n, u1, u2) for u1 in g for u2 in g])
    if n:
        norms = np.array([_support_norm(n, x, y) for x, y in pts])
    else:
        norms = np.hypot(pts[:, 0], pts[:, 1])
    assert norms.max() <= 1.0 + 1e-12
    assert np.abs(pts.mean(axis=0)).max() < 1e-3
    m2 = (pts ** 2).sum(axis=1).mean()
    want = 0.5 if n == 0 else (2.0 + np.cos(2 * np.pi / n)) / 6.0
    assert m2 == pytest.approx(want, abs=2e-4)
    assert (norms <= 0.5).mean() == pytest.approx(0.25, abs=3e-3)


@pytest.mark.parametrize("n", [0, 3, 4, 5, 6, 8])
def test_ring_taps_lie_on_the_aperture_shape(n):
    """Tap t of the 81-tap kernel: centre, then rings k = 1..4 of 8k taps in the
    directions 2 pi m / (8k), each on the aperture's boundary scaled by k / 4."""
    assert np.allclose(oracle.ring_tap(n, 0), [0.0, 0.0, 0.0])
    t = 1
    for k in range(1, 5):
        for m in range(8 * k):
            x, y, frac = oracle.ring_tap(n, t)
            assert frac == k / 4.0
            th = 2 * np.pi * m / (8 * k)
            # same direction as the circular tap
            assert x * np.sin(th) - y * np.cos(th) == pytest.approx(0.0, abs=1e-12)
            assert x * np.cos(th) + y * np.sin(th) > 0.0
            norm = np.hypot(x, y) if n == 0 else _support_norm(n, x, y)
            assert norm == pytest.approx(1.0, abs=1e-12)
            t += 1
    assert t == 81


# ---------------------------------------------------------------------------
# post-process filter values (Section 3.1.1-3.1.2): consequences of the weights that the
# uniform-image fixed point does not see
# ---------------------------------------------------------------------------

def _pp_params(**kw):
    return oracle.params(dict(default_params(), **kw))


def _main_filter(pre, z, R):
    """The oracle's A4 on hand-made inputs: pre (H2, W2, 4) = (rgb, rho), z (H2, W2),
    every tile's dilated radius R."""
    H2, W2 = z.shape
    T = 8
    TH, TW = -(-H2 // T), -(-W2 // T)
    dil = np.zeros((TH, TW, 2))
    dil[..., 0] = dil[..., 1] = R
    pre = np.ascontiguousarray(pre, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    out = np.zeros((H2, W2, 4))
    p = _pp_params()
    oracle.lib().or_main_filter(C.byref(p), W2, H2, oracle._p(pre), oracle._p(z), oracle._p(dil), oracle._p(out))
    return out


def _prefilter(pp_in, R):
    H2, W2 = pp_in.shape[:2]
    TH, TW = -(-H2 // 8), -(-W2 // 8)
    dil = np.zeros((TH, TW, 2))
    dil[..., 0] = dil[..., 1] = R
    pp_in = np.ascontiguousarray(pp_in, dtype=np.float64)
    out = np.zeros((H2, W2, 4))
    p = _pp_params()
    oracle.lib().or_prefilter(C.byref(p), W2, H2, oracle._p(pp_in), oracle._p(dil), oracle._p(out))
    return out


def _ring_taps():
    """The 81-tap layout as the paper describes it (Section 3.1.2): the centre and rings
    k = 1..4 of 8k taps at radius k/4 of the kernel radius, evenly spaced in angle."""
    taps = [(0.0, 0.0, 0.0)]
    for k in range(1, 5):
        for m in range(8 * k):
            th = 2 * math.pi * m / (8 * k)
            taps.append((math.cos(th), math.sin(th), k / 4.0))
    return taps


A_COL, B_COL = np.array([0.9, 0.2, 0.1]), np.array([0.1, 0.3, 0.8])


def _two_regions(W2, H2, xb, left, right):
    """Columns x <= xb take `left` = (colour, rho, z), the others `right`."""
    pre = np.zeros((H2, W2, 4))
    z = np.zeros((H2, W2))
    for (sl, (col, rho, zz)) in ((np.s_[:, :xb + 1], left), (np.s_[:, xb + 1:], right)):
        pre[sl + (np.s_[:3],)] = col
        pre[sl + (3,)] = rho
        z[sl] = zz
    return pre, z


def test_main_filter_in_focus_pixel_in_front_stays_sharp():
    """A pixel in focus (rho 0) nearer than a blurred region beside it takes nothing of
    that region: every tap that lands there is background for it, and a background tap
    counts only within min(its CoC, the centre's CoC) = 0 (+ half the ramp) of the centre.
    A foreground/background split that used the tap's own CoC for the background would
    blur it."""
    W2, H2, R = 64, 48, 12.0
    pre, z = _two_regions(W2, H2, 31, (A_COL, 0.0, 2.0), (B_COL, 12.0, 10.0))
    out = _main_filter(pre, z, R)
    for x in range(20, 32):
        assert np.abs(out[24, x, :3] - A_COL).max() < 1e-12, x


def test_main_filter_foreground_bleeds_within_its_radius():
    """A blurred foreground (rho -12, 1 m) beside an in-focus background (rho 0, 10 m):
    background pixels within the foreground's reach take some of its colour (the
    foreground scatters over the background, Section 3.1.2), the share falls with the
    distance, and from the kernel radius on none is left.  A split that limited the
    foreground's coverage by the centre's CoC would show no bleeding at all."""
    W2, H2, R = 64, 48, 12.0
    pre, z = _two_regions(W2, H2, 23, (A_COL, -12.0, 1.0), (B_COL, 0.0, 10.0))
    out = _main_filter(pre, z, R)
    share = lambda x: float((out[24, x, 0] - B_COL[0]) / (A_COL[0] - B_COL[0]))
    shares = [share(x) for x in range(24, 24 + int(R))]
    assert shares[0] > 0.05 and min(shares) > 0.0, shares
    # the ring taps are discrete, so the share falls in steps: taken two columns at a
    # time it decreases strictly
    pairs = [0.5 * (a + b) for a, b in zip(shares[0::2], shares[1::2])]
    assert all(a > b for a, b in zip(pairs, pairs[1:])), shares
    for x in range(24 + int(R), W2):
        assert np.abs(out[24, x, :3] - B_COL).max() < 1e-12, x


def test_main_filter_sample_alpha_is_inverse_area():
    """sampleAlpha (Section 3.1.2, 'pixel area over blur-disk area'): with the same taps
    landing on a fully covering foreground, doubling the foreground's CoC quarters its
    weight against the in-focus centre.  From out = (w0 B + g w0 A) / (w0 + g w0) the ratio
    g = (out - B) / (A - out) of the two runs must be (26 / 13)^2 = 4; the boundary column
    is chosen so that no tap's bilinear footprint straddles it."""
    W2, H2, R = 80, 48, 12.0
    x0, y0 = 40, 24
    xs = [x0 + d * R * ux for (ux, uy, d) in _ring_taps()]
    # the last foreground column c: no tap with floor(x) == c (no straddling footprint),
    # at least a few taps on the foreground side
    c = next(c for c in range(x0 - 2, x0 - int(R), -1)
             if all(math.floor(x) != c for x in xs) and sum(x < c + 1 for x in xs) >= 4)
    gs = []
    for rho in (-13.0, -26.0):
        pre, z = _two_regions(W2, H2, c, (A_COL, rho, 1.0), (B_COL, 0.0, 10.0))
        out = _main_filter(pre, z, R)
        g = (out[y0, x0, :3] - B_COL) / (A_COL - out[y0, x0, :3])
        assert np.allclose(g, g[0], rtol=1e-9)
        gs.append(g[0])
    assert abs(gs[0] / gs[1] - 4.0) < 1e-9, gs


def test_filters_with_uniform_coc_are_plain_means_of_their_taps():
    """With one CoC everywhere (covering every tap) and one depth, the main filter's taps
    all weigh the same and the prefilter's CoC-similarity weight is 1: each is the plain
    mean of its bilinear samples (scipy's map_coordinates, order 1, at the tap positions
    the paper describes; prefilter: the centre and 8 taps at angles k pi/4, radius
    max(R/8, sqrt(2)/2))."""
    from scipy.ndimage import map_coordinates
    rng = np.random.default_rng(3)
    W2, H2, R, rho = 72, 56, 9.0, 10.0
    col = rng.uniform(0.1, 0.9, (H2, W2, 3))
    pre = np.concatenate([col, np.full((H2, W2, 1), rho)], -1)
    z = np.full((H2, W2), 5.0)
    out = _main_filter(pre, z, R)
    taps = _ring_taps()
    for (j, i) in [(28, 36), (20, 25), (40, 50)]:
        ys = np.array([j + d * R * uy for (ux, uy, d) in taps])
        xs = np.array([i + d * R * ux for (ux, uy, d) in taps])
        want = [map_coordinates(col[..., ch], [ys, xs], order=1, mode="nearest").mean() for ch in range(3)]
        assert np.abs(out[j, i, :3] - want).max() < 1e-12, (j, i)
    pre_out = _prefilter(pre, R)
    rp = max(R / 8.0, math.sqrt(0.5))
    for (j, i) in [(28, 36), (3, 4)]:
        ys = np.array([j] + [j + rp * math.sin(k * math.pi / 4) for k in range(8)])
        xs = np.array([i] + [i + rp * math.cos(k * math.pi / 4) for k in range(8)])
        want = [map_coordinates(col[..., ch], [ys, xs], order=1, mode="nearest").mean() for ch in range(3)]
        assert np.abs(pre_out[j, i, :3] - want).max() < 1e-12, (j, i)


def test_prefilter_excludes_taps_of_a_different_coc():
    """The prefilter's CoC-similarity weight: neighbours whose CoC differs from the
    centre's by at least max(1, |rho_0|) take no part (the centre keeps its colour), and
    a difference of half that takes half a weight."""
    W2, H2, R = 32, 32, 16.0
    col = np.zeros((H2, W2, 4))
    col[..., :3] = B_COL
    col[..., 3] = 12.0
    j, i = 16, 16
    col[j, i, :3] = A_COL
    col[j, i, 3] = 4.0                      # |12 - 4| = 8 >= max(1, 4)
    out = _prefilter(col, R)
    assert np.abs(out[j, i, :3] - A_COL).max() < 1e-12
    # neighbours at rho 6 (difference 2 = half of max(1, 4)): every tap reads rho 6 and
    # B's colour (the taps at radius 2 hpx land on the neighbours), weight 1/2 each
    col[..., 3] = 6.0
    col[j, i, 3] = 4.0
    out = _prefilter(col, R)
    want = (A_COL + 8 * 0.5 * B_COL) / (1 + 8 * 0.5)
    assert np.abs(out[j, i, :3] - want).max() < 1e-12


def test_prefilter_similarity_scale_has_a_floor_of_one_pixel():
    """The CoC difference is measured against max(1, |rho_0|): for a nearly sharp centre
    (rho_0 = 0.5) a neighbour 0.5 away keeps half a weight (1 - 0.5 / 1), not none."""
    W2, H2, R = 32, 32, 16.0
    col = np.zeros((H2, W2, 4))
    col[..., :3] = B_COL
    col[..., 3] = 1.0
    j, i = 16, 16
    col[j, i, :3] = A_COL
    col[j, i, 3] = 0.5
    out = _prefilter(col, R)
    want = (A_COL + 8 * 0.5 * B_COL) / (1 + 8 * 0.5)
    assert np.abs(out[j, i, :3] - want).max() < 1e-12


def test_albedo_hash_matches_murmur3_test_vectors():
    """The albedo hash is murmur3's 32-bit finaliser.  For an empty key,
    MurmurHash3_x86_32 is the finaliser of the seed, and its published test vectors
    fix three values: seed 0 -> 0, seed 1 -> 0x514E28B7, seed 0xFFFFFFFF -> 0x81F16F39.
    The per-triangle albedo of seed 0 and triangle 0 then reads the finaliser of 0, 1
    and 2 (channel c takes 3 prim + c), so channel 0 is the range's floor 0.1 and
    channel 1 is fixed by the seed-1 vector."""
    L = oracle.lib()
    assert L.or_fmix32(0) == 0
    assert L.or_fmix32(1) == 0x514E28B7
    assert L.or_fmix32(0xFFFFFFFF) == 0x81F16F39
    col = np.zeros(3)
    L.or_albedo(0, 0, col.ctypes.data_as(C.c_void_p))
    assert col[0] == 0.1
    assert col[1] == pytest.approx(0.1 + 0.8 * (0x514E28B7 >> 8) / 2.0 ** 24, abs=1e-15)
    assert col[2] == pytest.approx(0.1 + 0.8 * (L.or_fmix32(2) >> 8) / 2.0 ** 24, abs=1e-15)
    # every albedo lies in [0.1, 0.9) and the channels of many triangles fill it evenly
    cols = np.zeros((4096, 3))
    for k in range(4096):
        L.or_albedo(7, k, cols[k].ctypes.data_as(C.c_void_p))
    assert cols.min() >= 0.1 and cols.max() < 0.9
    assert abs(cols.mean() - 0.5) < 0.01
    assert abs(np.corrcoef(cols[:, 0], cols[:, 1])[0, 1]) < 0.05
