"""Procedural scenes, camera poses and workload presets.

Units are metres.  The camera looks along +z with +y up; a pose is an orthonormal
basis (right, up, fwd) plus a position, all float32 so that the oracle and the CUDA
library read bit-identical values.

Placement only: objects are put inside an approximate view frustum (half-width
tangent sensor_w / (2 f)).  Nothing here evaluates the lens model of the method.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .rng import SplitMix64

# --------------------------------------------------------------------------
# geometry primitives (each returns verts (n,3) float64, tris (m,3) int64)
# --------------------------------------------------------------------------

_ICO_CACHE: dict[int, tuple[np.ndarray, np.ndarray]] = {}


def icosphere(level: int):
    """Unit icosphere: icosahedron (20 faces) subdivided `level` times (20*4^level faces)."""
    if level in _ICO_CACHE:
        return _ICO_CACHE[level]
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
         (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
         (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
         (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
         (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    verts = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    faces = list(f)
    for _ in range(level):
        mid = {}

        def midpoint(a, b):
            key = (min(a, b), max(a, b))
            if key not in mid:
                p = verts[a] + verts[b]
                verts.append(p / np.linalg.norm(p))
                mid[key] = len(verts) - 1
            return mid[key]

        nf = []
        for (a, b, c) in faces:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    out = (np.array(verts), np.array(faces, dtype=np.int64))
    _ICO_CACHE[level] = out
    return out


_BOX_V = np.array([[x, y, z] for x in (-0.5, 0.5) for y in (0.0, 1.0) for z in (-0.5, 0.5)])
# vertex index = 4*ix + 2*iy + iz
_BOX_F = np.array([
    (0, 1, 3), (0, 3, 2),        # x = -0.5
    (4, 6, 7), (4, 7, 5),        # x = +0.5
    (0, 4, 5), (0, 5, 1),        # y = 0
    (2, 3, 7), (2, 7, 6),        # y = 1
    (0, 2, 6), (0, 6, 4),        # z = -0.5
    (1, 5, 7), (1, 7, 3),        # z = +0.5
], dtype=np.int64)


def _rot_y(yaw):
    c, s = np.cos(yaw), np.sin(yaw)
    return c, s


def boxes(centers_xz, base_y, size, yaw):
    """Axis-aligned-in-y boxes standing on base_y. size: (n,3) (sx, sy, sz)."""
    n = len(centers_xz)
    v = _BOX_V[None, :, :] * size[:, None, :]                 # (n,8,3)
    c, s = _rot_y(yaw)
    x = v[..., 0] * c[:, None] + v[..., 2] * s[:, None]
    z = -v[..., 0] * s[:, None] + v[..., 2] * c[:, None]
    verts = np.stack([x + centers_xz[:, 0:1], v[..., 1] + base_y[:, None],
                      z + centers_xz[:, 1:2]], axis=-1).reshape(-1, 3)
    tris = (_BOX_F[None, :, :] + 8 * np.arange(n)[:, None, None]).reshape(-1, 3)
    return verts, tris


def spheres(centers, radii, level):
    uv, uf = icosphere(level)
    n = len(centers)
    verts = (uv[None] * radii[:, None, None] + centers[:, None, :]).reshape(-1, 3)
    tris = (uf[None] + len(uv) * np.arange(n)[:, None, None]).reshape(-1, 3)
    return verts, tris


def blades(base_xz, width, height, yaw):
    """Vertical grass-blade quads (2 triangles each) standing on y = 0."""
    n = len(base_xz)
    c, s = _rot_y(yaw)
    hw = 0.5 * width
    dx, dz = hw * c, -hw * s
    x0, z0 = base_xz[:, 0], base_xz[:, 1]
    p = np.stack([
        np.stack([x0 - dx, np.zeros(n), z0 - dz], -1),
        np.stack([x0 + dx, np.zeros(n), z0 + dz], -1),
        np.stack([x0 + dx, height, z0 + dz], -1),
        np.stack([x0 - dx, height, z0 - dz], -1),
    ], axis=1)                                               # (n,4,3)
    f = np.array([(0, 1, 2), (0, 2, 3)], dtype=np.int64)
    tris = (f[None] + 4 * np.arange(n)[:, None, None]).reshape(-1, 3)
    return p.reshape(-1, 3), tris


def ground(half=200.0):
    v = np.array([[-half, 0, -half], [half, 0, -half], [half, 0, half], [-half, 0, half]], dtype=np.float64)
    return v, np.array([(0, 2, 1), (0, 3, 2)], dtype=np.int64)


# --------------------------------------------------------------------------
# scene container
# --------------------------------------------------------------------------

@dataclass
class Scene:
    verts: np.ndarray          # (nv, 3) float32
    tris: np.ndarray           # (nt, 3) uint32
    mat: np.ndarray            # (nt,)   uint32: 0 diffuse (hash albedo), 1 emitter
    seed: int
    parts: dict = field(default_factory=dict)

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])

    @property
    def n_verts(self) -> int:
        return int(self.verts.shape[0])

    def tri_vertices(self) -> np.ndarray:
        """(nt, 3, 3) float32 triangle corner positions."""
        return self.verts[self.tris]


class _Builder:
    def __init__(self, seed):
        self.v, self.t, self.m, self.parts, self.nv = [], [], [], {}, 0
        self.seed = seed

    def add(self, name, verts, tris, mat=0):
        self.v.append(np.asarray(verts, dtype=np.float64))
        self.t.append(np.asarray(tris, dtype=np.int64) + self.nv)
        self.m.append(np.full(len(tris), mat, dtype=np.uint32))
        self.nv += len(verts)
        self.parts[name] = self.parts.get(name, 0) + len(tris)

    def build(self) -> Scene:
        if not self.v:
            return Scene(verts=np.zeros((0, 3), np.float32), tris=np.zeros((0, 3), np.uint32),
                         mat=np.zeros(0, np.uint32), seed=self.seed, parts={})
        return Scene(verts=np.concatenate(self.v).astype(np.float32),
                     tris=np.concatenate(self.t).astype(np.uint32),
                     mat=np.concatenate(self.m), seed=self.seed, parts=self.parts)


# --------------------------------------------------------------------------
# cameras
# --------------------------------------------------------------------------

def camera_pose(pos, pitch_deg=5.0, yaw_deg=0.0):
    """Orthonormal pose looking along +z, pitched down by pitch_deg, then yawed about +y."""
    p, y = math.radians(pitch_deg), math.radians(yaw_deg)
    right = np.array([math.cos(y), 0.0, -math.sin(y)])
    fwd0 = np.array([0.0, -math.sin(p), math.cos(p)])
    up0 = np.array([0.0, math.cos(p), math.sin(p)])
    # yaw about +y
    def ry(v):
        return np.array([v[0] * math.cos(y) + v[2] * math.sin(y), v[1],
                         -v[0] * math.sin(y) + v[2] * math.cos(y)])
    fwd, up = ry(fwd0), ry(up0)
    f32 = lambda a: np.asarray(a, dtype=np.float32)
    return dict(pos=f32(pos), right=f32(right), up=f32(up), fwd=f32(fwd))


@dataclass
class Camera:
    f_m: float
    f_number: float
    focus_m: float
    sensor_w_m: float
    pos: np.ndarray
    right: np.ndarray
    up: np.ndarray
    fwd: np.ndarray
    prev_pos: np.ndarray
    prev_right: np.ndarray
    prev_up: np.ndarray
    prev_fwd: np.ndarray
    frame_index: int = 0
    jitter: tuple = (0.0, 0.0)          # sub-pixel sampling offset of this frame (full-res px)
    prev_jitter: tuple = (0.0, 0.0)     # the previous frame's

    @staticmethod
    def from_poses(intr: dict, pose: dict, prev: dict | None = None, frame_index: int = 0):
        prev = prev or pose
        return Camera(f_m=intr["f_m"], f_number=intr["f_number"], focus_m=intr["focus_m"],
                      sensor_w_m=intr["sensor_w_m"],
                      pos=pose["pos"], right=pose["right"], up=pose["up"], fwd=pose["fwd"],
                      prev_pos=prev["pos"], prev_right=prev["right"], prev_up=prev["up"],
                      prev_fwd=prev["fwd"], frame_index=frame_index)


def halton(i: int, base: int) -> float:
    """Radical inverse of i in `base` (the Halton sequence)."""
    f, r = 1.0, 0.0
    while i > 0:
        f /= base
        r += f * (i % base)
        i //= base
    return r


def taa_jitter(k: int) -> tuple:
    """Camera jitter of frame k for temporal anti-aliasing: the 8-point Halton (2, 3)
    sequence, centred on the pixel (offsets in (-1/2, 1/2) full-resolution pixels)."""
    i = k % 8 + 1
    return (halton(i, 2) - 0.5, halton(i, 3) - 0.5)


def dolly_path(seed, start, n_frames, step_z=0.05, sway_sigma=0.01, pitch_deg=2.0):
    """Forward dolly with seeded lateral sway; returns n_frames poses."""
    rng = SplitMix64(seed ^ 0x5A5A5A5A)
    sway = rng.normal(n_frames) * sway_sigma
    sway[0] = 0.0
    poses = []
    for k in range(n_frames):
        p = np.array(start, dtype=np.float64) + np.array([sway[k], 0.0, step_z * k])
        poses.append(camera_pose(p, pitch_deg=pitch_deg))
    return poses


# --------------------------------------------------------------------------
# scenes
# --------------------------------------------------------------------------

def _frustum_x(rng, z, tanhx, spread=1.15):
    return rng.uniform(len(z), -1.0, 1.0) * z * tanhx * spread


def scene_c1(seed: int, cam_pos=(0.0, 1.2, 0.0), pitch_deg=5.0, f_m=0.05, sensor_w_m=0.036,
             aspect=144.0 / 256.0) -> Scene:
    """~2.8k triangles: ground, 8 level-2 icospheres (r 0.2-0.5 m) at 1-3 m inside the
    view, 20 boxes (0.5-2 m) standing on the ground at 10-30 m."""
    rng = SplitMix64(seed)
    b = _Builder(seed)
    b.add("ground", *ground())
    tanhx = sensor_w_m / (2 * f_m)
    tanhy = tanhx * aspect
    pose = camera_pose(cam_pos, pitch_deg)
    n = 8
    z = rng.uniform(n, 1.0, 3.0)
    sx = rng.uniform(n, -0.9, 0.9)
    sy = rng.uniform(n, -1.0, -0.1)
    r = rng.uniform(n, 0.2, 0.5)
    dirs = (pose["fwd"][None].astype(np.float64) + sx[:, None] * tanhx * pose["right"][None]
            + sy[:, None] * tanhy * pose["up"][None])
    centers = np.asarray(cam_pos)[None] + z[:, None] * dirs
    b.add("spheres", *spheres(centers, r, 2))
    nb = 20
    zb = rng.uniform(nb, 10.0, 30.0)
    xb = _frustum_x(rng, zb, tanhx, 0.9)
    size = np.stack([rng.uniform(nb, 0.5, 2.0), rng.uniform(nb, 0.5, 2.0),
                     rng.uniform(nb, 0.5, 2.0)], -1)
    b.add("boxes", *boxes(np.stack([xb, zb], -1), np.zeros(nb), size, rng.uniform(nb, 0, np.pi)))
    return b.build()


def scene_bokeh(seed: int, cam_pos=(0.0, 1.2, 0.0), pitch_deg=3.0, f_m=0.085, sensor_w_m=0.036,
                aspect=144.0 / 256.0) -> Scene:
    """Bright bokeh: emissive icospheres (material 1) out of focus in front of and far
    behind a focus distance of a few metres, diffuse boxes around it, on the ground."""
    rng = SplitMix64(seed)
    b = _Builder(seed)
    b.add("ground", *ground())
    tanhx = sensor_w_m / (2 * f_m)
    tanhy = tanhx * aspect
    pose = camera_pose(cam_pos, pitch_deg)

    def in_view(n, z0, z1, r0, r1):
        z = rng.uniform(n, z0, z1)
        sx = rng.uniform(n, -0.85, 0.85)
        sy = rng.uniform(n, -0.7, 0.7)
        r = rng.uniform(n, r0, r1)
        dirs = (pose["fwd"][None].astype(np.float64) + sx[:, None] * tanhx * pose["right"][None]
                + sy[:, None] * tanhy * pose["up"][None])
        return np.asarray(cam_pos)[None] + z[:, None] * dirs, r

    c, r = in_view(6, 0.8, 2.5, 0.02, 0.06)
    b.add("near_lights", *spheres(c, r, 1), mat=1)
    c, r = in_view(24, 25.0, 60.0, 0.1, 0.3)
    b.add("far_lights", *spheres(c, r, 1), mat=1)
    nb = 12
    zb = rng.uniform(nb, 4.0, 30.0)
    xb = _frustum_x(rng, zb, tanhx, 0.9)
    size = np.stack([rng.uniform(nb, 0.3, 1.5), rng.uniform(nb, 0.3, 1.5), rng.uniform(nb, 0.3, 1.5)], -1)
    b.add("boxes", *boxes(np.stack([xb, zb], -1), np.zeros(nb), size, rng.uniform(nb, 0, np.pi)))
    return b.build()


def scene_grass_field(seed: int, density: float = 1.0, f_m=0.035, sensor_w_m=0.036,
                      near=(1.3, 4.8), far=(8.0, 60.0)) -> Scene:
    """Lawn field: thin blade quads and fence bars in the near field (a 16-frame
    dolly advances 0.75 m, so from near[0] = 1.2 m its last frames see blades at
    0.45 m), a sparse box field and icospheres (level 4, level 5 from density 2) in the far field (8-60 m,
    sparse enough that sight lines reach the focus distance and beyond).
    density 1 gives ~500k triangles, density 4 ~2M: the blade count scales with it,
    the far field keeps its boxes per square metre and takes the rest of the
    triangle budget as spheres."""
    rng = SplitMix64(seed)
    b = _Builder(seed)
    b.add("ground", *ground())
    tanhx = sensor_w_m / (2 * f_m)
    nbl = int(180_000 * density)
    z = rng.uniform(nbl, *near)
    x = _frustum_x(rng, z, tanhx)
    b.add("blades", *blades(np.stack([x, z], -1), rng.uniform(nbl, 0.01, 0.03),
                            rng.uniform(nbl, 0.2, 0.6), rng.uniform(nbl, 0.0, np.pi)))
    nfb = int(150 * density)
    z = rng.uniform(nfb, *near)
    x = _frustum_x(rng, z, tanhx)
    size = np.stack([np.full(nfb, 0.03), rng.uniform(nfb, 0.4, 0.8), np.full(nfb, 0.03)], -1)
    b.add("fence", *boxes(np.stack([x, z], -1), np.zeros(nfb), size, rng.uniform(nfb, 0, np.pi)))
    # far field: object sizes follow the frustum width (relative to a 35 mm lens on
    # a 36 mm sensor), box count per ground area keeps the mean free path of a
    # ground-level sight line (~11 m, so the focus distance is seen)
    area = 1.15 * tanhx * (far[1] ** 2 - far[0] ** 2)
    sc = tanhx / (0.036 / (2 * 0.035))
    nbx = max(1, int(0.05 * area / sc))
    z = rng.uniform(nbx, *far)
    x = _frustum_x(rng, z, tanhx)
    size = sc * np.stack([rng.uniform(nbx, 0.5, 3.0), rng.uniform(nbx, 0.5, 3.0),
                          rng.uniform(nbx, 0.5, 3.0)], -1)
    b.add("boxes", *boxes(np.stack([x, z], -1), np.zeros(nbx), size, rng.uniform(nbx, 0, np.pi)))
    level = 4 if density < 2 else 5    # finer spheres rather than more of them
    per_sphere = 20 * 4 ** level
    nsp = max(1, int((500_000 * density - 2 * nbl - 12 * (nfb + nbx)) // per_sphere))
    z = rng.uniform(nsp, *far)
    x = _frustum_x(rng, z, tanhx)
    r = sc * rng.uniform(nsp, 0.3, 1.5)
    y = r + sc * rng.uniform(nsp, 0.0, 2.0)
    b.add("spheres", *spheres(np.stack([x, y, z], -1), r, level))
    return b.build()


def tiny_scene(seed: int, n_tris: int, ties: bool = True) -> Scene:
    """Random triangles in a 2 m box in front of the origin, plus (optionally) exact
    tie cases: a quad split into two triangles sharing an edge, and two coplanar
    overlapping triangles at the same depth."""
    rng = SplitMix64(seed)
    b = _Builder(seed)
    n = max(0, n_tris - (4 if ties else 0))
    if n:
        c = np.stack([rng.uniform(n, -1, 1), rng.uniform(n, -1, 1), rng.uniform(n, 2, 4)], -1)
        v = c[:, None, :] + rng.uniform(9 * n, -0.4, 0.4).reshape(n, 3, 3)
        b.add("random", v.reshape(-1, 3), np.arange(3 * n).reshape(n, 3))
    if ties:
        q = np.array([[-0.5, -0.5, 3.0], [0.5, -0.5, 3.0], [0.5, 0.5, 3.0], [-0.5, 0.5, 3.0]])
        b.add("shared_edge", q, np.array([(0, 1, 2), (0, 2, 3)]))
        t = np.array([[-0.3, -0.3, 2.5], [0.3, -0.3, 2.5], [0.0, 0.4, 2.5],
                      [-0.3, -0.3, 2.5], [0.3, -0.3, 2.5], [0.0, 0.4, 2.5]])
        b.add("coplanar", t, np.array([(0, 1, 2), (3, 4, 5)]))
    return b.build()


def plane_scene(planes, seed: int = 7) -> Scene:
    """Big single-triangle planes for closed-form tests.  Each entry of `planes` is
    (z, kind, x_edge, mat): a fronto-parallel triangle at depth z that covers the
    whole view (kind 'full'), or only the half-space x > x_edge ('right') or
    x < x_edge ('left'); a half-plane's edge lies exactly on the line x = x_edge."""
    b = _Builder(seed)
    for i, (z, kind, xe, mat) in enumerate(planes):
        if kind == "full":
            v = np.array([[-1000.0, -1000.0, z], [1000.0, -1000.0, z], [0.0, 1000.0, z]])
        elif kind == "right":
            v = np.array([[xe, -1000.0, z], [xe + 2000.0, 0.0, z], [xe, 1000.0, z]])
        elif kind == "left":
            v = np.array([[xe, -1000.0, z], [xe, 1000.0, z], [xe - 2000.0, 0.0, z]])
        else:
            raise ValueError(kind)
        b.add(f"plane{i}", v, np.array([(0, 1, 2)]), mat)
    return b.build()


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

def default_params(**over) -> dict:
    """Parameter block of the pass.  Constants the paper fixes: s = 0.8 (Section 4.2),
    variance weight 1e5 (Eq. 4), EMA blend 0.95 (Section 3.2.3), reconstruction weight
    2000 and clamp 0.9 (Eq. 5), smoothstep edge 0.3 (Eq. 7), LOD slope 0.05 and max 3
    (Eq. 8), depth range 10 cm (Section 4.2).  The others are readings of the text."""
    p = dict(s=0.8, var_w_mask=1e5, m=10, spp=1, ray_mode=0, depth_range_m=0.10,
             alpha=0.95, alpha_motion=0.8, var_w_recon=2000.0, b_max=0.9, h_edge=0.3,
             lod_scale=0.05, lod_max=3.0, max_coc_px=16.0, zof_ramp_px=0.25,
             cover_ramp_px=1.0, bright_lum=4.0, bright_ramp=1.0, mask_near_hpx=0.5,
             z_far_m=1.0e5, tile=8, seed=1, session=0, taa_alpha=0.0, aperture_blades=0,
             light_dir=(0.3, -1.0, 0.5), k_a=0.1, k_d=1.0, sky=(0.5, 0.6, 0.8),
             emit=8.0, albedo_seed=1)
    p.update(over)
    return p


@dataclass
class Workload:
    name: str
    W: int
    H: int
    intr: dict
    poses: list
    params: dict
    scene_fn: object
    _scene: Scene | None = None

    @property
    def scene(self) -> Scene:
        if self._scene is None:
            self._scene = self.scene_fn()
        return self._scene

    @property
    def n_frames(self) -> int:
        return len(self.poses)

    def camera(self, k: int) -> Camera:
        prev = self.poses[k - 1] if k > 0 else self.poses[k]
        cam = Camera.from_poses(self.intr, self.poses[k], prev, frame_index=k)
        if getattr(self, "jitter", False):
            cam.jitter = taa_jitter(k)
            cam.prev_jitter = taa_jitter(k - 1) if k > 0 else cam.jitter
        return cam


def make_workload(name: str, W: int | None = None, H: int | None = None,
                  n_frames: int | None = None, session: int = 0) -> Workload:
    """Workload presets.  Scene seed = 1000 + config number + 100 * session.

    c1  256x144, ~2.8k tris, 50 mm f/1.4 focus 15 m, 1 frame, 1 spp
    c2  1920x1080, ~500k tris, 35 mm f/2 focus 20 m, 16-frame dolly, 1 spp, CoC radius <= 32 px
    c3  3840x2160, ~2M tris, 85 mm f/1.2 focus 20 m, 16-frame dolly, 4 spp, CoC radius <= 64 px
    bokeh  256x144, emissive spheres near and far, 85 mm f/1.2 focus 5 m, 4 frames, 4 spp
    W/H override the resolution (for oracle-sized crops of the same scene and lens)."""
    if name == "c1":
        seed = 1001 + 100 * session
        intr = dict(f_m=0.05, f_number=1.4, focus_m=15.0, sensor_w_m=0.036)
        W, H = W or 256, H or 144
        poses = [camera_pose((0.0, 1.2, 0.0), 5.0)]
        params = default_params(spp=1, max_coc_px=16.0, seed=seed, session=session, albedo_seed=seed)
        fn = lambda: scene_c1(seed)
    elif name in ("c2", "c3"):
        cfg = 2 if name == "c2" else 3
        seed = 1000 + cfg + 100 * session
        if cfg == 2:
            intr = dict(f_m=0.035, f_number=2.0, focus_m=20.0, sensor_w_m=0.036)
            W, H = W or 1920, H or 1080
            params = default_params(spp=1, max_coc_px=32.0, seed=seed, session=session, albedo_seed=seed)
            dens = 1.0
        else:
            intr = dict(f_m=0.085, f_number=1.2, focus_m=20.0, sensor_w_m=0.036)
            W, H = W or 3840, H or 2160
            params = default_params(spp=4, max_coc_px=64.0, seed=seed, session=session, albedo_seed=seed)
            dens = 4.0
        # c2: a camera 0.7 m above the lawn sees the tall blades close to it, so during
        # the dolly the nearest blades come within 0.45 m and the CoC radius reaches its
        # 32 px clamp (c(0.5 m) = 31.9 px); c3's lens reaches its 64 px clamp from 1 m
        height, pitch = (0.7, 8.0) if cfg == 2 else (1.0, 4.0)
        near = (1.2, 4.7) if cfg == 2 else (1.3, 4.8)
        poses = dolly_path(seed, (0.0, height, 0.0), n_frames or 16, pitch_deg=pitch)
        f_m = intr["f_m"]
        fn = lambda: scene_grass_field(seed, dens, f_m=f_m, near=near)
    elif name == "bokeh":
        # bright bokeh (not a benchmark configuration): 85 mm f/1.2 focused at 5 m
        seed = 1004 + 100 * session
        intr = dict(f_m=0.085, f_number=1.2, focus_m=5.0, sensor_w_m=0.036)
        W, H = W or 256, H or 144
        poses = dolly_path(seed, (0.0, 1.2, 0.0), n_frames or 4, pitch_deg=3.0)
        params = default_params(spp=4, max_coc_px=16.0, seed=seed, session=session, albedo_seed=seed)
        fn = lambda: scene_bokeh(seed)
    else:
        raise ValueError(f"unknown workload {name!r}")
    if n_frames is not None:
        poses = poses[:n_frames]
    return Workload(name=name, W=W, H=H, intr=intr, poses=poses, params=params, scene_fn=fn)


WORKLOADS = ("c1", "c2", "c3")
