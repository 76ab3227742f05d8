"""FP64 CPU oracle of the hybrid depth-of-field pass -- TEST INFRASTRUCTURE.

Plain C written from the paper (Tan et al., arXiv 2210.06158), loaded through
ctypes.  Only the tests, the smoke check and the CPU-baseline leg of the benchmark
may use it; the product path (the CUDA library and its binding) never imports it.

`build()` compiles ``oracle/*.c`` with gcc into ``oracle/_build/liboracle.so``
(OpenMP over image rows; results do not depend on the thread count because every
pixel is computed independently).
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_BUILD = _HERE / "_build"
_LIB_PATH = _BUILD / "liboracle.so"
_SOURCES = ["or_camera.c", "or_scene.c", "or_gbuffer.c", "or_post.c", "or_rays.c",
            "or_temporal.c", "or_recon.c", "or_taa.c", "or_frame.c"]
_lock = threading.Lock()
_lib = None


# Relative tolerance of the hit-id tie classification: a ray within 1e-6 (|o| + s)
# of a triangle's edge segment, or two hits whose distances agree to that tolerance,
# may be resolved either way by an FP32 tracer.
HIT_TIE_REL_TOL = 1e-6


def build(force: bool = False) -> Path:
    """Compile the oracle (gcc, -O2, no FP contraction so x86 and Arm agree)."""
    srcs = [_HERE / s for s in _SOURCES]
    deps = srcs + [_HERE / "oracle.h", _HERE / "or_internal.h"]
    if not force and _LIB_PATH.exists():
        t = _LIB_PATH.stat().st_mtime
        if all(d.stat().st_mtime <= t for d in deps):
            return _LIB_PATH
    _BUILD.mkdir(exist_ok=True)
    tmp = _LIB_PATH.with_suffix(f".so.tmp{os.getpid()}")
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-fopenmp", "-Wall", "-Wno-unused-function", "-o", str(tmp)] + [str(s) for s in srcs] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(str(_LIB_PATH))
            _declare(L)
            _lib = L
    return _lib


# ----------------------------------------------------------------------------
# structures (mirror oracle.h)
# ----------------------------------------------------------------------------

_d3 = C.c_double * 3


class OrCamera(C.Structure):
    _fields_ = [("f", C.c_double), ("N", C.c_double), ("d", C.c_double), ("ws", C.c_double),
                ("O", _d3), ("R", _d3), ("U", _d3), ("F", _d3),
                ("pO", _d3), ("pR", _d3), ("pU", _d3), ("pF", _d3),
                ("frame", C.c_int64), ("jx", C.c_double), ("jy", C.c_double),
                ("pjx", C.c_double), ("pjy", C.c_double)]


class OrParams(C.Structure):
    _fields_ = [("s", C.c_double), ("var_w_mask", C.c_double), ("m", C.c_double),
                ("spp", C.c_int32), ("ray_mode", C.c_int32),
                ("depth_range", C.c_double), ("alpha", C.c_double), ("alpha_motion", C.c_double),
                ("var_w_recon", C.c_double), ("b_max", C.c_double), ("h_edge", C.c_double),
                ("lod_scale", C.c_double), ("lod_max", C.c_double), ("max_coc_px", C.c_double),
                ("zof_ramp", C.c_double), ("cover_ramp", C.c_double),
                ("bright_lum", C.c_double), ("bright_ramp", C.c_double),
                ("mask_near_hpx", C.c_double), ("z_far", C.c_double),
                ("tile", C.c_int32), ("pad0", C.c_int32),
                ("seed", C.c_uint64), ("session", C.c_uint64),
                ("light", _d3), ("k_a", C.c_double), ("k_d", C.c_double), ("sky", _d3),
                ("emit", C.c_double), ("albedo_seed", C.c_uint32), ("pad1", C.c_int32),
                ("taa_alpha", C.c_double), ("blades", C.c_double)]


_pd = C.POINTER(C.c_double)
_pi = C.POINTER(C.c_int32)


class OrFrame(C.Structure):
    _fields_ = [(n, _pd) for n in ("pp_in", "z_h", "n_h", "tile_raw", "tile_dil", "pre",
                                   "main_out", "pp_med", "xn", "xf")] + \
               [("nrays", _pi), ("ray_prim", _pi), ("ray_c", _pd)] + \
               [(n, _pd) for n in ("rt", "crt", "ct", "var", "rt_med", "recon", "out",
                                   "hist_in", "hist_out", "var_in", "var_out")] + \
               [("has_history", C.c_int32), ("max_rays", C.c_int32), ("nrays_force", _pi),
                ("ray_hit_force", _pi), ("taa_in", _pd), ("taa_out", _pd), ("has_taa_history", C.c_int32),
                ("pad_taa", C.c_int32)]


def _declare(L):
    vp = C.c_void_p
    L.or_scene_create.restype = vp
    L.or_scene_create.argtypes = [vp, C.c_int, vp, vp, C.c_int]
    L.or_scene_destroy.argtypes = [vp]
    L.or_scene_depth.argtypes = [vp]
    for fn in (L.or_closest, L.or_closest_brute):
        fn.restype = C.c_int
        fn.argtypes = [vp, vp, vp, vp]
    L.or_set_threads.restype = C.c_int
    L.or_set_threads.argtypes = [C.c_int]
    L.or_hit_check.restype = C.c_int
    L.or_hit_check.argtypes = [vp, vp, vp, C.c_int, C.c_int, C.c_double]
    L.or_coc.restype = C.c_double
    L.or_coc.argtypes = [C.POINTER(OrCamera), C.c_int, C.c_double]
    L.or_zof_bounds.argtypes = [C.POINTER(OrCamera), C.c_int, vp, vp]
    L.or_pixel_dir.argtypes = [C.POINTER(OrCamera), C.c_int, C.c_int, C.c_double, C.c_double, vp]
    L.or_philox4x64.argtypes = [vp, vp, vp]
    L.or_lens_ray.argtypes = [C.POINTER(OrCamera), C.POINTER(OrParams), C.c_int, C.c_int,
                              C.c_int, C.c_int, C.c_int, vp, vp]
    L.or_gbuffer.argtypes = [vp, C.POINTER(OrCamera), C.POINTER(OrParams), C.c_int, C.c_int,
                             vp, vp, vp, vp]
    L.or_frame.restype = C.c_int
    L.or_frame.argtypes = [vp, C.POINTER(OrCamera), C.POINTER(OrParams), C.c_int, C.c_int,
                           vp, vp, vp, C.POINTER(OrFrame)]
    L.or_median9.argtypes = [vp, C.c_int, vp]
    L.or_poly_rho.restype = C.c_double
    L.or_poly_rho.argtypes = [C.c_int, C.c_double]
    L.or_poly_area.restype = C.c_double
    L.or_poly_area.argtypes = [C.c_int]
    L.or_aperture_point.argtypes = [C.c_int, C.c_double, C.c_double, vp]
    L.or_ring_tap.argtypes = [C.c_int, C.c_int, vp]
    L.or_binomial5.argtypes = [vp, C.c_int, C.c_int, C.c_int, vp]
    L.or_sobel5.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, vp, vp]
    L.or_albedo.argtypes = [C.c_uint32, C.c_int, vp]
    L.or_fmix32.restype = C.c_uint32
    L.or_fmix32.argtypes = [C.c_uint32]
    L.or_shade.argtypes = [vp, C.POINTER(OrParams), C.c_int, vp, vp, C.c_double, vp, vp]
    # individual stages
    L.or_downscale.argtypes = [C.POINTER(OrCamera), C.POINTER(OrParams), C.c_int, C.c_int,
                               vp, vp, vp, vp, vp, vp]
    L.or_main_filter.argtypes = [C.POINTER(OrParams), C.c_int, C.c_int, vp, vp, vp, vp]
    L.or_prefilter.argtypes = [C.POINTER(OrParams), C.c_int, C.c_int, vp, vp, vp]
    L.or_accumulate.argtypes = [C.POINTER(OrCamera), C.POINTER(OrParams), C.c_int, C.c_int,
                                vp, vp, vp, vp, C.c_int, vp, vp, vp, vp]
    L.or_recon.argtypes = [C.POINTER(OrParams), C.c_int, C.c_int, vp, vp, vp, vp, vp]
    L.or_median_rt.argtypes = [C.c_int, C.c_int, vp, vp, vp]
    L.or_mask.argtypes = [C.POINTER(OrParams), C.c_int, C.c_int, vp, vp, vp, vp, vp, vp, vp]
    L.or_composite.argtypes = [C.POINTER(OrCamera), C.POINTER(OrParams), C.c_int, C.c_int,
                               vp, vp, vp, vp, vp, vp]
    L.or_taa.argtypes = [C.POINTER(OrCamera), C.POINTER(OrParams), C.c_int, C.c_int, vp, vp, vp, C.c_int, vp]


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# ----------------------------------------------------------------------------
# conversions from the shared input generators
# ----------------------------------------------------------------------------

def camera(cam) -> OrCamera:
    """synth.Camera (float32 pose) -> OrCamera (exact widening to double)."""
    c = OrCamera()
    c.f, c.N, c.d, c.ws = (float(np.float32(cam.f_m)), float(np.float32(cam.f_number)),
                           float(np.float32(cam.focus_m)), float(np.float32(cam.sensor_w_m)))
    for name, src in (("O", cam.pos), ("R", cam.right), ("U", cam.up), ("F", cam.fwd),
                      ("pO", cam.prev_pos), ("pR", cam.prev_right), ("pU", cam.prev_up),
                      ("pF", cam.prev_fwd)):
        setattr(c, name, _d3(*[float(np.float32(x)) for x in src]))
    c.frame = int(cam.frame_index)
    jx, jy = getattr(cam, "jitter", (0.0, 0.0))
    pjx, pjy = getattr(cam, "prev_jitter", (0.0, 0.0))
    c.jx, c.jy, c.pjx, c.pjy = (float(np.float32(v)) for v in (jx, jy, pjx, pjy))
    return c


def params(p: dict) -> OrParams:
    """parameter dict -> OrParams.  Real-valued parameters are rounded to float32 first,
    because the CUDA library receives them as float32."""
    f = lambda x: float(np.float32(x))
    o = OrParams()
    o.s, o.var_w_mask, o.m = f(p["s"]), f(p["var_w_mask"]), f(p["m"])
    o.spp, o.ray_mode = int(p["spp"]), int(p["ray_mode"])
    for k in ("depth_range", "alpha", "alpha_motion", "var_w_recon", "b_max", "h_edge",
              "lod_scale", "lod_max", "max_coc_px", "zof_ramp", "cover_ramp", "bright_lum",
              "bright_ramp", "mask_near_hpx", "z_far"):
        src = {"depth_range": "depth_range_m", "zof_ramp": "zof_ramp_px",
               "cover_ramp": "cover_ramp_px", "z_far": "z_far_m"}.get(k, k)
        setattr(o, k, f(p[src]))
    o.tile = int(p["tile"])
    o.seed, o.session = int(p["seed"]), int(p["session"])
    o.light = _d3(*[f(x) for x in p["light_dir"]])
    o.k_a, o.k_d = f(p["k_a"]), f(p["k_d"])
    o.sky = _d3(*[f(x) for x in p["sky"]])
    o.emit = f(p["emit"])
    o.albedo_seed = int(p["albedo_seed"]) & 0xFFFFFFFF
    o.taa_alpha = f(p.get("taa_alpha", 0.0))
    o.blades = float(int(p.get("aperture_blades", 0)))
    return o


class Scene:
    def __init__(self, scene):
        L = lib()
        self._v = np.ascontiguousarray(scene.verts, dtype=np.float32)
        self._t = np.ascontiguousarray(scene.tris, dtype=np.uint32)
        self._m = np.ascontiguousarray(scene.mat, dtype=np.uint32)
        self.n_tris = int(self._t.shape[0])
        self.ptr = L.or_scene_create(_p(self._v), int(self._v.shape[0]), _p(self._t), _p(self._m),
                                     self.n_tris)

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.or_scene_destroy(self.ptr)
            self.ptr = None

    @property
    def depth(self) -> int:
        return lib().or_scene_depth(self.ptr)

    def closest(self, o, d, brute=False):
        o = np.ascontiguousarray(o, dtype=np.float64)
        d = np.ascontiguousarray(d, dtype=np.float64)
        t = np.zeros(1)
        fn = lib().or_closest_brute if brute else lib().or_closest
        prim = fn(self.ptr, _p(o), _p(d), _p(t))
        return prim, (float(t[0]) if prim >= 0 else float("inf"))

    def hit_check(self, o, d, prim_kernel, prim_oracle, rel_tol=HIT_TIE_REL_TOL) -> int:
        """Validity of a closest hit computed in lower precision (prim_kernel, -1 = no
        hit) for the ray (o, d), against the FP64 answer prim_oracle: 0 = equal ids;
        1 = depth tie (both clean hits at distances rounding cannot order); 2 = the
        FP64 hit is grazed (within rel_tol (|o| + s) of an edge segment); 3 = the
        kernel's triangle is grazed; 4 = no hit reported and every hit is grazed;
        negative = invalid (-1 the kernel's triangle is not hit within rounding, -2 a
        clean hit lies certainly in front of it, -3 its clean hit lies certainly in
        front of the FP64 answer)."""
        o = np.ascontiguousarray(o, dtype=np.float64)
        d = np.ascontiguousarray(d, dtype=np.float64)
        return int(lib().or_hit_check(self.ptr, _p(o), _p(d), int(prim_kernel), int(prim_oracle), rel_tol))

    def near_tie(self, o, d, prim_kernel, prim_oracle, rel_tol=HIT_TIE_REL_TOL) -> bool:
        """True when prim_kernel is a valid answer (equal, or a rounding tie)."""
        return self.hit_check(o, d, prim_kernel, prim_oracle, rel_tol) >= 0


def set_threads(n: int) -> int:
    """Threads of the oracle's OpenMP row loops (results do not depend on it); returns
    the previous count.  n <= 0 only queries."""
    return int(lib().or_set_threads(int(n)))


def coc(cam, W, z) -> float:
    c = camera(cam)
    return lib().or_coc(C.byref(c), int(W), float(z))


def zof_bounds(cam, W):
    c = camera(cam)
    a, b = np.zeros(1), np.zeros(1)
    lib().or_zof_bounds(C.byref(c), int(W), _p(a), _p(b))
    return float(a[0]), float(b[0])


def philox4x64(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().or_philox4x64(_p(c), _p(k), _p(out))
    return out


def lens_ray(cam, prm, W, H, i, j, sample):
    c, p = camera(cam), params(prm)
    o, d = np.zeros(3), np.zeros(3)
    lib().or_lens_ray(C.byref(c), C.byref(p), int(W), int(H), int(i), int(j), int(sample), _p(o), _p(d))
    return o, d


def poly_rho(n: int, th: float) -> float:
    """Boundary radius of the regular n-gon aperture (circumradius 1, a vertex at angle
    0) in direction th; 1 for the circle (n = 0)."""
    return lib().or_poly_rho(int(n), float(th))


def poly_area(n: int) -> float:
    return lib().or_poly_area(int(n))


def aperture_point(n: int, u1: float, u2: float) -> np.ndarray:
    """Lens point of the unit-circumradius aperture from two uniforms."""
    out = np.zeros(2)
    lib().or_aperture_point(int(n), float(u1), float(u2), _p(out))
    return out


def ring_tap(n: int, t: int) -> np.ndarray:
    """Tap t of the 81-tap kernel on the aperture's shape: (x, y, ring fraction)."""
    out = np.zeros(3)
    lib().or_ring_tap(int(n), int(t), _p(out))
    return out


def pixel_dir(cam, W, H, x, y):
    c = camera(cam)
    d = np.zeros(3)
    lib().or_pixel_dir(C.byref(c), int(W), int(H), float(x), float(y), _p(d))
    return d


def gbuffer(scene: Scene, cam, prm, W, H) -> dict:
    """Pinhole G-buffer: colour (H,W,3), depth (H,W) (+inf on a miss), normal
    (H,W,3), prim (H,W) int32 (-1 on a miss); all float64 except prim."""
    c, p = camera(cam), params(prm)
    col = np.zeros((H, W, 3))
    dep = np.zeros((H, W))
    nrm = np.zeros((H, W, 3))
    prim = np.zeros((H, W), dtype=np.int32)
    lib().or_gbuffer(scene.ptr, C.byref(c), C.byref(p), int(W), int(H), _p(col), _p(dep), _p(nrm), _p(prim))
    return dict(color=col, depth=dep, normal=nrm, prim=prim)


def gbuffer_f32(gb: dict) -> dict:
    """Round an oracle G-buffer to the float32 RGBA / depth / normal-xyz0 layout that
    the frame takes as input."""
    H, W = gb["depth"].shape
    col = np.zeros((H, W, 4), dtype=np.float32)
    col[..., :3] = gb["color"]
    col[..., 3] = 1.0
    nrm = np.zeros((H, W, 4), dtype=np.float32)
    nrm[..., :3] = gb["normal"]
    return dict(color=col, depth=gb["depth"].astype(np.float32), normal=nrm)


class History:
    """Oracle-side session history: 12 doubles per half-resolution pixel plus the
    blurred variance, and whether a previous frame exists."""

    def __init__(self, W, H):
        n = (W // 2) * (H // 2)
        self.hist = np.zeros(12 * n)
        self.var = np.zeros(n)
        self.valid = False
        self.taa = np.zeros(W * H * 4)      # previous resolved (TAA) image
        self.taa_valid = False

    def copy(self) -> "History":
        h = History.__new__(History)
        h.hist, h.var, h.valid = self.hist.copy(), self.var.copy(), self.valid
        h.taa, h.taa_valid = self.taa.copy(), self.taa_valid
        return h


def taa(cam, prm, W, H, depth, cur, hist=None):
    """Final TAA of one image (Section 3.4): depth (H, W) float32, cur and hist (H, W, 4)
    float64; hist None = no previous frame."""
    d = np.ascontiguousarray(depth, dtype=np.float32)
    c0 = np.ascontiguousarray(cur, dtype=np.float64)
    h0 = np.ascontiguousarray(hist if hist is not None else np.zeros_like(c0), dtype=np.float64)
    out = np.zeros((H, W, 4))
    c, p = camera(cam), params(prm)
    lib().or_taa(C.byref(c), C.byref(p), int(W), int(H), _p(d), _p(c0), _p(h0), 1 if hist is not None else 0,
                 _p(out))
    return out


def max_rays(prm) -> int:
    return int(prm["spp"]) if int(prm["ray_mode"]) == 0 else int(prm["m"])


def frame(scene: Scene, cam, prm, W, H, gb32: dict, hist: History | None = None,
          keep_rays: bool = True, nrays_force=None, hit_force=None) -> dict:
    """Run one frame; returns every intermediate (numpy, float64) and updates `hist`.
    nrays_force (tests): int32 (H/2, W/2), a ray count to take instead of the mask's
    where >= 0 (the count decision's ties, where either count is valid).
    hit_force (tests): int32 (H/2, W/2, max_rays), a triangle id (-1 = miss) to take as
    the ray's hit where >= -1 (near ties, where either hit is valid)."""
    W2, H2 = W // 2, H // 2
    N = W2 * H2
    T = int(prm["tile"])
    TW, TH = -(-W2 // T), -(-H2 // T)
    mr = max(1, max_rays(prm))
    hist = hist if hist is not None else History(W, H)
    z = lambda *s: np.zeros(s)
    out = dict(pp_in=z(H2, W2, 4), z_h=z(H2, W2), n_h=z(H2, W2, 3), tile_raw=z(TH, TW, 2),
               tile_dil=z(TH, TW, 2), pre=z(H2, W2, 4), main_out=z(H2, W2, 4), pp_med=z(H2, W2, 4),
               xn=z(H2, W2), xf=z(H2, W2), nrays=np.zeros((H2, W2), dtype=np.int32),
               rt=z(H2, W2, 14), crt=z(H2, W2, 4), ct=z(H2, W2), var=z(H2, W2),
               rt_med=z(H2, W2, 4), recon=z(H2, W2, 4), out=z(H, W, 4),
               hist_out=z(12 * N), var_out=z(N))
    taa = float(prm.get("taa_alpha", 0.0)) > 0.0
    if taa:
        out["out_taa"] = z(H, W, 4)
    if keep_rays:
        out["ray_prim"] = np.full((H2, W2, mr), -2, dtype=np.int32)
        out["ray_c"] = z(H2, W2, mr)
    fr = OrFrame()
    for k in ("pp_in", "z_h", "n_h", "tile_raw", "tile_dil", "pre", "main_out", "pp_med", "xn",
              "xf", "rt", "crt", "ct", "var", "rt_med", "recon", "out", "hist_out", "var_out"):
        setattr(fr, k, out[k].ctypes.data_as(_pd))
    fr.nrays = out["nrays"].ctypes.data_as(_pi)
    fr.ray_prim = out["ray_prim"].ctypes.data_as(_pi) if keep_rays else None
    fr.ray_c = out["ray_c"].ctypes.data_as(_pd) if keep_rays else None
    fr.hist_in = hist.hist.ctypes.data_as(_pd)
    fr.var_in = hist.var.ctypes.data_as(_pd)
    fr.has_history = 1 if hist.valid else 0
    fr.max_rays = mr
    if taa:
        if hist.taa.size != W * H * 4:
            hist.taa = np.zeros(W * H * 4)
            hist.taa_valid = False
        taa_in = np.ascontiguousarray(hist.taa)
        fr.taa_in = taa_in.ctypes.data_as(_pd)
        fr.taa_out = out["out_taa"].ctypes.data_as(_pd)
        fr.has_taa_history = 1 if hist.taa_valid else 0
    if nrays_force is not None:
        force = np.ascontiguousarray(nrays_force, dtype=np.int32).reshape(-1)
        assert force.size == N
        fr.nrays_force = force.ctypes.data_as(_pi)
    if hit_force is not None:
        hforce = np.full((H2, W2, mr), -2, dtype=np.int32)
        k = min(mr, hit_force.shape[2])
        hforce[..., :k] = hit_force[..., :k]
        hforce = np.ascontiguousarray(hforce).reshape(-1)
        fr.ray_hit_force = hforce.ctypes.data_as(_pi)
    col = np.ascontiguousarray(gb32["color"], dtype=np.float32)
    dep = np.ascontiguousarray(gb32["depth"], dtype=np.float32)
    nrm = np.ascontiguousarray(gb32["normal"], dtype=np.float32)
    c, p = camera(cam), params(prm)
    rc = lib().or_frame(scene.ptr, C.byref(c), C.byref(p), int(W), int(H), _p(col), _p(dep), _p(nrm),
                        C.byref(fr))
    if rc != 0:
        raise ValueError(f"or_frame rejected the frame (W={W}, H={H})")
    hist.hist = out["hist_out"].copy()
    hist.var = out["var_out"].copy()
    hist.valid = True
    if taa:
        hist.taa = out["out_taa"].reshape(-1).copy()
        hist.taa_valid = True
    out["hist"] = out["hist_out"].reshape(H2, W2, 12)
    out["var_blur"] = out["var_out"].reshape(H2, W2)
    return out
