"""Thin Python binding of libdof (include/dof.h): ctypes marshalling only.

Every step of the pass runs in the CUDA library; torch is used for device memory
(tensors whose data pointers are handed to the library) and for the current CUDA
stream.  There is no CPU fallback: if the library cannot be loaded, every call
raises.
"""

from __future__ import annotations

import ctypes as C
import threading
from pathlib import Path

import numpy as np

_PKG = Path(__file__).resolve().parent
_LIB_PATH = _PKG / "_lib" / "libdof.so"
_lib = None
_lock = threading.Lock()

DOF_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "OOM", -3: "BUDGET", -4: "CUDA", -5: "TIMEOUT",
          -6: "DEVICE_CHECK", -7: "MISMATCH"}
DOF_HIST_RECORD_RAYS = 1
DOF_HIST_TIMING = 2
DOF_HIST_TAA = 4
# timing slots (dof_kernel_times), named after the kernels they bracket; k_trace_rays
# times whichever tracer runs, and the fused slots (dilate, variance blur, mips) read 0
KERNELS = ["k_downscale_tiles", "k_tile_dilate", "k_prefilter", "k_main_filter", "k_median_pp", "k_edges",
           "k_mask_compact", "k_trace_rays", "k_shade", "k_accumulate", "k_var_blur", "k_median_rt", "k_mips", "k_recon",
           "k_composite", "k_taa"]
BUF = dict(PP_IN=0, Z_H=1, TILES=2, TILES_DIL=3, PRE=4, MAIN=5, PP_MED=6, XN=7, XF=8,
           NRAYS=9, RAY_PRIM=10, RT=11, CRT=12, CT=13, VAR=14, VAR_BLUR=15, RT_MED=16,
           RECON=17, HIST=18, COMPOSITE=19)


class DofError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libdof error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


_f3 = C.c_float * 3


class DofCamera(C.Structure):
    _fields_ = [("f_m", C.c_float), ("f_number", C.c_float), ("focus_m", C.c_float),
                ("sensor_w_m", C.c_float), ("pos", _f3), ("right", _f3), ("up", _f3), ("fwd", _f3),
                ("prev_pos", _f3), ("prev_right", _f3), ("prev_up", _f3), ("prev_fwd", _f3),
                ("frame_index", C.c_uint32), ("jitter", C.c_float * 2), ("prev_jitter", C.c_float * 2)]


class DofParams(C.Structure):
    _fields_ = [("s", C.c_float), ("var_w_mask", C.c_float), ("m", C.c_uint32), ("spp", C.c_uint32),
                ("ray_mode", C.c_uint32), ("depth_range_m", C.c_float), ("alpha", C.c_float),
                ("alpha_motion", C.c_float), ("var_w_recon", C.c_float), ("b_max", C.c_float),
                ("h_edge", C.c_float), ("lod_scale", C.c_float), ("lod_max", C.c_float),
                ("max_coc_px", C.c_float), ("zof_ramp_px", C.c_float), ("cover_ramp_px", C.c_float),
                ("bright_lum", C.c_float), ("bright_ramp", C.c_float), ("mask_near_hpx", C.c_float),
                ("z_far_m", C.c_float), ("tile", C.c_uint32), ("albedo_seed", C.c_uint32),
                ("seed", C.c_uint64), ("session", C.c_uint64), ("light_dir", _f3), ("k_a", C.c_float),
                ("k_d", C.c_float), ("sky", _f3), ("emit", C.c_float), ("image_storage", C.c_uint32),
                ("taa_alpha", C.c_float), ("aperture_blades", C.c_uint32)]


class DofGBuffer(C.Structure):
    _fields_ = [("color", C.c_void_p), ("depth", C.c_void_p), ("normal", C.c_void_p),
                ("width", C.c_uint32), ("height", C.c_uint32), ("fmt", C.c_uint32)]


class DofFrameReq(C.Structure):
    _fields_ = [("scene", C.c_void_p), ("gbuf", C.POINTER(DofGBuffer)), ("cam", C.POINTER(DofCamera)),
                ("params", C.POINTER(DofParams)), ("hist", C.c_void_p), ("out", C.c_void_p)]


MAX_BATCH = 32


class DofSceneInfo(C.Structure):
    _fields_ = [("n_tris", C.c_uint32), ("n_nodes", C.c_uint32), ("depth", C.c_uint32),
                ("stack_limit", C.c_uint32), ("device_bytes", C.c_uint64),
                ("bounds_lo", _f3), ("bounds_hi", _f3), ("n_large", C.c_uint32), ("n_nodes4", C.c_uint32), ("depth4", C.c_uint32),
                ("pad", C.c_uint32)]


class DofFrameStats(C.Structure):
    _fields_ = [("frames", C.c_uint64), ("masked_pixels", C.c_uint32), ("rays", C.c_uint32),
                ("device_status", C.c_int32), ("pad", C.c_uint32), ("node_visits", C.c_uint64),
                ("tri_tests", C.c_uint64)]


# every symbol the header declares, with its signature
_SIGS = {
    "dof_ctx_create": (C.c_int, [C.c_int, C.c_size_t, C.POINTER(C.c_void_p)]),
    "dof_ctx_destroy": (None, [C.c_void_p]),
    "dof_ctx_bytes_in_use": (C.c_size_t, [C.c_void_p]),
    "dof_ctx_set_option": (C.c_int, [C.c_void_p, C.c_int, C.c_int64]),
    "dof_params_default": (None, [C.POINTER(DofParams)]),
    "dof_last_error": (C.c_char_p, []),
    "dof_scene_upload": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p, C.c_void_p, C.c_uint32,
                                   C.c_void_p, C.POINTER(C.c_void_p)]),
    "dof_scene_destroy": (None, [C.c_void_p]),
    "dof_scene_info": (C.c_int, [C.c_void_p, C.POINTER(DofSceneInfo)]),
    "dof_gbuffer": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(DofCamera), C.POINTER(DofParams), C.c_uint32,
                              C.c_uint32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "dof_gbuffer_raster": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(DofCamera), C.POINTER(DofParams),
                                     C.c_uint32, C.c_uint32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p]),
    "dof_frame_host": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.POINTER(DofCamera), C.POINTER(DofParams), C.c_void_p, C.c_void_p, C.c_void_p]),
    "dof_frame_host_join": (C.c_int, [C.c_void_p, C.c_void_p]),
    "dof_launch_count": (C.c_ulonglong, []),
    "dof_history_create": (C.c_int, [C.c_void_p, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32,
                                     C.POINTER(C.c_void_p)]),
    "dof_history_destroy": (None, [C.c_void_p]),
    "dof_history_reset": (C.c_int, [C.c_void_p]),
    "dof_history_export": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_size_t), C.c_void_p]),
    "dof_history_import": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "dof_frame": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(DofGBuffer), C.POINTER(DofCamera),
                            C.POINTER(DofParams), C.c_void_p, C.c_void_p, C.c_void_p]),
    "dof_frame_stats": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(DofFrameStats)]),
    "dof_batch_frame": (C.c_int, [C.c_void_p, C.POINTER(DofFrameReq), C.c_uint32, C.c_void_p]),
    "dof_graph_create": (C.c_int, [C.c_void_p, C.POINTER(DofFrameReq), C.c_uint32, C.POINTER(C.c_void_p)]),
    "dof_graph_launch": (C.c_int, [C.c_void_p, C.POINTER(DofFrameReq), C.c_uint32, C.c_void_p]),
    "dof_graph_destroy": (None, [C.c_void_p]),
    "dof_debug_buffer": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_void_p), C.POINTER(C.c_size_t)]),
    "dof_kernel_times": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_uint32)]),
    "dof_debug_read": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_size_t]),
    "dof_coc_tiles_noalloc": (C.c_int, [C.c_void_p, C.c_uint32, C.c_uint32, C.POINTER(DofCamera),
                                        C.POINTER(DofParams), C.c_void_p, C.c_void_p]),
}


def library_path() -> Path:
    return _LIB_PATH


def lib():
    """Load libdof.so (built in-tree by `_build.build()`); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not _LIB_PATH.exists():
                raise RuntimeError(f"libdof.so not built ({_LIB_PATH}); run __graft_entry__.build()")
            L = C.CDLL(str(_LIB_PATH))
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(rc):
    if rc != DOF_OK:
        raise DofError(rc, lib().dof_last_error().decode())


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


# ---------------------------------------------------------------------------
# structures from the shared input generators
# ---------------------------------------------------------------------------

def camera_struct(cam) -> DofCamera:
    c = DofCamera()
    c.f_m, c.f_number, c.focus_m, c.sensor_w_m = cam.f_m, cam.f_number, cam.focus_m, cam.sensor_w_m
    for name in ("pos", "right", "up", "fwd", "prev_pos", "prev_right", "prev_up", "prev_fwd"):
        setattr(c, name, _f3(*[float(x) for x in np.asarray(getattr(cam, name), dtype=np.float32)]))
    c.frame_index = int(cam.frame_index)
    jx, jy = getattr(cam, "jitter", (0.0, 0.0))
    pjx, pjy = getattr(cam, "prev_jitter", (0.0, 0.0))
    c.jitter[0], c.jitter[1] = float(jx), float(jy)
    c.prev_jitter[0], c.prev_jitter[1] = float(pjx), float(pjy)
    return c


def params_struct(p: dict) -> DofParams:
    o = DofParams()
    lib().dof_params_default(C.byref(o))
    for k in ("s", "var_w_mask", "depth_range_m", "alpha", "alpha_motion", "var_w_recon", "b_max", "h_edge",
              "lod_scale", "lod_max", "max_coc_px", "zof_ramp_px", "cover_ramp_px", "bright_lum",
              "bright_ramp", "mask_near_hpx", "z_far_m", "k_a", "k_d", "emit", "taa_alpha"):
        if k in p:
            setattr(o, k, float(p[k]))
    for k in ("m", "spp", "ray_mode", "tile", "seed", "session", "image_storage", "aperture_blades"):
        if k in p:
            setattr(o, k, int(p[k]))
    if "albedo_seed" in p:
        o.albedo_seed = int(p["albedo_seed"]) & 0xFFFFFFFF
    if "light_dir" in p:
        o.light_dir = _f3(*[float(x) for x in p["light_dir"]])
    if "sky" in p:
        o.sky = _f3(*[float(x) for x in p["sky"]])
    return o


# ---------------------------------------------------------------------------
# objects
# ---------------------------------------------------------------------------

class Context:
    def __init__(self, device: int = 0, mem_budget_bytes: int = 0):
        self.ptr = C.c_void_p()
        _check(lib().dof_ctx_create(int(device), int(mem_budget_bytes), C.byref(self.ptr)))
        self.device = device

    def close(self):
        if self.ptr:
            lib().dof_ctx_destroy(self.ptr)
            self.ptr = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_bvh_builder(self, name: str):
        """'ploc' (default) or 'lbvh' for scenes uploaded afterwards."""
        _check(lib().dof_ctx_set_option(self.ptr, 1, {"ploc": 0, "lbvh": 1}[name]))

    def set_ploc_radius(self, r: int):
        """PLOC search radius for scenes uploaded afterwards (tree quality vs build time)."""
        _check(lib().dof_ctx_set_option(self.ptr, 5, int(r)))

    def set_bvh_rotations(self, passes: int):
        """Passes of tree rotations after the BVH build of scenes uploaded afterwards."""
        _check(lib().dof_ctx_set_option(self.ptr, 13, int(passes)))

    def set_bvh_width(self, width: int):
        """Tree the rays traverse: 4 (collapsed 4-wide nodes, default) or 2 (binary)."""
        _check(lib().dof_ctx_set_option(self.ptr, 6, int(width)))

    def set_trace(self, blocks_per_sm=None, refill_idle=None, steps=None, bvh_width=None, ray_grid=None, stack=None,
                  packets=None, stats=None):
        """Launch shape / scheduling of the persistent tracer, the tree it traverses, the
        order it takes the rays in (lens-cell grid; 1 = pixel order), its traversal
        stack depth (raised to what the tree needs), whether a warp's rays traverse
        the binary tree as one packet, and whether that packet tracer counts node
        visits and triangle tests for stats() -- no effect on results."""
        for opt, v in ((2, blocks_per_sm), (3, refill_idle), (4, steps), (6, bvh_width), (7, ray_grid), (11, stack),
                       (12, None if packets is None else int(bool(packets))),
                       (14, None if stats is None else int(bool(stats)))):
            if v is not None:
                _check(lib().dof_ctx_set_option(self.ptr, opt, int(v)))

    def set_gather(self, block=None, main_form=None, recon_block=None):
        """Launch shapes of the 81-tap gathers -- block (main filter) and recon_block
        (reconstruction) = (width, height) in half-resolution pixels (width >= 8, whole
        warps, 64..512 threads) -- and the main filter's form: 0 = halo tile in shared
        memory when it fits in 64 KB, 1 = through L1, 2 = halo tile up to the SM's opt-in
        shared memory, 3 = through L1 by columns of four pixels (no effect on results)."""
        for opt, b in ((8, block), (10, recon_block)):
            if b is not None:
                w, h = (int(v) for v in b)
                _check(lib().dof_ctx_set_option(self.ptr, opt, w | (h << 16)))
        if main_form is not None:
            _check(lib().dof_ctx_set_option(self.ptr, 9, int(main_form)))

    @property
    def bytes_in_use(self) -> int:
        return int(lib().dof_ctx_bytes_in_use(self.ptr))


class Scene:
    """Device scene + LBVH.  `scene` is a synth.Scene (host arrays, copied)."""

    def __init__(self, ctx: Context, scene, stream=None):
        self.ctx = ctx
        v = np.ascontiguousarray(scene.verts, dtype=np.float32)
        t = np.ascontiguousarray(scene.tris, dtype=np.uint32)
        m = np.ascontiguousarray(scene.mat, dtype=np.uint32)
        self.ptr = C.c_void_p()
        _check(lib().dof_scene_upload(ctx.ptr, v.ctypes.data_as(C.c_void_p), v.shape[0],
                                      t.ctypes.data_as(C.c_void_p), m.ctypes.data_as(C.c_void_p),
                                      t.shape[0], _stream_ptr(stream), C.byref(self.ptr)))

    def info(self) -> DofSceneInfo:
        i = DofSceneInfo()
        _check(lib().dof_scene_info(self.ptr, C.byref(i)))
        return i

    def close(self):
        if self.ptr:
            lib().dof_scene_destroy(self.ptr)
            self.ptr = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class History:
    def __init__(self, ctx: Context, width: int, height: int, max_rays: int = 1, record_rays: bool = False,
                 timing: bool = False, taa: bool = False):
        self.ctx = ctx
        self.width, self.height, self.max_rays = width, height, max_rays
        self.ptr = C.c_void_p()
        flags = (DOF_HIST_RECORD_RAYS if record_rays else 0) | (DOF_HIST_TIMING if timing else 0) | \
            (DOF_HIST_TAA if taa else 0)
        _check(lib().dof_history_create(ctx.ptr, width, height, max_rays, flags, C.byref(self.ptr)))

    def reset(self):
        _check(lib().dof_history_reset(self.ptr))

    def export(self, stream=None) -> bytes:
        """Checkpoint of the session (host bytes)."""
        n = C.c_size_t()
        _check(lib().dof_history_export(self.ptr, None, C.byref(n), _stream_ptr(stream)))
        buf = (C.c_char * n.value)()
        _check(lib().dof_history_export(self.ptr, buf, C.byref(n), _stream_ptr(stream)))
        return bytes(buf[:n.value])

    def load(self, data: bytes, stream=None):
        """Resume from a checkpoint made by export()."""
        buf = C.create_string_buffer(data, len(data))
        _check(lib().dof_history_import(self.ptr, buf, len(data), _stream_ptr(stream)))

    def stats(self, stream=None) -> DofFrameStats:
        s = DofFrameStats()
        _check(lib().dof_frame_stats(self.ptr, _stream_ptr(stream), C.byref(s)))
        return s

    def kernel_times(self, stream=None):
        """(dict kernel -> summed ms, frames) since the previous call (DOF_HIST_TIMING)."""
        ms = (C.c_float * len(KERNELS))()
        n = C.c_uint32()
        _check(lib().dof_kernel_times(self.ptr, _stream_ptr(stream), ms, C.byref(n)))
        return {k: float(ms[i]) for i, k in enumerate(KERNELS)}, int(n.value)

    def buffer(self, name: str):
        """(device pointer, bytes) of an intermediate buffer of the last frame."""
        p, n = C.c_void_p(), C.c_size_t()
        _check(lib().dof_debug_buffer(self.ptr, BUF[name], C.byref(p), C.byref(n)))
        return p.value, n.value

    def read(self, name: str, dtype=np.float32, shape=None):
        """Copy an intermediate buffer to a numpy array (synchronous)."""
        p, n = self.buffer(name)
        out = np.empty(n, dtype=np.uint8)
        _check(lib().dof_debug_read(self.ptr, BUF[name], out.ctypes.data_as(C.c_void_p), n))
        a = out.view(dtype)
        return a.reshape(shape) if shape is not None else a

    def close(self):
        if self.ptr:
            lib().dof_history_destroy(self.ptr)
            self.ptr = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gbuffer(ctx: Context, scene: Scene, cam, params: dict, width: int, height: int, out=None, stream=None,
            raster: bool = False):
    """G-buffer producer on the device; returns dict of torch tensors (color, depth,
    normal, prim).  raster=True produces the same bits object-order
    (dof_gbuffer_raster) instead of by one primary ray per pixel (dof_gbuffer)."""
    import torch
    dev = torch.device("cuda", ctx.device)
    if out is None:
        out = dict(color=torch.empty((height, width, 4), dtype=torch.float32, device=dev),
                   depth=torch.empty((height, width), dtype=torch.float32, device=dev),
                   normal=torch.empty((height, width, 4), dtype=torch.float32, device=dev),
                   prim=torch.empty((height, width), dtype=torch.int32, device=dev))
    c, p = camera_struct(cam), params_struct(params)
    fn = lib().dof_gbuffer_raster if raster else lib().dof_gbuffer
    _check(fn(ctx.ptr, scene.ptr, C.byref(c), C.byref(p), width, height, _ptr(out["color"]), _ptr(out["depth"]),
              _ptr(out["normal"]), _ptr(out.get("prim")), _stream_ptr(stream)))
    return out


def gbuffer_struct(color, depth, normal=None) -> DofGBuffer:
    g = DofGBuffer()
    g.color = color.data_ptr()
    g.depth = depth.data_ptr()
    g.normal = normal.data_ptr() if normal is not None else None
    g.height, g.width = int(depth.shape[0]), int(depth.shape[1])
    # half colour / normal planes: DOF_FMT_F16 (both planes in one format)
    half = str(color.dtype) == "torch.float16"
    if normal is not None and (str(normal.dtype) == "torch.float16") != half:
        raise ValueError("gbuffer: colour and normal planes must share one precision")
    g.fmt = 1 if half else 0
    return g


def frame(ctx: Context, scene: Scene, gbuf: dict, cam, params, hist: History, out=None, stream=None,
          cam_struct: DofCamera | None = None, params_s: DofParams | None = None):
    """Run one frame of the pass.  gbuf: dict of device tensors (color HxWx4, depth HxW,
    normal HxWx4); returns the output tensor (HxWx4 float32)."""
    import torch
    H, W = gbuf["depth"].shape
    if out is None:
        out = torch.empty((H, W, 4), dtype=torch.float32, device=gbuf["depth"].device)
    g = gbuffer_struct(gbuf["color"], gbuf["depth"], gbuf.get("normal"))
    c = cam_struct if cam_struct is not None else camera_struct(cam)
    p = params_s if params_s is not None else params_struct(params)
    _check(lib().dof_frame(ctx.ptr, scene.ptr, C.byref(g), C.byref(c), C.byref(p), hist.ptr, _ptr(out),
                           _stream_ptr(stream)))
    return out


def frame_host(ctx: Context, scene: Scene, gbuf: dict, cam, params, hist: History, out, stream=None,
               cam_struct: DofCamera | None = None, params_s: DofParams | None = None):
    """One frame from and to host memory (dof_frame_host): gbuf holds host tensors
    (color HxWx4, depth HxW, normal HxWx4 or absent), out a host HxWx4 float32 tensor;
    pinned tensors let the copies overlap the neighbouring frames' passes.  Returns
    before the copies end: call frame_host_join (then synchronise) before reading out."""
    c = cam_struct if cam_struct is not None else camera_struct(cam)
    p = params_s if params_s is not None else params_struct(params)
    for k in ("color", "depth", "normal"):
        t = gbuf.get(k)
        if t is not None and (t.is_cuda or not t.is_contiguous()):
            raise ValueError(f"frame_host: {k} must be a contiguous host tensor")
    if out.is_cuda or not out.is_contiguous():
        raise ValueError("frame_host: out must be a contiguous host tensor")
    _check(lib().dof_frame_host(ctx.ptr, scene.ptr, _ptr(gbuf["color"]), _ptr(gbuf["depth"]),
                                _ptr(gbuf.get("normal")), C.byref(c), C.byref(p), hist.ptr, _ptr(out),
                                _stream_ptr(stream)))
    return out


def launch_count() -> int:
    """Kernel launches the library has enqueued in this process (dof_launch_count)."""
    return int(lib().dof_launch_count())


def frame_host_join(hist: History, stream=None):
    """Make `stream` wait for the copy-outs of the host frames enqueued so far."""
    _check(lib().dof_frame_host_join(hist.ptr, _stream_ptr(stream)))


def coc_tiles_noalloc(depth, cam, params, out=None, stream=None):
    """Dilated tile map (near CoC radius, |rho|) per 8x8 half-resolution tile from a
    full-resolution depth tensor, through the allocation-free entry point (the library
    allocates nothing; `out` is created here by torch if not given)."""
    import torch
    H, W = depth.shape
    TW, TH = -(-(W // 2) // 8), -(-(H // 2) // 8)
    if out is None:
        out = torch.empty((TH, TW, 2), dtype=torch.float32, device=depth.device)
    c, p = camera_struct(cam), params_struct(params)
    _check(lib().dof_coc_tiles_noalloc(_ptr(depth), W, H, C.byref(c), C.byref(p), _ptr(out), _stream_ptr(stream)))
    return out


def _requests(items):
    import torch
    n = len(items)
    reqs = (DofFrameReq * max(1, n))()
    keep = []
    outs = []
    for k, it in enumerate(items):
        gb = it["gbuf"]
        H, W = gb["depth"].shape
        out = it.get("out")
        if out is None:
            out = torch.empty((H, W, 4), dtype=torch.float32, device=gb["depth"].device)
        g = gbuffer_struct(gb["color"], gb["depth"], gb.get("normal"))
        c = it["cam"] if isinstance(it["cam"], DofCamera) else camera_struct(it["cam"])
        p = it["params"] if isinstance(it["params"], DofParams) else params_struct(it["params"])
        keep += [g, c, p]
        reqs[k].scene = it["scene"].ptr
        reqs[k].gbuf = C.pointer(g)
        reqs[k].cam = C.pointer(c)
        reqs[k].params = C.pointer(p)
        reqs[k].hist = it["hist"].ptr
        reqs[k].out = out.data_ptr()
        outs.append(out)
    return reqs, keep, outs


def batch_frame(ctx: Context, items, stream=None):
    """Frames of several sessions in one launch per pass.  items: list of dicts with
    keys scene (Scene), gbuf (dict of device tensors), cam (synth.Camera or a
    DofCamera), params (dict or DofParams), hist (History), out (tensor, optional).
    Returns the output tensors."""
    reqs, keep, outs = _requests(items)
    _check(lib().dof_batch_frame(ctx.ptr, reqs, len(items), _stream_ptr(stream)))
    return outs


class Graph:
    """A captured step of batch_frame over fixed histories (CUDA graph).  Create it from
    the items of one step; launch(items) runs a step with new cameras, parameters,
    G-buffers or outputs (same sessions and launch shapes)."""

    def __init__(self, ctx: Context, items):
        self.ctx = ctx
        reqs, keep, _ = _requests(items)
        self.ptr = C.c_void_p()
        _check(lib().dof_graph_create(ctx.ptr, reqs, len(items), C.byref(self.ptr)))

    def launch(self, items, stream=None):
        reqs, keep, outs = _requests(items)
        _check(lib().dof_graph_launch(self.ptr, reqs, len(items), _stream_ptr(stream)))
        return outs

    def close(self):
        if self.ptr:
            lib().dof_graph_destroy(self.ptr)
            self.ptr = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
