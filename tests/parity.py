"""Helpers of the GPU parity tests: run the CUDA path (through the C ABI) and the FP64
oracle on the same seeded inputs and compare them element by element.

Tolerance accounting
  * hit ids: bit-exact, except rays whose kernel answer the oracle's hit_check
    accepts as a floating-point near tie (the kernel's triangle is hit within
    1e-6 (|o| + s) of rounding, no clean hit lies certainly in front of it, and a
    clean kernel hit is not certainly in front of the oracle's); every mismatch must
    classify, and they are at most 1e-4 of the rays;
  * images: max |d| <= 2e-3 and PSNR >= 50 dB in linear RGB; the max excludes the
    taint cone of mismatched rays (the pixel, the reconstruction footprint, the
    median and the upsampling, carried through the history by the motion), whose
    share is reported;
  * intermediates: tighter bounds from the FP32 arithmetic (see each test).
"""

from __future__ import annotations

import math

import numpy as np
import scipy.ndimage as ndi

import oracle

SQRT2 = math.sqrt(2.0)


def psnr(a, b):
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return float("inf") if mse == 0 else 10.0 * math.log10(1.0 / mse)


def ssim(a, b, mask=None):
    """Mean structural similarity (Wang, Bovik, Sheikh and Simoncelli 2004) of two linear
    RGB images with peak 1: Gaussian window sigma 1.5 (truncated at 3.5 sigma, 11 taps),
    C1 = (0.01)^2, C2 = (0.03)^2, per channel, averaged over the channels and over the
    pixels of `mask` (all pixels if None)."""
    from scipy.ndimage import gaussian_filter
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    c1, c2 = 0.01 ** 2, 0.03 ** 2
    g = lambda x: gaussian_filter(x, 1.5, mode="reflect", truncate=3.5)
    vals = []
    for c in range(a.shape[-1]):
        x, y = a[..., c], b[..., c]
        mx, my = g(x), g(y)
        sxx, syy, sxy = g(x * x) - mx * mx, g(y * y) - my * my, g(x * y) - mx * my
        m = ((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2))
        vals.append(m if mask is None else m[mask])
    return float(np.mean(vals))


class GpuRunner:
    """One session on the CUDA path: scene + history, frames through dof_frame."""

    def __init__(self, workload, params=None, max_rays=None, record_rays=True, ctx=None):
        import torch
        from paper_2210_06158_gb300 import dof
        self.dof, self.torch = dof, torch
        self.w = workload
        self.params = dict(params or workload.params)
        mr = max_rays or oracle.max_rays(self.params)
        self.ctx = ctx or dof.Context(0)
        self.scene = dof.Scene(self.ctx, workload.scene)
        self.taa = float(self.params.get("taa_alpha", 0.0)) > 0.0
        self.hist = dof.History(self.ctx, workload.W, workload.H, max_rays=mr, record_rays=record_rays, taa=self.taa)
        self.max_rays = mr
        self.dev = torch.device("cuda", 0)

    def frame(self, cam, gb32, read=True):
        torch = self.torch
        g = {k: torch.from_numpy(np.ascontiguousarray(v)).to(self.dev) for k, v in gb32.items()}
        out = self.dof.frame(self.ctx, self.scene, g, cam, self.params, self.hist)
        torch.cuda.synchronize()
        res = dict(out=out.cpu().numpy())
        if read:
            res.update(self.read_all())
            if self.taa:
                res["composite"] = self.hist.read("COMPOSITE", shape=(self.w.H, self.w.W, 4))
        res["stats"] = self.hist.stats()
        return res

    def read_img(self, name, H2, W2):
        """A colour image buffer as float32 (H2, W2, 4): with FP16 storage
        (image_storage = 1) its first H2 * W2 half4 texels hold the image."""
        if int(self.params.get("image_storage", 0)) == 1:
            a = self.hist.read(name, np.float16)[:H2 * W2 * 4]
            return a.reshape(H2, W2, 4).astype(np.float32)
        return self.hist.read(name, shape=(H2, W2, 4))

    def read_pre(self, H2, W2):
        """The prefilter's output (rgb, rho) as float32 (H2, W2, 4): with FP16 storage
        each texel is a 16-byte record, (r, g) and (b, 0) as half2, then rho and z."""
        if int(self.params.get("image_storage", 0)) == 1:
            raw = self.hist.read("PRE", np.uint32).reshape(H2, W2, 4)
            rgb = raw[..., :2].copy().view(np.float16).reshape(H2, W2, 4)[..., :3].astype(np.float32)
            return np.concatenate([rgb, raw[..., 2:3].view(np.float32)], axis=-1)
        return self.hist.read("PRE", shape=(H2, W2, 4))

    def read_all(self):
        H2, W2 = self.w.H // 2, self.w.W // 2
        N = H2 * W2
        T = int(self.params["tile"])
        TH, TW = -(-H2 // T), -(-W2 // T)
        h = self.hist
        r = {}
        r["pp_in"] = h.read("PP_IN", shape=(H2, W2, 4))
        r["z_h"] = h.read("Z_H", shape=(H2, W2))
        r["tile_raw"] = h.read("TILES", shape=(TH, TW, 2))
        r["tile_dil"] = h.read("TILES_DIL", shape=(TH, TW, 2))
        r["pre"] = self.read_pre(H2, W2)
        r["main_out"] = self.read_img("MAIN", H2, W2)
        r["pp_med"] = self.read_img("PP_MED", H2, W2)
        r["xn"] = h.read("XN", shape=(H2, W2))
        r["xf"] = h.read("XF", shape=(H2, W2))
        r["nrays"] = h.read("NRAYS", np.int32, shape=(H2, W2))
        rp = h.read("RAY_PRIM", np.int32)
        r["ray_prim"] = rp.reshape(H2, W2, self.max_rays) if rp.size else None
        rt = h.read("RT", shape=(4, H2, W2, 4))
        o = np.zeros((H2, W2, 14), np.float32)
        o[..., 0] = rt[1, ..., 3]
        o[..., 1] = rt[0, ..., 3]
        o[..., 2:5] = rt[0, ..., :3]
        o[..., 5:8] = rt[1, ..., :3]
        o[..., 8] = rt[2, ..., 0]
        o[..., 9] = rt[2, ..., 1]
        o[..., 10:13] = rt[3, ..., :3]
        o[..., 13] = rt[2, ..., 2]
        r["rt"] = o
        r["crt"] = self.read_img("CRT", H2, W2)
        r["ct"] = h.read("CT", shape=(H2, W2))
        r["var"] = h.read("VAR", shape=(H2, W2))
        r["var_blur"] = h.read("VAR_BLUR", shape=(H2, W2))
        r["rt_med"] = self.read_img("RT_MED", H2, W2)
        r["recon"] = self.read_img("RECON", H2, W2)
        hh = h.read("HIST", shape=(3, H2, W2, 4))
        hist = np.zeros((H2, W2, 12), np.float32)
        hist[..., 0:3] = hh[0, ..., :3]
        hist[..., 3:6] = hh[1, ..., :3]
        hist[..., 6] = hh[0, ..., 3]
        hist[..., 7] = hh[1, ..., 3]
        hist[..., 8:12] = hh[2]
        # the device keeps (mean, variance) of the luminance; the oracle (mean, mean of squares)
        hist[..., 11] = hh[2, ..., 3] + hh[2, ..., 2].astype(np.float64) ** 2
        r["hist"] = hist
        return r


def oracle_inputs(w, frame_idx, osc=None):
    osc = osc or oracle.Scene(w.scene)
    cam = w.camera(frame_idx)
    gb = oracle.gbuffer(osc, cam, w.params, w.W, w.H)
    return osc, cam, oracle.gbuffer_f32(gb)


def classify_hits(osc, w, params, cam, gpu, ref):
    """Returns (n_rays, n_mismatch, n_invalid, mismatch mask per hpx).  A mismatch is
    valid when oracle.Scene.hit_check accepts the kernel's triangle for the ray (the
    oracle's FP64 ray of that pixel and sample)."""
    nr = ref["nrays"]
    H2, W2 = nr.shape
    mism = np.zeros((H2, W2), bool)
    n_rays = int(nr.sum())
    n_mis = n_bad = 0
    gp, op = gpu["ray_prim"], ref["ray_prim"]
    mr = min(gp.shape[2], op.shape[2])
    for s in range(mr):
        valid = nr > s
        diff = valid & (gp[..., s] != op[..., s])
        for (j, i) in np.argwhere(diff):
            n_mis += 1
            o, d = oracle.lens_ray(cam, params, w.W, w.H, i, j, s)
            code = osc.hit_check(o, d, int(gp[j, i, s]), int(op[j, i, s]))
            if code < 0:
                n_bad += 1
                print(f"invalid hit at hpx ({i},{j}) sample {s}: kernel {int(gp[j, i, s])} "
                      f"oracle {int(op[j, i, s])} code {code}")
            mism[j, i] = True
    return n_rays, n_mis, n_bad, mism


def mask_ties(ref, params):
    """hpx on a tile whose dilated near radius lies within 1e-5 of the mask threshold:
    whether the pixel gets rays is decided on a rounding tie there."""
    H2, W2 = ref["nrays"].shape
    T = int(params["tile"])
    thr = float(np.float32(params["mask_near_hpx"]))
    tie_t = np.abs(ref["tile_dil"][..., 0] - thr) <= 1e-5 * max(thr, 1e-3)
    return np.repeat(np.repeat(tie_t, T, 0), T, 1)[:H2, :W2]


def count_ties(ref, params, band=None):
    """hpx whose ray count may be decided on a rounding tie: x_f (Eq. 4) within `band`
    (default 1e-3 m) of an integer the count can jump at, or a mask tie.  Used only to
    widen the taint of comparisons that do not force the counts."""
    H2, W2 = ref["nrays"].shape
    out = np.zeros((H2, W2), bool)
    if int(params["ray_mode"]) == 1:
        # adaptive count clamp(ceil(x_f), 1, m) jumps only where x_f crosses 1..m-1
        xf = ref["xf"]
        k = np.round(xf)
        jump = (k >= 1) & (k <= float(params["m"]) - 1)
        b = 1e-3 * max(1.0, float(params["m"])) if band is None else band
        out |= jump & (np.abs(xf - k) <= b) & (ref["nrays"] > 0)
    return out | mask_ties(ref, params)


def weight_ties(ref):
    """hpx with a ray whose hit CoC lies within 1e-5 of the far-weight boundary
    c = -sqrt2."""
    H2, W2 = ref["nrays"].shape
    out = np.zeros((H2, W2), bool)
    if "ray_c" in ref:
        c = ref["ray_c"]
        k = np.arange(c.shape[2])[None, None, :] < ref["nrays"][..., None]
        near = k & (np.abs(c + SQRT2) <= 1e-5 * SQRT2)
        out |= near.any(-1)
    return out


def threshold_ties(ref, params, cam, w):
    return count_ties(ref, params) | weight_ties(ref)


def taint_radius(params):
    rmax = 0.5 * float(params["max_coc_px"])
    lod = min(float(params["lod_max"]), rmax * float(params["lod_scale"]))
    return int(math.ceil(rmax)) + 2 ** (int(math.ceil(lod)) + 1) + 2


def dilate(mask, r):
    """Binary dilation by a (2r+1)^2 square (separable running max, zero outside)."""
    if r <= 0 or not mask.any():
        return mask.copy()
    return ndi.maximum_filter(mask.astype(np.uint8), size=2 * r + 1, mode="constant", cval=0).astype(bool)


def full_res(mask_h, W, H):
    m = np.repeat(np.repeat(mask_h, 2, 0), 2, 1)[:H, :W]
    return dilate(m, 2)


def max_hdr(a, b):
    """Largest error of a against b, absolute where |b| <= 1 and relative above: the
    image bounds are stated for display-range linear RGB (peak 1); HDR values (emitters)
    carry FP32 rounding in proportion to their magnitude."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    d = np.abs(a - b) / np.maximum(1.0, np.abs(b))
    return float(d.max()) if d.size else 0.0


def max_abs(a, b, mask=None):
    d = np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64))
    if mask is not None:
        d = d[~mask] if d.ndim == mask.ndim else d[~mask]
    return float(d.max()) if d.size else 0.0
