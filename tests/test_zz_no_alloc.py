"""The allocation-free tile-map entry point agrees with the tile stage of dof_frame and
with the FP64 oracle's tile dilation.

dof_coc_tiles_noalloc serves callers that cannot allocate device memory at the point
where they need the tile map (an engine that reserved all device memory up front, or
a frame loop that must not trigger the implicit device synchronisation of
cudaMalloc/cudaFree).  It keeps its intermediate in a built-in device array shared
by all calls.  This file is collected last so that, if it fails, a run that stops at
the first failure has already run every other test."""

import ctypes as C

import numpy as np
import pytest

import oracle
from synth import make_workload

pytestmark = pytest.mark.gpu

TILE_TOL = 2e-5      # the tile tolerance of the parity tests (FP32 CoC vs the FP64 oracle)


def _tiles_via_frame(w, gb):
    """The dilated tile map the existing entry point (dof_frame) computes."""
    from parity import GpuRunner
    g = GpuRunner(w, w.params, record_rays=False)
    g.frame(w.camera(0), gb, read=False)
    T = int(w.params["tile"])
    H2, W2 = w.H // 2, w.W // 2
    return g.hist.read("TILES_DIL", shape=(-(-H2 // T), -(-W2 // T), 2))


def test_noalloc_tiles_match_dof_frame_and_oracle_two_calls():
    import torch
    from paper_2210_06158_gb300 import _build, dof
    _build.build()
    oracle.build()
    dev = torch.device("cuda", 0)
    # two calls in a row on the shared scratch: a larger frame, then a smaller one
    cases = [make_workload("c2", W=322, H=182), make_workload("c1", W=160, H=90)]
    for w in cases:
        osc = oracle.Scene(w.scene)
        cam = w.camera(0)
        gb = oracle.gbuffer_f32(oracle.gbuffer(osc, cam, w.params, w.W, w.H))
        want_frame = _tiles_via_frame(w, gb)
        want_oracle = oracle.frame(osc, cam, w.params, w.W, w.H, gb)["tile_dil"]
        depth = torch.from_numpy(np.ascontiguousarray(gb["depth"])).to(dev)
        got = dof.coc_tiles_noalloc(depth, cam, w.params)
        torch.cuda.synchronize()
        got = got.cpu().numpy()
        assert got.shape == want_frame.shape == want_oracle.shape
        assert np.abs(got - want_frame).max() <= TILE_TOL
        assert np.abs(got.astype(np.float64) - want_oracle).max() <= TILE_TOL
        assert want_oracle[..., 1].max() > 0.5           # a non-trivial tile map


def test_noalloc_allocates_nothing():
    """Free device memory and torch's allocator are unchanged across calls (after the
    first call in this process, which may load the library's device code)."""
    import torch
    from paper_2210_06158_gb300 import _build, dof
    _build.build()
    w = make_workload("c2", W=640, H=360)
    dev = torch.device("cuda", 0)
    depth = torch.rand((w.H, w.W), dtype=torch.float32, device=dev) * 50.0 + 0.5
    out = torch.empty((-(-(w.H // 2) // 8), -(-(w.W // 2) // 8), 2), dtype=torch.float32, device=dev)
    dof.coc_tiles_noalloc(depth, w.camera(0), w.params, out=out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(dev)
    alloc0 = torch.cuda.memory_allocated(dev)
    for _ in range(3):
        dof.coc_tiles_noalloc(depth, w.camera(0), w.params, out=out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(dev)
    assert free1 == free0
    assert torch.cuda.memory_allocated(dev) == alloc0


def test_noalloc_rejects_oversize_and_bad_lens():
    import torch
    from paper_2210_06158_gb300 import _build, dof
    _build.build()
    w = make_workload("c1")
    dev = torch.device("cuda", 0)
    depth = torch.ones((4100, 4100), dtype=torch.float32, device=dev)   # 257 x 257 tiles > 65536
    with pytest.raises(dof.DofError) as e:
        dof.coc_tiles_noalloc(depth, w.camera(0), w.params)
    assert e.value.code == -1 and "scratch" in str(e.value)
    # host-side rejections (nothing is launched): sizes beyond 16384, non-finite lens
    small = torch.ones((16, 16), dtype=torch.float32, device=dev)
    out = torch.empty((1, 1, 2), dtype=torch.float32, device=dev)
    L = dof.lib()
    for W, H in ((1 << 31, 2), (2, 1 << 31), (16386, 2)):
        c, p = dof.camera_struct(w.camera(0)), dof.params_struct(w.params)
        rc = L.dof_coc_tiles_noalloc(C.c_void_p(small.data_ptr()), W, H, C.byref(c), C.byref(p),
                                     C.c_void_p(out.data_ptr()), None)
        assert rc == -1, (W, H, rc)
    for field, val in (("focus_m", float("inf")), ("f_m", float("nan")), ("f_number", float("inf"))):
        c, p = dof.camera_struct(w.camera(0)), dof.params_struct(w.params)
        setattr(c, field, val)
        rc = L.dof_coc_tiles_noalloc(C.c_void_p(small.data_ptr()), 16, 16, C.byref(c), C.byref(p),
                                     C.c_void_p(out.data_ptr()), None)
        assert rc == -1, (field, rc)
        assert b"finite" in L.dof_last_error()
