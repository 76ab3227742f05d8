"""The allocation-free tile-map entry point agrees with the tile stage of dof_frame.

dof_coc_tiles_noalloc serves callers that cannot allocate device memory at the point
where they need the tile map (an engine that reserved all device memory up front, or
a frame loop that must not trigger the implicit device synchronisation of
cudaMalloc/cudaFree).  It keeps its intermediate in a built-in device array shared
by all calls.  This file is collected last so that, if it fails, a run that stops at
the first failure has already run every other test."""

import numpy as np
import pytest

import oracle
from synth import make_workload

pytestmark = pytest.mark.gpu


def _tiles_via_frame(w, gb):
    """The dilated tile map the existing entry point (dof_frame) computes."""
    from parity import GpuRunner
    g = GpuRunner(w, w.params, record_rays=False)
    g.frame(w.camera(0), gb, read=False)
    T = int(w.params["tile"])
    H2, W2 = w.H // 2, w.W // 2
    return g.hist.read("TILES_DIL", shape=(-(-H2 // T), -(-W2 // T), 2))


def test_noalloc_tiles_match_dof_frame_two_calls():
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
        want = _tiles_via_frame(w, gb)
        depth = torch.from_numpy(np.ascontiguousarray(gb["depth"])).to(dev)
        got = dof.coc_tiles_noalloc(depth, cam, w.params)
        torch.cuda.synchronize()
        got = got.cpu().numpy()
        assert got.shape == want.shape
        assert np.abs(got - want).max() <= 2e-5          # the tile tolerance of the parity tests
        assert want[..., 1].max() > 0.5                  # a non-trivial tile map


def test_noalloc_rejects_oversize():
    import torch
    from paper_2210_06158_gb300 import _build, dof
    _build.build()
    w = make_workload("c1")
    dev = torch.device("cuda", 0)
    depth = torch.ones((4100, 4100), dtype=torch.float32, device=dev)   # 257 x 257 tiles > 65536
    with pytest.raises(dof.DofError) as e:
        dof.coc_tiles_noalloc(depth, w.camera(0), w.params)
    assert e.value.code == -1 and "scratch" in str(e.value)
