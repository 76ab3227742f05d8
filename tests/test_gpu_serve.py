"""Served frames (continuous batching over dof_batch_frame, two streams) equal the
frames of each session run alone."""

import numpy as np
import pytest

from synth import make_workload

pytestmark = pytest.mark.gpu


def test_served_results_equal_alone():
    import torch
    from paper_2210_06158_gb300 import _build, dof
    from paper_2210_06158_gb300.serve import GpuExecutor, Server, SessionSpec, poisson_arrivals
    _build.build()
    ex = GpuExecutor(budget_bytes=8 << 30, gbuf_ring=3)
    srv = Server(ex, max_batch=8)
    specs = {}
    for k, (name, W, H, fps) in enumerate([("c1", 256, 144, 60.0), ("c2", 320, 180, 30.0), ("c3", 192, 108, 60.0)]):
        w = make_workload(name, W=W, H=H, n_frames=3, session=k)
        poses = w.poses if len(w.poses) >= 3 else w.poses * 3
        specs[k] = SessionSpec(name, W, H, fps, scene=w.scene, params=dict(w.params), poses=poses, intr=w.intr)
        assert srv.admit(k, specs[k])
    st = srv.run(poisson_arrivals(5, specs, duration_s=0.5))
    assert st["frames"] > 10 and st["failed"] == 0
    torch.cuda.synchronize()
    # replay each session's served frame sequence alone
    for sid, frames in st["per_session"].items():
        s = ex.sessions[sid]
        h = dof.History(ex.ctx, specs[sid].width, specs[sid].height, max_rays=s["hist"].max_rays)
        out = None
        prev = None
        for f in frames:
            cam = ex.camera(s, f)
            out = dof.frame(ex.ctx, s["scene"], s["gbs"][f % ex.ring], None, None, h, cam_struct=cam,
                            params_s=s["pstruct"])
        torch.cuda.synchronize()
        assert torch.equal(out, s["out"]), sid
