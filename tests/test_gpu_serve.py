"""Served frames (continuous batching over dof_batch_frame, two streams) equal the
frames of each session run alone: every served frame, in the batched FP32 form (with
the tracer and the gathers tuned at start-up) and in the batched FP16-storage form."""

import pytest

from synth import make_workload

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fp16", [False, True])
def test_every_served_frame_equals_alone(fp16):
    import torch
    from paper_2210_06158_gb300 import _build, dof
    from paper_2210_06158_gb300.serve import GpuExecutor, Server, SessionSpec, poisson_arrivals
    _build.build()
    ex = GpuExecutor(budget_bytes=8 << 30, gbuf_ring=3, fp16=fp16, record=True)
    srv = Server(ex, max_batch=8)
    specs = {}
    sizes = [("c1", 256, 144, 60.0), ("c2", 320, 180, 30.0), ("c3", 192, 108, 60.0), ("c2", 160, 90, 60.0)]
    for k, (name, W, H, fps) in enumerate(sizes):
        w = make_workload(name, W=W, H=H, n_frames=3, session=k)
        poses = w.poses if len(w.poses) >= 3 else w.poses * 3
        specs[k] = SessionSpec(name, W, H, fps, scene=w.scene, params=dict(w.params), poses=poses, intr=w.intr)
        assert srv.admit(k, specs[k])
    if not fp16:
        pick = ex.tune(frames=1)                  # start-up tuning (histories start afresh)
        assert set(pick) >= {"bvh_width", "ray_grid", "packets"}
        assert set(ex.gathers) == {False, True}   # the gathers' picks per image storage
    st = srv.run(poisson_arrivals(5, specs, duration_s=0.5))
    assert st["frames"] > 10 and st["failed"] == 0
    assert st["mean_batch"] > 1.0                 # requests did share launches
    torch.cuda.synchronize()
    assert len(ex.records) == st["frames"]
    # replay each session's served frame sequence alone and compare every frame
    n_cmp = 0
    for sid, frames in st["per_session"].items():
        s = ex.sessions[sid]
        h = dof.History(ex.ctx, specs[sid].width, specs[sid].height, max_rays=s["hist"].max_rays)
        for f in frames:
            out = dof.frame(ex.ctx, s["scene"], s["gbs"][f % ex.ring], None, None, h, cam_struct=ex.camera(s, f),
                            params_s=s["pstruct"])
            torch.cuda.synchronize()
            assert torch.equal(out, ex.records[(sid, f)]), (sid, f)
            n_cmp += 1
        h.close()
    assert n_cmp == st["frames"]
