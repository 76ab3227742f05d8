"""Host logic of the autotuners (paper_2210_06158_gb300/tune.py) on the CPU: the device
timer is replaced by a clock that advances by a synthetic cost of the setting in force,
so the searches can be checked against the known optimum."""
import types

import pytest

from paper_2210_06158_gb300 import tune


class _Clock:
    def __init__(self):
        self.t = 0.0


def _fake_cuda(monkeypatch, clock):
    import torch

    class Event:
        def __init__(self, enable_timing=True):
            self.t = None

        def record(self, stream=None):
            self.t = clock.t

        def synchronize(self):
            pass

        def elapsed_time(self, end):
            return end.t - self.t

    monkeypatch.setattr(torch.cuda, "Event", Event)


class _Ctx:
    def __init__(self):
        self.cfg = dict(tune.DEFAULT)
        self.radius = 48
        self.width = 4

    def set_trace(self, **kw):
        self.cfg.update(kw)

    def set_gather(self, block=None, main_form=None, recon_block=None):
        if block is not None:
            self.cfg["gather_block"] = tuple(block)
        if main_form is not None:
            self.cfg["main_form"] = main_form
        if recon_block is not None:
            self.cfg["recon_block"] = tuple(recon_block)

    def set_ploc_radius(self, r):
        self.radius = r

    def set_bvh_width(self, w):
        self.width = w


def _cost(cfg):
    # separable, minimum at width 2, lens grid 8, stack 64, 6 blocks per SM, refill 12, 32 steps, packets
    return (1.0 + (0.3 if cfg["bvh_width"] == 4 else 0.0) + 0.04 * abs(cfg["ray_grid"] - 8)
            + (0.1 if cfg["packets"] == 0 else 0.0)
            + 0.001 * abs(cfg["stack"] - 64)
            + 0.05 * abs(cfg["blocks_per_sm"] - 6)
            + 0.02 * abs(cfg["refill_idle"] - 12) + 0.001 * abs(cfg["steps"] - 32))


def test_tune_trace_finds_the_optimum_of_a_separable_cost(monkeypatch):
    clock = _Clock()
    _fake_cuda(monkeypatch, clock)
    ctx = _Ctx()

    def run_frame(k):
        clock.t += _cost(ctx.cfg)

    best, seen = tune.tune_trace(ctx, run_frame, frames=3, stream=types.SimpleNamespace())
    assert best == {"bvh_width": 2, "ray_grid": 8, "stack": 64, "blocks_per_sm": 6, "refill_idle": 12, "steps": 32,
                    "packets": 1}
    assert ctx.cfg == best                         # the context keeps the winner
    for key, ms in seen.items():
        assert ms == pytest.approx(_cost(dict(key)))
    # every candidate lies in the search space
    for key in seen:
        for name, v in dict(key).items():
            assert v in tune.SPACE[name]


def test_tune_trace_keeps_the_default_within_one_percent(monkeypatch):
    """A candidate must beat the incumbent by more than 1% to replace it (timing noise)."""
    clock = _Clock()
    _fake_cuda(monkeypatch, clock)
    ctx = _Ctx()

    def run_frame(k):
        c = ctx.cfg
        clock.t += 1.0 - (0.005 if c["blocks_per_sm"] == 12 else 0.0)

    best, _ = tune.tune_trace(ctx, run_frame, frames=2, stream=types.SimpleNamespace())
    assert best == tune.DEFAULT


def test_tune_scene_keeps_the_fastest_tree_and_closes_the_others(monkeypatch):
    clock = _Clock()
    _fake_cuda(monkeypatch, clock)
    ctx = _Ctx()
    made, closed = [], []

    class FakeScene:
        def __init__(self, c, host):
            self.radius = c.radius
            made.append(self)

        def close(self):
            closed.append(self)

    from paper_2210_06158_gb300 import dof
    monkeypatch.setattr(dof, "Scene", FakeScene)

    def run_frame(sc, k):
        # fastest: radius 24 with the binary tree
        clock.t += 1.0 + 0.01 * abs(sc.radius - 24) + (0.2 if ctx.width == 4 else 0.0)

    scene, best, seen = tune.tune_scene(ctx, object(), run_frame, frames=2, stream=types.SimpleNamespace())
    assert best == {"ploc_radius": 24, "bvh_width": 2}
    assert scene.radius == 24 and scene not in closed
    assert len(made) == len(tune.SCENE_RADII) and len(closed) == len(made) - 1
    assert (ctx.radius, ctx.width) == (24, 2)
    assert set(seen) == {(r, w) for r in tune.SCENE_RADII for w in (4, 2)}


def test_tune_trace_times_every_candidate_on_the_same_frames(monkeypatch):
    """Frames of a moving camera differ in cost; each candidate must see the same ones."""
    clock = _Clock()
    _fake_cuda(monkeypatch, clock)
    ctx = _Ctx()
    calls = []

    def run_frame(k):
        calls.append(k)
        clock.t += 1.0 + 0.1 * k       # later frames cost more

    tune.tune_trace(ctx, run_frame, frames=3, stream=types.SimpleNamespace())
    assert calls[:3] == [0, 1, 2]                        # the session warmed up once
    timed = calls[3:]
    assert len(timed) % 4 == 0
    for m in range(len(timed) // 4):
        assert timed[4 * m:4 * m + 4] == [0, 0, 1, 2]   # warm-up, then frames 0 .. 2


def test_tune_trace_rejects_a_win_that_a_second_timing_does_not_confirm(monkeypatch):
    """A candidate that looks 5% faster once (noise) but not when timed again is not taken."""
    clock = _Clock()
    _fake_cuda(monkeypatch, clock)
    ctx = _Ctx()
    timed = {}

    def run_frame(k):
        key = tuple(sorted(ctx.cfg.items()))
        if k == 0 and key not in timed:
            timed[key] = 0
        if k == 0:
            timed[key] += 1
        lucky = ctx.cfg["blocks_per_sm"] == 12 and timed[key] <= 2   # fast only on its first timing
        clock.t += 0.95 if lucky else 1.0

    best, _ = tune.tune_trace(ctx, run_frame, frames=2, stream=types.SimpleNamespace())
    assert best == tune.DEFAULT


def test_tune_trace_searches_only_the_widths_given(monkeypatch):
    clock = _Clock()
    _fake_cuda(monkeypatch, clock)
    ctx = _Ctx()

    def run_frame(k):
        clock.t += _cost(dict(ctx.cfg, bvh_width=2 if ctx.cfg["bvh_width"] == 4 else 4))   # 4 would win

    best, seen = tune.tune_trace(ctx, run_frame, frames=2, stream=types.SimpleNamespace(), widths=(2,))
    assert best["bvh_width"] == 2
    assert all(dict(key)["bvh_width"] == 2 for key in seen)


def test_tune_gathers_finds_the_optimum_and_leaves_it_on_the_context(monkeypatch):
    clock = _Clock()
    _fake_cuda(monkeypatch, clock)
    ctx = _Ctx()
    ctx.cfg.update(tune.GATHER_DEFAULT)
    shape_cost = {(32, 8): 0.2, (16, 16): 0.1, (64, 4): 0.3, (32, 4): 0.25, (16, 8): 0.15, (32, 16): 0.0,
                  (64, 8): 0.05}
    form_cost = {0: 0.1, 1: 0.2, 2: 0.0, 3: 0.15}

    recon_cost = {(32, 8): 0.1, (16, 16): 0.0, (64, 4): 0.2, (32, 4): 0.12, (16, 8): 0.02, (32, 16): 0.05,
                  (64, 8): 0.3}

    def run_frame(k):
        clock.t += (1.0 + shape_cost[ctx.cfg["gather_block"]] + form_cost[ctx.cfg["main_form"]]
                    + recon_cost[ctx.cfg["recon_block"]])

    best, seen = tune.tune_gathers(ctx, run_frame, frames=2, stream=types.SimpleNamespace())
    assert best == {"gather_block": (32, 16), "main_form": 2, "recon_block": (16, 16)}
    assert ctx.cfg["gather_block"] == (32, 16) and ctx.cfg["main_form"] == 2 and ctx.cfg["recon_block"] == (16, 16)
    for key in seen:
        for name, v in dict(key).items():
            assert v in tune.GATHER_SPACE[name]


def test_tune_gathers_keeps_the_default_within_one_percent(monkeypatch):
    clock = _Clock()
    _fake_cuda(monkeypatch, clock)
    ctx = _Ctx()
    ctx.cfg.update(tune.GATHER_DEFAULT)

    def run_frame(k):
        clock.t += 1.0 - (0.004 if ctx.cfg["gather_block"] == (16, 16) else 0.0)

    best, _ = tune.tune_gathers(ctx, run_frame, frames=2, stream=types.SimpleNamespace())
    assert best == tune.GATHER_DEFAULT


def test_tune_trace_reports_packets_with_the_binary_tree(monkeypatch):
    """Warp packets always traverse the binary tree: a pick with packets names width 2."""
    clock = _Clock()
    _fake_cuda(monkeypatch, clock)
    ctx = _Ctx()

    def run_frame(k):
        c = ctx.cfg
        clock.t += 1.0 - (0.2 if c["packets"] else 0.0) - (0.1 if c["bvh_width"] == 4 and not c["packets"] else 0.0)

    best, seen = tune.tune_trace(ctx, run_frame, frames=2, stream=types.SimpleNamespace())
    assert best["packets"] == 1 and best["bvh_width"] == 2
    assert all(dict(k)["bvh_width"] == 2 for k in seen if dict(k)["packets"])


def test_tune_trace_is_not_fooled_by_a_warming_session(monkeypatch):
    """A fresh session's first frames can be cheaper (adaptive ray counts start from an
    empty history): the tuner warms the session up before it times the incumbent, so the
    optimum still wins."""
    clock = _Clock()
    _fake_cuda(monkeypatch, clock)
    ctx = _Ctx()
    calls = [0]

    def run_frame(k):
        calls[0] += 1
        clock.t += _cost(ctx.cfg) * (0.4 if calls[0] <= 4 else 1.0)

    best, _ = tune.tune_trace(ctx, run_frame, frames=3, stream=types.SimpleNamespace())
    assert best == {"bvh_width": 2, "ray_grid": 8, "stack": 64, "blocks_per_sm": 6, "refill_idle": 12, "steps": 32,
                    "packets": 1}


def test_tune_trace_starts_from_a_given_point(monkeypatch):
    """A second search starts from the first one's pick (and stays there when no move
    beats it)."""
    clock = _Clock()
    _fake_cuda(monkeypatch, clock)
    ctx = _Ctx()

    def run_frame(k):
        clock.t += _cost(ctx.cfg)

    first, _ = tune.tune_trace(ctx, run_frame, frames=2, stream=types.SimpleNamespace())
    again, seen = tune.tune_trace(ctx, run_frame, frames=2, rounds=1, stream=types.SimpleNamespace(), start=first)
    assert again == first
    assert tuple(sorted(first.items())) in seen


def test_bench_settings_pin_every_tuned_key():
    """bench.py --settings: the keys the tuners report, blocks as WxH, the rest at their
    defaults; an unknown key is refused."""
    import sys, os
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.parse_settings(None) is None
    s = bench.parse_settings("ploc_radius=96, bvh_width=2,ray_grid=1,packets=1,main_filter_block=64x4,"
                             "main_filter_form=3")
    assert s["ploc_radius"] == 96 and s["packets"] == 1 and s["ray_grid"] == 1
    assert s["main_filter_block"] == (64, 4) and s["main_filter_form"] == 3
    assert s["recon_block"] == (32, 8) and s["stack"] == tune.DEFAULT["stack"]
    assert set(tune.DEFAULT) <= set(s)
    with pytest.raises(SystemExit):
        bench.parse_settings("radius=3")
