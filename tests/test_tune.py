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

    def set_ploc_radius(self, r):
        self.radius = r

    def set_bvh_width(self, w):
        self.width = w


def _cost(cfg):
    # separable, minimum at width 2, 6 blocks per SM, refill 12, 32 steps
    return (1.0 + (0.3 if cfg["bvh_width"] == 4 else 0.0) + 0.05 * abs(cfg["blocks_per_sm"] - 6)
            + 0.02 * abs(cfg["refill_idle"] - 12) + 0.001 * abs(cfg["steps"] - 32))


def test_tune_trace_finds_the_optimum_of_a_separable_cost(monkeypatch):
    clock = _Clock()
    _fake_cuda(monkeypatch, clock)
    ctx = _Ctx()

    def run_frame(k):
        clock.t += _cost(ctx.cfg)

    best, seen = tune.tune_trace(ctx, run_frame, frames=3, stream=types.SimpleNamespace())
    assert best == {"bvh_width": 2, "blocks_per_sm": 6, "refill_idle": 12, "steps": 32}
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
