"""Serving loop: admission, continuous batching, per-session ordering, latency
statistics and failure handling, on a virtual-clock fake executor (host only)."""

import numpy as np
import pytest

from paper_2210_06158_gb300.serve import (FakeExecutor, Server, SessionSpec, percentile,
                                          poisson_arrivals)


def specs(n, W=1280, H=720, fps=60.0):
    return {k: SessionSpec(f"s{k}", W, H, fps) for k in range(n)}


def test_percentile_matches_numpy_nearest_rank():
    rng = np.random.default_rng(0)
    xs = list(rng.exponential(size=101))
    for q in (50, 90, 99):
        assert percentile(xs, q) == np.percentile(xs, q, method="inverted_cdf")


def test_admission_by_budget_and_release():
    ex = FakeExecutor(budget_bytes=3 * 1280 * 720 * 400)
    srv = Server(ex)
    ok = [srv.admit(k, s) for k, s in specs(5).items()]
    assert ok == [True, True, True, False, False]
    assert srv.rejected == [3, 4]
    srv.release(0)
    assert srv.admit(3, specs(4)[3])
    assert ex.used <= ex.budget


def test_all_served_in_order_one_inflight_per_session():
    ex = FakeExecutor(budget_bytes=1 << 40, ms_per_mpix=0.5)
    srv = Server(ex, max_batch=8)
    ss = specs(6, fps=30.0)
    for k, s in ss.items():
        srv.admit(k, s)
    arr = poisson_arrivals(1, ss, duration_s=1.0)
    st = srv.run(arr)
    assert st["frames"] + st["dropped"] == len(arr)
    assert st["dropped"] == 0                      # light load: nothing superseded
    for sid, frames in st["per_session"].items():
        assert frames == sorted(frames) and len(set(frames)) == len(frames)
    assert st["p50_ms"] <= st["p99_ms"]
    assert st["p99_ms"] < 5.0


def test_continuous_batching_under_load():
    """Arrivals during a running batch join the next one: batches grow with load,
    latency stays bounded because a session keeps only its newest pending frame."""
    ex = FakeExecutor(budget_bytes=1 << 40, ms_per_mpix=4.0)        # ~3.7 ms per 720p frame
    srv = Server(ex, max_batch=32)
    ss = specs(40, fps=60.0)
    for k, s in ss.items():
        srv.admit(k, s)
    arr = poisson_arrivals(2, ss, duration_s=0.5)
    st = srv.run(arr)
    assert st["mean_batch"] > 4 and st["max_batch"] <= 32
    assert st["frames"] + st["dropped"] == len(arr)
    assert st["p99_ms"] < 500.0


def test_failing_session_is_evicted_others_continue():
    ex = FakeExecutor(budget_bytes=1 << 40, fail_on={2})
    srv = Server(ex, max_batch=1)                  # one request per batch: failures stay local
    ss = specs(4, fps=30.0)
    for k, s in ss.items():
        srv.admit(k, s)
    arr = poisson_arrivals(3, ss, duration_s=1.0)
    st = srv.run(arr)
    assert st["failed"] == 1 and 2 not in srv.specs
    assert set(st["per_session"]) == {0, 1, 3}
    n_other = sum(1 for t, sid in arr if sid != 2)
    assert st["frames"] + st["dropped"] == n_other
