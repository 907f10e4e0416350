"""Host arithmetic of the bench's serving figures (no GPU): latency runs from
each event's scheduled arrival to its result, events/s is completions over
the span from the first arrival to the last completion on the server's
clock, and the per-run statistics are differences of the server's counters."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class FakeEvents:
    def __init__(self, n):
        self.n_events = n


class FakeServer:
    """Finishes every request at once with a fixed latency per request id,
    in two drains; counters advance by fixed amounts per schedule."""

    def __init__(self, latency_of):
        self.latency_of = latency_of
        self.batches, self.events_batched, self.busy = 10, 40, 1.5
        self.pending = None

    def stats(self):
        return {"batches": self.batches, "mean_batch_events": self.events_batched / self.batches,
                "peak_bytes": 3 << 30, "feed_lag_s": 2e-4, "launch_busy_s": self.busy,
                "upload_ms": 0.5 * self.batches, "kernel_ms": 2.0 * self.batches,
                "download_ms": 0.25 * self.batches, "batch_wall_ms": 4.0 * self.batches,
                "timed_batches": self.batches}

    def submit_schedule(self, ev, arrival, first_id=0):
        assert first_id == 0
        self.pending = np.arange(ev.n_events, dtype=np.int64)
        self.batches += 5
        self.events_batched += ev.n_events
        self.busy += 0.25

    def drain(self, max_results, timeout_s=0.0):
        take = self.pending[:(len(self.pending) + 1) // 2]    # half now, the rest next time
        self.pending = self.pending[len(take):]
        return take, np.zeros(len(take), np.int32), self.latency_of(take)


def test_all_at_once_span_is_the_largest_latency():
    n = 100
    lat = lambda ids: 1e-3 + 1e-5 * ids.astype(np.float64)
    r = bench.serve(None, FakeServer(lat), FakeEvents(n), None, 4 << 30)
    assert r["events"] == n
    span = 1e-3 + 1e-5 * (n - 1)
    assert r["span_ms"] == pytest.approx(span * 1e3)
    assert r["value"] == pytest.approx(n / span)
    assert r["max_ms"] == pytest.approx(span * 1e3)
    assert r["p50_ms"] == pytest.approx(np.percentile(lat(np.arange(n)), 50) * 1e3)
    assert r["mean_batch_events"] == pytest.approx(n / 5)          # this run's batches only
    assert r["launcher_busy_fraction"] == pytest.approx(0.25 / span)
    assert r["generator_max_lag_ms"] == pytest.approx(0.2)
    assert r["budget_gb"] == 4.0
    # per-batch split from this run's counter differences
    assert r["per_batch_ms"] == pytest.approx({"upload_ms": 0.5, "kernel_ms": 2.0, "download_ms": 0.25,
                                               "batch_wall_ms": 4.0})


def test_open_loop_span_runs_from_first_arrival_to_last_completion():
    n, rate = 200, 5000.0
    arrival = bench.synth.poisson_arrivals(rate, n, seed=11)   # the schedule serve() draws
    lat = lambda ids: np.full(len(ids), 2e-3)
    r = bench.serve(None, FakeServer(lat), FakeEvents(n), rate, 2 << 30)
    span = arrival.max() + 2e-3 - arrival.min()
    assert r["span_ms"] == pytest.approx(span * 1e3)
    assert r["value"] == pytest.approx(n / span)
    assert r["offered_hz"] == rate
    assert r["p99_ms"] == pytest.approx(2.0)
