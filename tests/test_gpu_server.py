"""Continuous-batching request loop: every served result equals the result of
the same event reconstructed alone; events submitted while others run are
admitted as slots and budget free up; a host-side batch failure completes its
requests with an error and the loop continues."""
import time

import numpy as np
import pytest

import oracle
from paper_2207_03936_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def collect(server, n, timeout=60.0):
    got = {}
    t0 = time.time()
    while len(got) < n and time.time() - t0 < timeout:
        for r in server.poll(256, timeout_s=0.05):
            got[r.request_id] = r
    return got


def test_served_results_equal_results_alone():
    from paper_2207_03936_gb300 import sbt
    ev = synth.make_events(2, 300, workers=1)
    h = sbt.sbt_create(ev.module_z, sbt.default_config())
    srv = sbt.Server(h, memory_budget_bytes=64 << 20, max_streams=4, max_batch_events=32)
    try:
        arrival = synth.poisson_arrivals(20000.0, ev.n_events, seed=3)
        srv.submit_schedule(ev, arrival)
        got = collect(srv, ev.n_events)
        st = srv.stats()
    finally:
        srv.close()
        h.close()
    assert len(got) == ev.n_events
    assert st["batches"] > 1 and st["peak_bytes"] <= 64 << 20
    assert 0.0 <= st["feed_lag_s"] < 1.0 and st["launch_busy_s"] > 0.0
    for e in range(ev.n_events):
        lo, hi = ev.event_offsets[e], ev.event_offsets[e + 1]
        one = oracle.event(ev.x[lo:hi], ev.y[lo:hi], ev.z[lo:hi], ev.module[lo:hi], ev.module_z)
        r = got[e]
        assert r.status == 0
        assert np.array_equal(r.hit_offsets, one.hit_offsets)
        assert np.array_equal(r.track_hits, one.track_hits)
        assert np.array_equal(r.params, one.params)
        assert r.latency_s > 0


def test_overlapping_admission_and_failure_recovery():
    from paper_2207_03936_gb300 import sbt
    ev = synth.make_events(2, 120, workers=1)
    h = sbt.sbt_create(ev.module_z, sbt.default_config())
    # a small budget forces several batches in flight and waiting admissions
    srv = sbt.Server(h, memory_budget_bytes=8 << 20, max_streams=3, max_batch_events=8)
    try:
        srv.inject_failure()
        for e in range(ev.n_events):
            lo, hi = ev.event_offsets[e], ev.event_offsets[e + 1]
            srv.submit(e, ev.x[lo:hi], ev.y[lo:hi], ev.z[lo:hi], ev.module[lo:hi])
        got = collect(srv, ev.n_events)
        st = srv.stats()
    finally:
        srv.close()
        h.close()
    assert len(got) == ev.n_events
    failed = [r for r in got.values() if r.status == sbt.SBT_ERR_CUDA]
    assert 1 <= len(failed) <= 8 and st["failed_batches"] == 1
    assert st["batches"] >= ev.n_events / 8
    ok = [r for r in got.values() if r.status == 0]
    assert len(ok) == ev.n_events - len(failed)
    for r in ok:
        e = r.request_id
        lo, hi = ev.event_offsets[e], ev.event_offsets[e + 1]
        one = oracle.event(ev.x[lo:hi], ev.y[lo:hi], ev.z[lo:hi], ev.module[lo:hi], ev.module_z)
        assert np.array_equal(r.track_hits, one.track_hits)


def test_served_results_keep_storage_and_event_cut_settings():
    """Server slots reconstruct with the settings of the handle they are
    created from: fp16 hit storage and the global event cut."""
    from paper_2207_03936_gb300 import sbt
    ev = synth.make_events(2, 120, workers=1)
    sizes = np.diff(ev.event_offsets)
    thr = int(np.quantile(sizes, 0.8))
    h = sbt.sbt_create(ev.module_z, sbt.default_config(fp16_hits=1, gec_max_hits=thr))
    srv = sbt.Server(h, memory_budget_bytes=64 << 20, max_streams=2, max_batch_events=16)
    try:
        srv.submit_schedule(ev, np.zeros(ev.n_events))
        got = collect(srv, ev.n_events)
    finally:
        srv.close()
        h.close()
    assert len(got) == ev.n_events
    cfg = oracle.config()
    for e in range(ev.n_events):
        r = got[e]
        if sizes[e] > thr:
            assert r.status == sbt.SBT_EVENT_CUT and len(r.hit_offsets) == 1
            continue
        lo, hi = ev.event_offsets[e], ev.event_offsets[e + 1]
        one = oracle.event(oracle.round_fp16(ev.x[lo:hi]), oracle.round_fp16(ev.y[lo:hi]),
                           oracle.round_fp16(ev.z[lo:hi]), ev.module[lo:hi], ev.module_z, cfg)
        assert r.status == 0
        assert np.array_equal(r.hit_offsets, one.hit_offsets)
        assert np.array_equal(r.track_hits, one.track_hits)
        assert np.array_equal(r.params.view(np.uint32), one.params.view(np.uint32))


def test_consecutive_schedules_reuse_the_pinned_batch():
    """A second open-loop schedule on the same server takes the pinned host
    batch the first one returned to the pool (smaller, so it fits) and serves
    the same results as each event alone."""
    from paper_2207_03936_gb300 import sbt
    ev1 = synth.make_events(2, 80, seed=1, workers=1)
    ev2 = synth.make_events(2, 40, seed=2, workers=1)
    h = sbt.sbt_create(ev1.module_z, sbt.default_config())
    srv = sbt.Server(h, memory_budget_bytes=64 << 20, max_streams=3, max_batch_events=16)
    try:
        srv.submit_schedule(ev1, np.zeros(ev1.n_events))
        got1 = collect(srv, ev1.n_events)
        srv.submit_schedule(ev2, synth.poisson_arrivals(50000.0, ev2.n_events, seed=5), first_id=1000)
        got2 = collect(srv, ev2.n_events)
    finally:
        srv.close()
        h.close()
    assert sorted(got1) == list(range(ev1.n_events))
    assert sorted(got2) == list(range(1000, 1000 + ev2.n_events))
    for ev, got, base in ((ev1, got1, 0), (ev2, got2, 1000)):
        for e in range(ev.n_events):
            lo, hi = ev.event_offsets[e], ev.event_offsets[e + 1]
            one = oracle.event(ev.x[lo:hi], ev.y[lo:hi], ev.z[lo:hi], ev.module[lo:hi], ev.module_z)
            r = got[base + e]
            assert r.status == 0
            assert np.array_equal(r.hit_offsets, one.hit_offsets)
            assert np.array_equal(r.track_hits, one.track_hits)
            assert np.array_equal(r.params, one.params)


def test_served_results_keep_module_pairs():
    """Slots of a server made from a module-pair handle reconstruct with the
    pair geometry: every served event equals the oracle's pair reading."""
    from paper_2207_03936_gb300 import sbt
    ev = synth.make_events(2, 60, seed=3, workers=1, pairs=True)
    h = sbt.sbt_create(ev.module_z, sbt.default_config(), module_z2=ev.module_z2)
    srv = sbt.Server(h, memory_budget_bytes=64 << 20, max_streams=2, max_batch_events=16)
    try:
        srv.submit_schedule(ev, np.zeros(ev.n_events))
        got = collect(srv, ev.n_events)
    finally:
        srv.close()
        h.close()
    assert len(got) == ev.n_events
    for e in range(ev.n_events):
        lo, hi = ev.event_offsets[e], ev.event_offsets[e + 1]
        one = oracle.event(ev.x[lo:hi], ev.y[lo:hi], ev.z[lo:hi], ev.module[lo:hi], ev.module_z,
                           module_z2=ev.module_z2)
        r = got[e]
        assert r.status == 0
        assert np.array_equal(r.hit_offsets, one.hit_offsets)
        assert np.array_equal(r.track_hits, one.track_hits)
        assert np.array_equal(r.params, one.params)
