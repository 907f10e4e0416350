"""Invariants the paper's algorithm statement fixes, checked on the synthetic
workloads, and the physics indicators of the introduction against truth."""
import numpy as np
import pytest

import oracle
from paper_2207_03936_gb300 import synth, validation

CFG = dict(k_doublets=4, max_scatter_seed=0.04, max_scatter_follow=0.04,
           max_chi2_tracklet=20.0, hit_sigma=0.012)


def check_invariants(ev, res, cfg):
    MZ = ev.module_z
    MZ2 = ev.module_z2    # module pairs: plane of hits with x < 0
    th, ho = res.track_hits, res.hit_offsets
    # each hit in at most one track
    assert np.bincount(th, minlength=ev.n_hits).max(initial=0) <= 1
    lens = np.diff(ho)
    assert (lens >= 3).all()
    assert np.array_equal(res.ndof, 2 * lens - 4)
    for e in range(ev.n_events):
        lo, hi = ev.event_offsets[e], ev.event_offsets[e + 1]
        t0, t1 = res.track_offsets[e], res.track_offsets[e + 1]
        mins = []
        for t in range(t0, t1):
            h = th[ho[t]:ho[t + 1]]
            assert ((h >= lo) & (h < hi)).all()           # hits of its own event
            mod = ev.module[h]
            assert (np.diff(mod) >= 1).all()               # traversal order
            assert (np.diff(mod) <= 2).all()               # never two modules missed
            x, y, z = ev.x[h], ev.y[h], ev.z[h]
            for k in range(2, len(h)):
                dz = np.float32(z[k - 1] - z[k - 2])
                zt = MZ2[mod[k]] if MZ2 is not None and x[k] < 0 else MZ[mod[k]]
                tz = np.float32(np.float32(zt - z[k - 1]) / dz)
                xp = np.float32(x[k - 1] + np.float32(np.float32(x[k - 1] - x[k - 2]) * tz))
                yp = np.float32(y[k - 1] + np.float32(np.float32(y[k - 1] - y[k - 2]) * tz))
                dx, dy = np.float32(x[k] - xp), np.float32(y[k] - yp)
                sc = np.float32(np.float32(dx * dx) + np.float32(dy * dy))
                lim = cfg["max_scatter_seed"] if k == 2 else cfg["max_scatter_follow"]
                assert sc < np.float32(lim)
            if len(h) == 3:
                assert res.chi2[t] < np.float32(cfg["max_chi2_tracklet"])
            p, c2 = oracle.fit(x, y, z, cfg["hit_sigma"])
            assert np.array_equal(p, res.params[t]) and c2 == res.chi2[t]
            mins.append(h.min())
        assert (np.diff(mins) > 0).all()                   # canonical order


@pytest.mark.parametrize("config,n", [(1, None), (2, 150), (3, 40)])
def test_invariants(config, n):
    ev = synth.make_events(config, n, workers=1)
    res = oracle.reconstruct(ev.x, ev.y, ev.z, ev.module, ev.event_offsets, ev.module_z,
                             oracle.config(**CFG))
    assert (res.status == 0).all()
    check_invariants(ev, res, CFG)


@pytest.mark.parametrize("config", [1, 2])
def test_physics_indicators_against_truth(config):
    # thresholds fixed once from the first oracle run on these workloads
    ev = synth.make_events(config, workers=1)
    res = oracle.reconstruct(ev.x, ev.y, ev.z, ev.module, ev.event_offsets, ev.module_z,
                             oracle.config(**CFG))
    ind = validation.indicators(res.hit_offsets, res.track_hits, ev.mc, ev.n_particles)
    assert ind["efficiency"] >= 0.995
    assert ind["fake_fraction"] <= 0.005
    assert ind["clone_fraction"] <= 0.015
    assert ind["hit_purity"] >= 0.995
    assert ind["hit_efficiency"] >= 0.98


@pytest.mark.parametrize("config,n", [(2, 150), (3, 30)])
def test_invariants_ascending_traversal(config, n):
    """The same hits traversed in ascending z (module ids reversed): the
    track invariants hold in the new module order."""
    ev = synth.reverse_traversal(synth.make_events(config, n, workers=1))
    res = oracle.reconstruct(ev.x, ev.y, ev.z, ev.module, ev.event_offsets, ev.module_z,
                             oracle.config(**CFG))
    assert (res.status == 0).all()
    check_invariants(ev, res, CFG)


@pytest.mark.parametrize("config", [1, 2])
def test_physics_indicators_ascending_traversal(config):
    # same thresholds as the descending traversal
    ev = synth.reverse_traversal(synth.make_events(config, workers=1))
    res = oracle.reconstruct(ev.x, ev.y, ev.z, ev.module, ev.event_offsets, ev.module_z,
                             oracle.config(**CFG))
    ind = validation.indicators(res.hit_offsets, res.track_hits, ev.mc, ev.n_particles)
    assert ind["efficiency"] >= 0.995
    assert ind["fake_fraction"] <= 0.005
    assert ind["clone_fraction"] <= 0.015
    assert ind["hit_purity"] >= 0.995
    assert ind["hit_efficiency"] >= 0.98


def test_batch_equals_single_event_calls():
    ev = synth.make_events(2, 25, workers=1)
    res = oracle.reconstruct(ev.x, ev.y, ev.z, ev.module, ev.event_offsets, ev.module_z,
                             oracle.config(**CFG), n_threads=3)
    for e in range(ev.n_events):
        lo, hi = ev.event_offsets[e], ev.event_offsets[e + 1]
        one = oracle.event(ev.x[lo:hi], ev.y[lo:hi], ev.z[lo:hi], ev.module[lo:hi], ev.module_z,
                           oracle.config(**CFG))
        t0, t1 = res.track_offsets[e], res.track_offsets[e + 1]
        assert t1 - t0 == one.n_tracks
        h0, h1 = res.hit_offsets[t0], res.hit_offsets[t1]
        assert np.array_equal(res.track_hits[h0:h1] - lo, one.track_hits)
        assert np.array_equal(res.params[t0:t1], one.params)
