"""The 100k-event uneven workload in the launch configuration the benchmark
times (persistent launch under a CUDA graph): sampled events against the
oracle one by one, and properties that hold for every event."""
import numpy as np
import pytest

import oracle
from paper_2207_03936_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CFG = dict(k_doublets=4, max_scatter_seed=0.04, max_scatter_follow=0.04, max_chi2_tracklet=20.0,
           hit_sigma=0.012)


def test_full_uneven_workload():
    from paper_2207_03936_gb300 import sbt
    ev = synth.make_events(3)
    h = sbt.sbt_create(ev.module_z, sbt.default_config(**CFG))
    try:
        dev = [torch.from_numpy(a).cuda() for a in (ev.x, ev.y, ev.z, ev.module, ev.event_offsets)]
        sbt.sbt_autotune(h, *dev)
        out = sbt.sbt_reconstruct_batched(h, *dev)
        out = sbt.sbt_reconstruct_batched(h, *dev, out=out)  # graph replay
        torch.cuda.synchronize()
        r = out.compact()
    finally:
        h.close()
    assert (r["event_status"] == 0).all() and r["counts"][2] == 0
    to, ho, th = r["track_offsets"], r["hit_offsets"], r["track_hits"]
    lens = np.diff(ho)
    assert (lens >= 3).all() and np.array_equal(r["ndof"], 2 * lens - 4)
    assert np.bincount(th, minlength=ev.n_hits).max() <= 1
    # hits of each track belong to its event, tracks ordered by smallest hit
    trk_ev = np.repeat(np.arange(ev.n_events), np.diff(to))
    hit_ev = np.repeat(trk_ev, lens)
    assert np.array_equal(np.searchsorted(ev.event_offsets, th, side="right") - 1, hit_ev)
    first = np.minimum.reduceat(th, ho[:-1]) if len(lens) else np.zeros(0)
    same = trk_ev[1:] == trk_ev[:-1]
    assert (np.diff(first)[same] > 0).all()
    # sampled events: the largest ones and a random draw, one by one
    rng = np.random.default_rng(0)
    sizes = np.diff(ev.event_offsets)
    sample = np.unique(np.concatenate([np.argsort(sizes)[-6:], rng.choice(ev.n_events, 40, False)]))
    for e in sample:
        lo, hi = ev.event_offsets[e], ev.event_offsets[e + 1]
        one = oracle.event(ev.x[lo:hi], ev.y[lo:hi], ev.z[lo:hi], ev.module[lo:hi], ev.module_z,
                           oracle.config(**CFG))
        t0, t1 = to[e], to[e + 1]
        assert t1 - t0 == one.n_tracks
        assert np.array_equal(th[ho[t0]:ho[t1]] - lo, one.track_hits)
        assert np.array_equal(r["params"][t0:t1].view(np.uint32), one.params.view(np.uint32))
        assert np.array_equal(r["chi2"][t0:t1].view(np.uint32), one.chi2.view(np.uint32))
