"""The seeded input generator: the same batch whatever the number of worker
processes (chunks of events are independent random streams), and the
module-pair geometry's one-sided planes."""
import numpy as np
import pytest

from paper_2207_03936_gb300 import synth

FIELDS = ("x", "y", "z", "module", "event_offsets", "mc")


@pytest.mark.parametrize("pairs", [False, True])
def test_batch_does_not_depend_on_worker_count(pairs):
    a = synth.make_events(3, 4500, seed=9, workers=1, pairs=pairs)   # three chunks of events
    b = synth.make_events(3, 4500, seed=9, workers=3, pairs=pairs)
    for f in FIELDS:
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    assert a.n_particles == b.n_particles


def test_subset_and_reverse_keep_the_pair_planes():
    ev = synth.make_events(2, 30, workers=1, pairs=True)
    sub = ev.subset(5, 10)
    assert np.array_equal(sub.module_z2, ev.module_z2)
    lo, hi = ev.event_offsets[5], ev.event_offsets[15]
    assert np.array_equal(sub.x, ev.x[lo:hi]) and sub.event_offsets[-1] == hi - lo
    rev = synth.reverse_traversal(ev)
    M = synth.N_PAIRS
    assert np.array_equal(rev.module_z2, ev.module_z2[::-1])
    assert np.array_equal(rev.module_z[rev.module], ev.module_z[ev.module])
    assert np.array_equal(rev.module_z2[rev.module], ev.module_z2[ev.module])
    assert rev.module.max() == M - 1


def test_pair_planes_and_occupancy():
    ev = synth.make_events(2, 200, workers=1, pairs=True)
    single = synth.make_events(2, 200, workers=1)
    # every plane holds hits of its own side only, at its own z
    for m in range(synth.N_PAIRS):
        on = ev.module == m
        assert set(np.unique(ev.z[on & (ev.x >= 0)])) <= {ev.module_z[m]}
        assert set(np.unique(ev.z[on & (ev.x < 0)])) <= {ev.module_z2[m]}
    # a track crosses half the planes it would cross with full annuli
    ratio = ev.n_hits / single.n_hits
    assert 0.4 < ratio < 0.6
    assert 1500 < ev.n_hits / ev.n_events < 2800      # the upgrade configuration's ~2000 hits/event
