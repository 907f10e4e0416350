"""Pins of the sort stage: a stable sort by (module, phi16) (section "Sort by phi")."""
import numpy as np

import oracle
from paper_2207_03936_gb300 import synth


def test_sort_equals_numpy_stable_lexsort():
    ev = synth.make_events(2, 20)
    for e in range(ev.n_events):
        lo, hi = ev.event_offsets[e], ev.event_offsets[e + 1]
        x, y, m = ev.x[lo:hi], ev.y[lo:hi], ev.module[lo:hi]
        perm, offs, phs = oracle.sort_event(x, y, m, 52)
        ph = oracle.phi16(x, y)
        ref = np.lexsort((np.arange(hi - lo), ph, m))
        assert np.array_equal(perm, ref)
        assert np.array_equal(phs, ph[ref])
        ref_offs = np.concatenate([[0], np.cumsum(np.bincount(m, minlength=52))])
        assert np.array_equal(offs, ref_offs)


def test_sort_ties_keep_input_order():
    x = np.array([3.0, 1.0, 3.0, 3.0, 1.0], np.float32)
    y = np.array([4.0, 1.0, 4.0, 4.0, 1.0], np.float32)
    m = np.array([2, 0, 2, 2, 0], np.int32)
    perm, offs, _ = oracle.sort_event(x, y, m, 4)
    assert perm.tolist() == [1, 4, 0, 2, 3]
    assert offs.tolist() == [0, 2, 2, 5, 5]


def test_sort_rejects_bad_module():
    import pytest
    with pytest.raises(ValueError):
        oracle.sort_event(np.ones(2, np.float32), np.ones(2, np.float32),
                          np.array([0, 52], np.int32), 52)
