"""Pins of the alignment objective and its gradient (the differentiation
workload: the least-squares fit of the tracklet filter applied to every
track, summed, as a function of per-module placement parameters)."""
import numpy as np
import pytest

import oracle
from paper_2207_03936_gb300 import synth

SIGMA = 0.012


def truth_tracks(ev):
    """Particles with >= 3 hits as fixed tracks, hits in traversal order."""
    mc = ev.mc
    idx = np.nonzero(mc >= 0)[0]
    order = np.lexsort((ev.module[idx], mc[idx]))
    idx = idx[order]
    pid = mc[idx]
    starts = np.concatenate([[0], np.nonzero(np.diff(pid))[0] + 1, [len(idx)]])
    lens = np.diff(starts)
    keep = np.repeat(lens >= 3, lens)
    idx = idx[keep]
    lens = lens[lens >= 3]
    ho = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    return ho, idx.astype(np.int32)


@pytest.fixture(scope="module")
def aligned_events():
    ev = synth.make_events(5, 12, workers=1)
    ho, th = truth_tracks(ev)
    return ev, ho, th


def central_differences(fun, align):
    """Fourth-order central differences (h^4 truncation), per parameter."""
    fd = np.zeros_like(align)
    for m in range(align.shape[0]):
        for k in range(6):
            h = 1e-4 if k < 3 else 1e-5

            def at(d):
                a = align.copy()
                a[m, k] += d
                return fun(a)

            fd[m, k] = (-at(2 * h) + 8 * at(h) - 8 * at(-h) + at(-2 * h)) / (12 * h)
    return fd


def f(ev, ho, th, align):
    return oracle.align_chi2(ev.x, ev.y, ev.z, ev.module, ho, th, ev.module_z, align, SIGMA,
                             want_grad=False)[0]


def test_gradient_matches_central_differences(aligned_events):
    ev, ho, th = aligned_events
    rng = np.random.default_rng(4)
    align = np.concatenate([rng.normal(0, 0.005, (52, 3)), rng.normal(0, 5e-5, (52, 3))], 1)
    v, g = oracle.align_chi2(ev.x, ev.y, ev.z, ev.module, ho, th, ev.module_z, align, SIGMA)
    assert abs(v - f(ev, ho, th, align)) == 0.0
    fd = central_differences(lambda a: f(ev, ho, th, a), align)
    scale = np.abs(fd).max()
    err = np.abs(g - fd)
    assert (err <= 1e-6 * np.maximum(np.abs(fd), 1e-3 * scale)).all(), err.max()


def test_global_motions_leave_chi2_unchanged(aligned_events):
    # translating every module, or rotating every module about the beam (z)
    # axis, moves all hits rigidly: every line refits to the same chi2
    ev, ho, th = aligned_events
    rng = np.random.default_rng(5)
    align = np.concatenate([rng.normal(0, 0.005, (52, 3)), rng.normal(0, 5e-5, (52, 3))], 1)
    _, g = oracle.align_chi2(ev.x, ev.y, ev.z, ev.module, ho, th, ev.module_z, align, SIGMA)
    # at align != 0 only the translations are rigid motions of the aligned hits
    tot = np.abs(g).sum(0)
    for k in (0, 1, 2):
        assert abs(g[:, k].sum()) <= 1e-9 * tot[k]
    _, g0 = oracle.align_chi2(ev.x, ev.y, ev.z, ev.module, ho, th, ev.module_z,
                              np.zeros((52, 6)), SIGMA)
    tot0 = np.abs(g0).sum(0)
    for k in (0, 1, 2, 5):
        assert abs(g0[:, k].sum()) <= 1e-9 * tot0[k]


def test_exact_lines_have_zero_chi2_and_gradient():
    from tests.hand_events import line_hits, assemble
    parts = [line_hits(5.0 + i, -3.0 + 0.5 * i, 0.002 * i, -0.001, range(4 + i, 30 + i))
             for i in range(5)]
    x, y, z, m, g = assemble(parts)
    ho = np.concatenate([[0], np.cumsum([len(p) for p in g])]).astype(np.int32)
    th = np.concatenate(g).astype(np.int32)
    mz = synth.module_z_traversal()
    v, gr = oracle.align_chi2(x, y, z, m, ho, th, mz, np.zeros((52, 6)), SIGMA)
    # only fp32 representation of the hits remains (~1e-6 mm per coordinate)
    assert v < 1e-3
    assert np.abs(gr).max() < 1.0


def test_objective_at_zero_equals_sum_of_track_fits(aligned_events):
    ev, ho, th = aligned_events
    v, _ = oracle.align_chi2(ev.x, ev.y, ev.z, ev.module, ho, th, ev.module_z,
                             np.zeros((52, 6)), SIGMA, want_grad=False)
    tot = 0.0
    for t in range(len(ho) - 1):
        h = th[ho[t]:ho[t + 1]]
        _, c2 = oracle.fit(ev.x[h], ev.y[h], ev.z[h], SIGMA)
        tot += float(c2)
    assert abs(v - tot) <= 1e-3 * v


def _lstsq_chi2(x, y, z, sigma):
    A = np.stack([np.ones_like(z, dtype=np.float64), np.asarray(z, np.float64)], 1)
    r = 0.0
    for v in (x, y):
        coef = np.linalg.lstsq(A, np.asarray(v, np.float64), rcond=None)[0]
        r += float(((np.asarray(v, np.float64) - A @ coef) ** 2).sum())
    return r / sigma ** 2


def _odd_tracks():
    """Two noisy measurements of one line on each of the 52 modules (as from
    two overlapping sensors), assembled into tracks of unusual shape: one
    with both hits of every module (104 hits, above the 64 of one hit per
    module), one with a repeated module in the middle, and a normal one."""
    from tests.hand_events import MZ
    rng = np.random.default_rng(12)
    mods = np.arange(52)
    zz = MZ[mods].astype(np.float64)
    xa = (6.0 + 0.003 * zz + rng.normal(0, 0.012, 52)).astype(np.float32)
    ya = (-4.0 + 0.002 * zz + rng.normal(0, 0.012, 52)).astype(np.float32)
    xb = (6.0 + 0.003 * zz + rng.normal(0, 0.012, 52)).astype(np.float32)
    yb = (-4.0 + 0.002 * zz + rng.normal(0, 0.012, 52)).astype(np.float32)
    x = np.concatenate([xa, xb])
    y = np.concatenate([ya, yb])
    z = np.concatenate([MZ, MZ]).astype(np.float32)
    m = np.concatenate([mods, mods]).astype(np.int32)
    both = np.stack([np.arange(52), 52 + np.arange(52)], 1).reshape(-1)   # 104 hits, 2 per module
    dup = np.array([3, 4, 5, 5 + 52, 6, 7])                             # module 5 twice
    normal = np.arange(10, 30)
    return x, y, z, m, [both, dup, normal]


def test_long_tracks_and_repeated_modules_follow_least_squares():
    x, y, z, m, tracks = _odd_tracks()
    from tests.hand_events import MZ
    th = np.concatenate(tracks).astype(np.int32)
    ho = np.concatenate([[0], np.cumsum([len(t) for t in tracks])]).astype(np.int32)
    v, g, sk = oracle.align_chi2(x, y, z, m, ho, th, MZ, np.zeros((52, 6)), SIGMA, count_skipped=True)
    ref = sum(_lstsq_chi2(x[t], y[t], z[t], SIGMA) for t in tracks)
    assert sk == 0
    assert abs(v - ref) <= 1e-9 * ref
    # the gradient of these tracks against central differences
    rng = np.random.default_rng(13)
    align = np.concatenate([rng.normal(0, 0.005, (52, 3)), rng.normal(0, 5e-5, (52, 3))], 1)
    _, g = oracle.align_chi2(x, y, z, m, ho, th, MZ, align, SIGMA)
    fd = central_differences(lambda a: oracle.align_chi2(x, y, z, m, ho, th, MZ, a, SIGMA, False)[0], align)
    scale = np.abs(fd).max()
    assert (np.abs(g - fd) <= 1e-6 * np.maximum(np.abs(fd), 1e-3 * scale)).all()


def test_tracks_without_a_line_fit_are_skipped_and_counted():
    # a track contributes only when it has a straight-line fit and its indices
    # are in range: one hit, no hit, two hits on one module, an index past the
    # hits and a module id past the modules are each skipped and counted
    x, y, z, m, tracks = _odd_tracks()
    from tests.hand_events import MZ
    # hit 104: a module id out of range; index 105: past the hits
    x, y, z = (np.append(a, np.float32(a[0])) for a in (x, y, z))
    m = np.append(m, np.int32(52))
    bad = [np.array([11]), np.array([], np.int64), np.array([5, 5 + 52]), np.array([1, 2, 105]),
           np.array([58, 59, 104, 61])]
    good = tracks
    allt = [good[0], bad[0], good[1], bad[1], bad[2], good[2], bad[3], bad[4]]
    th = np.concatenate(allt).astype(np.int32)
    ho = np.concatenate([[0], np.cumsum([len(t) for t in allt])]).astype(np.int32)
    v, g, sk = oracle.align_chi2(x, y, z, m, ho, th, MZ, np.zeros((52, 6)), SIGMA, count_skipped=True)
    thg = np.concatenate(good).astype(np.int32)
    hog = np.concatenate([[0], np.cumsum([len(t) for t in good])]).astype(np.int32)
    vg, gg = oracle.align_chi2(x, y, z, m, hog, thg, MZ, np.zeros((52, 6)), SIGMA)
    assert sk == len(bad)
    assert v == vg and np.array_equal(g, gg)
