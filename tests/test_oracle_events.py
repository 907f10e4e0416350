"""Hand-built events with outcomes known by construction (section "Track
seeding and track following" and "Tracklet filter")."""
import math

import numpy as np

import oracle
from paper_2207_03936_gb300 import synth
from tests.hand_events import (MZ, assemble, following_tie, line_hits, seeding_tie, seeding_tie_third,
                               single_track, tracklet_conflict)


def tracks_of(res):
    return [res.track_hits[res.hit_offsets[t]:res.hit_offsets[t + 1]].tolist()
            for t in range(res.n_tracks)]


def run(x, y, z, m, **cfg):
    return oracle.event(x, y, z, m, MZ, oracle.config(**cfg))


def test_empty_and_degenerate_events():
    e = np.zeros(0, np.float32)
    r = run(e, e, e, np.zeros(0, np.int32))
    assert r.n_tracks == 0
    # hits on a single module never make a track
    x, y, z, m = line_hits(5.0, 6.0, 0.0, 0.0, [7, 7, 7])
    assert run(x, y, z, m).n_tracks == 0


def test_single_straight_track_found_whole():
    x, y, z, m, g = single_track()
    r = run(x, y, z, m)
    assert tracks_of(r) == [g.tolist()]
    assert r.ndof[0] == 2 * 52 - 4
    np.testing.assert_allclose(r.params[0], [8.0, 5.0, 0.004, -0.003], atol=2e-5)


def test_one_missing_module_is_bridged():
    x, y, z, m, g = single_track(missing=(20,))
    assert tracks_of(run(x, y, z, m)) == [g.tolist()]


def test_two_consecutive_missing_modules_split_the_track():
    x, y, z, m, g = single_track(missing=(20, 21))
    got = tracks_of(run(x, y, z, m))
    first = [h for h, mod in zip(g, [k for k in range(52) if k not in (20, 21)]) if mod < 20]
    second = [h for h, mod in zip(g, [k for k in range(52) if k not in (20, 21)]) if mod > 21]
    assert sorted(got) == sorted([first, second])


def test_three_hit_track_passes_filter_and_tight_cut_rejects_it():
    x, y, z, m = line_hits(6.0, -7.0, 0.01, 0.002, [30, 31, 32],
                           jitter=(np.array([0.0, 0.01, 0.0]), np.zeros(3)))
    r = run(x, y, z, m)
    assert tracks_of(r) == [[0, 1, 2]]
    # moving the middle hit by d makes the second difference 2 d, and the
    # residual sum of three equally spaced points is |second difference|^2 / 6
    q = (2 * 0.01) ** 2 / 6 / 0.012 ** 2
    assert abs(float(r.chi2[0]) - q) < 1e-2 * q
    assert run(x, y, z, m, max_chi2_tracklet=q * 0.5).n_tracks == 0


def test_crossing_tracks_distinct_scatter():
    zc = float(MZ[11])
    pa = np.array([10.0, 3.0])
    ta = np.array([0.004, 0.001])
    tb = np.array([-0.003, 0.006])
    pb = pa + np.array([0.0, 0.15])       # B passes 0.15 mm above A at module 11
    a0 = pa - ta * zc
    b0 = pb - tb * zc
    mods = [k for k in range(0, 24) if k != 11]
    A = line_hits(a0[0], a0[1], ta[0], ta[1], mods)
    B = line_hits(b0[0], b0[1], tb[0], tb[1], mods)
    h = pa + np.array([0.0, 0.06])       # 0.06 mm from A, 0.09 mm from B: both under 0.2 mm
    shared = (np.array([h[0]], np.float32), np.array([h[1]], np.float32),
              np.array([MZ[11]], np.float32), np.array([11], np.int32))
    x, y, z, m, g = assemble([A, B, shared], shuffle_seed=7)
    got = sorted(tracks_of(run(x, y, z, m)), key=len)
    a_full = sorted(g[0].tolist() + [int(g[2][0])], key=lambda i: m[i])
    b_miss = g[1].tolist()
    assert sorted(got) == sorted([a_full, b_miss])


def test_equal_scatter_tie_goes_to_smaller_track_key():
    # B is the exact mirror of A in y; the lines meet on the x axis at module 11
    # where the only hit sits 0.05 mm off both predictions, so the two claims
    # carry bitwise-equal scatter.  The tie goes to the smaller track key (the
    # seed's middle-hit sorted position): A, whose hits have positive phi and
    # therefore sort first on every module.
    zc = float(MZ[11])
    t = np.array([0.003, 0.02])
    mods = [k for k in range(0, 24) if k != 11]
    A = line_hits(12.0 - t[0] * zc, 0.0 - t[1] * zc, t[0], t[1], mods)
    B = (A[0].copy(), -A[1], A[2].copy(), A[3].copy())
    shared = (np.array([12.05], np.float32), np.array([0.0], np.float32),
              np.array([MZ[11]], np.float32), np.array([11], np.int32))
    x, y, z, m, g = assemble([A, B, shared], shuffle_seed=9)
    got = tracks_of(run(x, y, z, m))
    a_full = sorted(g[0].tolist() + [int(g[2][0])], key=lambda i: m[i])
    assert sorted(got) == sorted([a_full, g[1].tolist()])


def test_phi_wrap_track_along_positive_x():
    # hits alternate just above and below the +x axis: phi16 near 0 and near 65535
    mods = list(range(5, 25))
    jit = np.where(np.arange(20) % 2 == 0, 0.003, -0.003)
    x, y, z, m = line_hits(9.0, 0.0, 0.002, 0.0, mods, jitter=(np.zeros(20), jit))
    ph = oracle.phi16(x, y)
    assert (ph < 100).any() and (ph > 65400).any()
    r = run(x, y, z, m)
    assert tracks_of(r) == [list(range(20))]


def test_input_order_does_not_change_tracks():
    ev = synth.make_events(2, 30)
    rng = np.random.default_rng(2)
    for e in range(ev.n_events):
        lo, hi = ev.event_offsets[e], ev.event_offsets[e + 1]
        x, y, z, m = ev.x[lo:hi], ev.y[lo:hi], ev.z[lo:hi], ev.module[lo:hi]
        a = {tuple(t) for t in tracks_of(run(x, y, z, m))}
        p = rng.permutation(hi - lo)
        b = tracks_of(run(x[p], y[p], z[p], m[p]))
        b = {tuple(int(p[i]) for i in t) for t in b}
        assert a == b


def test_overlapping_tracklets_smaller_chi2_survives():
    # reading R7: both tracklets pass the cut with three unflagged hits; they
    # share hit A, and the one with the smaller chi2 keeps it although its
    # track key is the larger one
    x, y, z, m, (t1, t2) = tracklet_conflict(equal_chi2=False)
    q1 = float(oracle.fit(x[t1], y[t1], z[t1], 0.012)[1])
    q2 = float(oracle.fit(x[t2], y[t2], z[t2], 0.012)[1])
    assert q1 < q2 < 20.0
    r = run(x, y, z, m)
    assert tracks_of(r) == [t1]
    assert int(r.stats[0, 1]) == 2 and int(r.stats[0, 2]) == 1   # two tracklets, one accepted
    # with the cut between the two chi2 values only track 1 passes: same result
    assert tracks_of(run(x, y, z, m, max_chi2_tracklet=(q1 + q2) / 2)) == [t1]
    # with the cut below both neither survives
    assert tracks_of(run(x, y, z, m, max_chi2_tracklet=q1 * 0.5)) == []


def test_overlapping_tracklets_equal_chi2_go_to_smaller_track_key():
    # the two tracklets are mirror images in y, so their chi2 are bitwise
    # equal; the claim goes to the smaller track key, track 2 (its middle
    # hit has the smaller phi16 and sorts first on module 31)
    x, y, z, m, (t1, t2) = tracklet_conflict(equal_chi2=True)
    q1 = oracle.fit(x[t1], y[t1], z[t1], 0.012)[1]
    q2 = oracle.fit(x[t2], y[t2], z[t2], 0.012)[1]
    assert q1.view(np.uint32) == q2.view(np.uint32)
    perm, offs, _ = oracle.sort_event(x, y, m, 52)
    pos = np.argsort(perm)
    assert pos[t2[1]] < pos[t1[1]]
    assert tracks_of(run(x, y, z, m)) == [t2]


def _f32_scatter(ax, ay, az, cx, cy, cz, bx, by, zt):
    f = np.float32
    tz = f(f(f(zt) - f(cz)) / f(f(cz) - f(az)))
    xp = f(f(cx) + f(f(f(cx) - f(ax)) * tz))
    yp = f(f(cy) + f(f(f(cy) - f(ay)) * tz))
    dx, dy = f(f(bx) - xp), f(f(by) - yp)
    return f(f(dx * dx) + f(dy * dy))


def test_following_tie_goes_to_smaller_sorted_position():
    # reading R5: two hits on module 15 at bitwise-equal scatter from the
    # track's prediction; the one with the smaller sorted position is taken
    x, y, z, m, track = following_tie()
    k = [i for i in range(len(x)) if m[i] == 15]
    assert len(k) == 2
    prev = [i for i in track if m[i] in (13, 14)]
    s = [_f32_scatter(x[prev[0]], y[prev[0]], z[prev[0]], x[prev[1]], y[prev[1]], z[prev[1]],
                      x[i], y[i], MZ[15]) for i in k]
    assert s[0].view(np.uint32) == s[1].view(np.uint32) and s[0] < 0.04
    assert tracks_of(run(x, y, z, m)) == [track]


def test_seeding_tie_goes_to_smaller_outer_position():
    # reading R4: the triplets (A1, C, B1) and (A2, C, B2) have bitwise-equal
    # scatter; the kept one has the outer hit of smaller sorted position
    x, y, z, m, tl = seeding_tie()
    a1, c, b1 = tl
    a2 = [i for i in range(len(x)) if m[i] == 30 and i != a1][0]
    b2 = [i for i in range(len(x)) if m[i] == 32 and i != b1][0]
    s1 = _f32_scatter(x[a1], y[a1], z[a1], x[c], y[c], z[c], x[b1], y[b1], MZ[32])
    s2 = _f32_scatter(x[a2], y[a2], z[a2], x[c], y[c], z[c], x[b2], y[b2], MZ[32])
    assert s1.view(np.uint32) == s2.view(np.uint32) and s1 < 0.04
    assert tracks_of(run(x, y, z, m)) == [tl]


def test_seeding_tie_goes_to_smaller_third_position():
    # reading R4: one doublet, two third hits at bitwise-equal scatter; the
    # kept one has the smaller sorted position
    x, y, z, m, tl = seeding_tie_third()
    a, c, b1 = tl
    b2 = [i for i in range(len(x)) if m[i] == 32 and i != b1][0]
    s1 = _f32_scatter(x[a], y[a], z[a], x[c], y[c], z[c], x[b1], y[b1], MZ[32])
    s2 = _f32_scatter(x[a], y[a], z[a], x[c], y[c], z[c], x[b2], y[b2], MZ[32])
    assert s1.view(np.uint32) == s2.view(np.uint32) and s1 < 0.04
    assert tracks_of(run(x, y, z, m)) == [tl]
