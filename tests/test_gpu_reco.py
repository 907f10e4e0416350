"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle.

Track sets, hit lists, fitted parameters and chi2 must be bit-identical to the
oracle's (fp32 decision arithmetic, every operation rounded as written on
both sides); the stated tolerance for the fit parameters (1e-5 relative) is
therefore met with margin zero.
"""
import numpy as np
import pytest

import oracle
from paper_2207_03936_gb300 import synth
from tests.hand_events import (MZ, assemble, following_tie, line_hits, seeding_tie, seeding_tie_third,
                               single_track, tracklet_conflict)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CFG = dict(k_doublets=4, max_scatter_seed=0.04, max_scatter_follow=0.04, max_chi2_tracklet=20.0,
           hit_sigma=0.012)


@pytest.fixture(scope="module")
def sbt():
    from paper_2207_03936_gb300 import sbt as s
    s.lib()
    return s


@pytest.fixture(scope="module")
def handle(sbt):
    h = sbt.sbt_create(MZ, sbt.default_config(**CFG))
    yield h
    h.close()


def to_dev(ev):
    d = "cuda"
    return (torch.from_numpy(ev.x).to(d), torch.from_numpy(ev.y).to(d), torch.from_numpy(ev.z).to(d),
            torch.from_numpy(ev.module).to(d), torch.from_numpy(ev.event_offsets).to(d))


def arrays(x, y, z, m):
    off = np.array([0, len(x)], np.int32)
    return synth.Events(np.asarray(x, np.float32), np.asarray(y, np.float32),
                        np.asarray(z, np.float32), np.asarray(m, np.int32), off,
                        np.full(len(x), -1, np.int32), 0, MZ)


def run_gpu(sbt, handle, ev, batched=False):
    fn = sbt.sbt_reconstruct_batched if batched else sbt.sbt_reconstruct
    out = fn(handle, *to_dev(ev))
    torch.cuda.synchronize()
    return out.compact()


def assert_same(g, o):
    assert (g["event_status"] == o.status).all()
    assert int(g["counts"][2]) == 0
    assert np.array_equal(g["track_offsets"], o.track_offsets)
    assert np.array_equal(g["hit_offsets"], o.hit_offsets)
    assert np.array_equal(g["track_hits"], o.track_hits)
    assert np.array_equal(g["ndof"], o.ndof)
    # bit-identical fits (the contract is 1e-5 relative)
    assert np.array_equal(g["params"].view(np.uint32), o.params.view(np.uint32))
    assert np.array_equal(g["chi2"].view(np.uint32), o.chi2.view(np.uint32))


def oracle_of(ev):
    return oracle.reconstruct(ev.x, ev.y, ev.z, ev.module, ev.event_offsets, ev.module_z,
                              oracle.config(**CFG))


def test_phi16_bit_exact(sbt):
    rng = np.random.default_rng(0)
    ang = np.linspace(-np.pi, np.pi, 200001)
    r = rng.uniform(0.01, 60.0, ang.shape[0])
    x = np.concatenate([r * np.cos(ang), rng.uniform(-50, 50, 100000), [0.0, -1.0, 1.0, 0.0, -3.0]])
    y = np.concatenate([r * np.sin(ang), rng.uniform(-50, 50, 100000), [0.0, 0.0, 0.0, 2.0, -0.0]])
    x, y = x.astype(np.float32), y.astype(np.float32)
    g = sbt.sbt_debug_phi16(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(g.cpu().numpy().view(np.uint16), oracle.phi16(x, y))


def test_sort_stage_bit_exact(sbt, handle):
    ev = synth.make_events(2, 60, workers=1)
    phi, perm, mo = sbt.sbt_debug_sort(handle, *[to_dev(ev)[i] for i in (0, 1, 3, 4)])
    torch.cuda.synchronize()
    phi = phi.cpu().numpy().view(np.uint16)
    perm = perm.cpu().numpy()
    mo = mo.cpu().numpy()
    for e in range(ev.n_events):
        lo, hi = ev.event_offsets[e], ev.event_offsets[e + 1]
        p, o, ph = oracle.sort_event(ev.x[lo:hi], ev.y[lo:hi], ev.module[lo:hi], 52)
        assert np.array_equal(perm[lo:hi], p)
        assert np.array_equal(phi[lo:hi], ph)
        assert np.array_equal(mo[e], o)


def test_sort_crowded_buckets_bit_exact(sbt):
    """Sort parity where (module, coarse phi) buckets hold many hits: equal
    phi16 values (order by input index), a dense phi band, and a sparse rest."""
    rng = np.random.default_rng(5)
    parts = []
    # 3000 hits at one point (identical phi16), 2500 in a narrow phi band,
    # 40 alone in their buckets, all on modules 3 and 7, plus a sparse spread
    parts.append((np.full(3000, 7.0), np.full(3000, 2.0), np.full(3000, 3)))
    ang = rng.uniform(0.30, 0.32, 2500)
    parts.append((10 * np.cos(ang), 10 * np.sin(ang), np.full(2500, 7)))
    ang = np.linspace(-3.1, 3.1, 40)
    parts.append((20 * np.cos(ang), 20 * np.sin(ang), np.full(40, 3)))
    ang = rng.uniform(-np.pi, np.pi, 900)
    parts.append((15 * np.cos(ang), 15 * np.sin(ang), rng.integers(0, 52, 900)))
    x = np.concatenate([p[0] for p in parts]).astype(np.float32)
    y = np.concatenate([p[1] for p in parts]).astype(np.float32)
    m = np.concatenate([p[2] for p in parts]).astype(np.int32)
    perm0 = rng.permutation(len(x))
    x, y, m = x[perm0], y[perm0], m[perm0]
    z = MZ[m].astype(np.float32)
    ev = arrays(x, y, z, m)
    h = sbt.sbt_create(MZ, sbt.default_config(max_hits_per_event=8192, **CFG))
    try:
        phi, perm, mo = sbt.sbt_debug_sort(h, *[to_dev(ev)[i] for i in (0, 1, 3, 4)])
        torch.cuda.synchronize()
    finally:
        h.close()
    p, o, ph = oracle.sort_event(ev.x, ev.y, ev.module, 52)
    assert np.array_equal(perm.cpu().numpy(), p)
    assert np.array_equal(phi.cpu().numpy().view(np.uint16), ph)
    assert np.array_equal(mo.cpu().numpy()[0], o)


@pytest.mark.parametrize("batched", [False, True])
def test_small_workload_bit_exact(sbt, handle, batched):
    ev = synth.make_events(1, workers=1)
    assert_same(run_gpu(sbt, handle, ev, batched), oracle_of(ev))


@pytest.mark.parametrize("batched", [False, True])
def test_upgrade_workload_bit_exact(sbt, handle, batched):
    ev = synth.make_events(2)
    assert_same(run_gpu(sbt, handle, ev, batched), oracle_of(ev))


@pytest.mark.parametrize("config,n", [(2, 300), (3, 150)])
def test_ascending_traversal_bit_exact(sbt, config, n):
    """Traversal in ascending z (module ids and plane positions reversed):
    the same kernels, plain and batched, against the oracle."""
    ev = synth.reverse_traversal(synth.make_events(config, n))
    h = sbt.sbt_create(ev.module_z, sbt.default_config(**CFG))
    try:
        o = oracle_of(ev)
        assert_same(run_gpu(sbt, h, ev, False), o)
        assert_same(run_gpu(sbt, h, ev, True), o)
    finally:
        h.close()


def oracle_without(o, keep):
    """The oracle's CSR tracks with the events where keep is False emptied."""
    to, ho = o.track_offsets, o.hit_offsets
    tracks = np.concatenate([np.arange(to[e], to[e + 1]) for e in range(len(keep)) if keep[e]]
                            + [np.zeros(0, np.int64)]).astype(np.int64)
    lens = ho[tracks + 1] - ho[tracks]
    hits = np.concatenate([o.track_hits[ho[t]:ho[t + 1]] for t in tracks] + [np.zeros(0, np.int32)])
    per_event = np.array([(to[e + 1] - to[e]) if keep[e] else 0 for e in range(len(keep))])
    return dict(track_offsets=np.concatenate([[0], np.cumsum(per_event)]).astype(np.int32),
                hit_offsets=np.concatenate([[0], np.cumsum(lens)]).astype(np.int32),
                track_hits=hits.astype(np.int32), params=o.params[tracks], chi2=o.chi2[tracks],
                ndof=o.ndof[tracks])


@pytest.mark.parametrize("batched", [False, True])
def test_global_event_cut(sbt, batched):
    """Events above gec_max_hits are rejected (status SBT_EVENT_CUT, no tracks,
    not counted as failed); every other event is reconstructed exactly as
    without the cut."""
    ev = synth.make_events(3, 200)
    sizes = np.diff(ev.event_offsets)
    thr = int(np.quantile(sizes, 0.9))
    keep = sizes <= thr
    h = sbt.sbt_create(ev.module_z, sbt.default_config(gec_max_hits=thr, **CFG))
    try:
        g = run_gpu(sbt, h, ev, batched)
    finally:
        h.close()
    assert (g["event_status"][~keep] == sbt.SBT_EVENT_CUT).all()
    assert (g["event_status"][keep] == sbt.SBT_OK).all()
    assert int(g["counts"][3]) == 0 and int(g["counts"][2]) == 0
    want = oracle_without(oracle_of(ev), keep)
    for k in ("track_offsets", "hit_offsets", "track_hits", "ndof"):
        assert np.array_equal(g[k], want[k]), k
    assert np.array_equal(g["params"].view(np.uint32), want["params"].view(np.uint32))
    assert np.array_equal(g["chi2"].view(np.uint32), want["chi2"].view(np.uint32))


@pytest.mark.parametrize("config,n", [(2, 300), (3, 150)])
def test_fp16_hit_storage_bit_exact(sbt, config, n):
    """fp16 hit storage: plain and batched equal the oracle run on coordinates
    rounded to fp16; the sort stage equals the oracle's sort of them."""
    ev = synth.make_events(config, n)
    h = sbt.sbt_create(ev.module_z, sbt.default_config(fp16_hits=1, **CFG))
    try:
        o = oracle.reconstruct(ev.x, ev.y, ev.z, ev.module, ev.event_offsets, ev.module_z,
                               oracle.config(**CFG), fp16_hits=True)
        assert_same(run_gpu(sbt, h, ev, False), o)
        assert_same(run_gpu(sbt, h, ev, True), o)
        phi, perm, mo = sbt.sbt_debug_sort(h, *[to_dev(ev)[i] for i in (0, 1, 3, 4)])
        torch.cuda.synchronize()
    finally:
        h.close()
    phi = phi.cpu().numpy().view(np.uint16)
    perm = perm.cpu().numpy()
    xr, yr = oracle.round_fp16(ev.x), oracle.round_fp16(ev.y)
    for e in range(0, ev.n_events, 7):
        lo, hi = ev.event_offsets[e], ev.event_offsets[e + 1]
        p, _, ph = oracle.sort_event(xr[lo:hi], yr[lo:hi], ev.module[lo:hi], 52)
        assert np.array_equal(perm[lo:hi], p)
        assert np.array_equal(phi[lo:hi], ph)


def test_uneven_workload_bit_exact(sbt, handle):
    ev = synth.make_events(3, 400)
    o = oracle_of(ev)
    assert_same(run_gpu(sbt, handle, ev, False), o)
    assert_same(run_gpu(sbt, handle, ev, True), o)


@pytest.mark.parametrize("threads", [64, 128, 256])
def test_block_sizes_agree(sbt, threads):
    ev = synth.make_events(2, 120, workers=1)
    h = sbt.sbt_create(MZ, sbt.default_config(threads_per_block=threads, **CFG))
    try:
        o = oracle_of(ev)
        assert_same(run_gpu(sbt, h, ev, False), o)
        assert_same(run_gpu(sbt, h, ev, True), o)
    finally:
        h.close()


def test_hand_built_events(sbt, handle):
    cases = []
    x, y, z, m, _ = single_track()
    cases.append((x, y, z, m))
    x, y, z, m, _ = single_track(missing=(20, 21))
    cases.append((x, y, z, m))
    t = np.array([0.003, 0.02])
    zc = float(MZ[11])
    mods = [k for k in range(0, 24) if k != 11]
    A = line_hits(12.0 - t[0] * zc, -t[1] * zc, t[0], t[1], mods)
    B = (A[0].copy(), -A[1], A[2].copy(), A[3].copy())
    S = (np.array([12.05], np.float32), np.array([0.0], np.float32), np.array([MZ[11]], np.float32),
         np.array([11], np.int32))
    x, y, z, m, _ = assemble([A, B, S], shuffle_seed=9)
    cases.append((x, y, z, m))
    jit = np.where(np.arange(20) % 2 == 0, 0.003, -0.003)
    cases.append(line_hits(9.0, 0.0, 0.002, 0.0, range(5, 25), jitter=(np.zeros(20), jit)))
    # ties and conflicts decided by the keys: overlapping tracklets (smaller
    # chi2, then smaller key), following and seeding ties at bitwise-equal scatter
    for build in (lambda: tracklet_conflict(False), lambda: tracklet_conflict(True), following_tie,
                  seeding_tie, seeding_tie_third):
        cases.append(build()[:4])
    xs, ys, zs, ms, offs = [], [], [], [], [0]
    for (x, y, z, m) in cases:
        xs.append(x); ys.append(y); zs.append(z); ms.append(m); offs.append(offs[-1] + len(x))
    ev = synth.Events(np.concatenate(xs), np.concatenate(ys), np.concatenate(zs),
                      np.concatenate(ms).astype(np.int32), np.array(offs, np.int32),
                      np.zeros(offs[-1], np.int32), 0, MZ)
    o = oracle_of(ev)
    assert_same(run_gpu(sbt, handle, ev, False), o)
    assert_same(run_gpu(sbt, handle, ev, True), o)


def test_edge_cases_empty_and_degenerate(sbt, handle):
    # empty batch
    ev = synth.Events(*(np.zeros(0, np.float32),) * 3, np.zeros(0, np.int32), np.zeros(1, np.int32),
                      np.zeros(0, np.int32), 0, MZ)
    for b in (False, True):
        g = run_gpu(sbt, handle, ev, b)
        assert g["counts"][0] == 0 and g["counts"][1] == 0
    # zero-hit events between real ones, and hits on one module only
    base = synth.make_events(2, 5, workers=1)
    lo, hi = base.event_offsets[1], base.event_offsets[2]
    one_mod = np.full(7, 3, np.int32)
    x = np.concatenate([base.x[lo:hi], np.linspace(6, 9, 7, dtype=np.float32)])
    y = np.concatenate([base.y[lo:hi], np.linspace(6, 9, 7, dtype=np.float32)])
    z = np.concatenate([base.z[lo:hi], np.full(7, MZ[3], np.float32)])
    m = np.concatenate([base.module[lo:hi], one_mod])
    n1 = hi - lo
    offs = np.array([0, 0, n1, n1, n1 + 7, n1 + 7], np.int32)
    ev = synth.Events(x, y, z, m, offs, np.zeros(len(x), np.int32), 0, MZ)
    o = oracle_of(ev)
    for b in (False, True):
        assert_same(run_gpu(sbt, handle, ev, b), o)


def test_bad_module_and_oversize_events_are_reported(sbt):
    ev = synth.make_events(2, 6, workers=1)
    m = ev.module.copy()
    lo = ev.event_offsets[2]
    m[lo + 3] = 52                      # event 2: module id out of range
    sizes = np.diff(ev.event_offsets)
    big = int(np.argmax(sizes))
    h = sbt.sbt_create(MZ, sbt.default_config(max_hits_per_event=int(sizes[big]) - 1, **CFG))
    try:
        bad = synth.Events(ev.x, ev.y, ev.z, m, ev.event_offsets, ev.mc, 0, MZ)
        for b in (False, True):
            g = run_gpu(sbt, h, bad, b)
            st = g["event_status"]
            assert st[2] == sbt.SBT_ERR_ARG
            if big != 2:
                assert st[big] == sbt.SBT_ERR_CAPACITY
            assert g["counts"][3] == (st != 0).sum()
            # the other events are untouched
            ok = [e for e in range(ev.n_events) if st[e] == 0]
            for e in ok:
                lo_, hi_ = ev.event_offsets[e], ev.event_offsets[e + 1]
                one = oracle.event(ev.x[lo_:hi_], ev.y[lo_:hi_], ev.z[lo_:hi_], m[lo_:hi_], MZ,
                                   oracle.config(**CFG))
                t0, t1 = g["track_offsets"][e], g["track_offsets"][e + 1]
                assert t1 - t0 == one.n_tracks
                hs = g["track_hits"][g["hit_offsets"][t0]:g["hit_offsets"][t1]] - lo_
                assert np.array_equal(hs, one.track_hits)
            for e in range(ev.n_events):
                if st[e] != 0:
                    assert g["track_offsets"][e] == g["track_offsets"][e + 1]
    finally:
        h.close()


def test_forming_track_overflow_fails_only_that_event(sbt):
    ev = synth.make_events(2, 20, workers=1)
    # the oracle's peak of alive forming tracks per event bounds the GPU's
    # (which drops dead 3-hit tracks earlier); a cap between the events' peaks
    # makes some events overflow and leaves others untouched
    peaks = oracle_of(ev).stats[:, 4]
    cap = int(np.percentile(peaks, 30))
    h = sbt.sbt_create(MZ, sbt.default_config(max_forming_tracks=cap, **CFG))
    try:
        for b in (False, True):
            g = run_gpu(sbt, h, ev, b)
            st = g["event_status"]
            assert (st == sbt.SBT_ERR_CAPACITY).any() and (st == 0).any()
            assert set(np.unique(st)) <= {0, sbt.SBT_ERR_CAPACITY}
            for e in np.nonzero(st == 0)[0]:
                lo, hi = ev.event_offsets[e], ev.event_offsets[e + 1]
                one = oracle.event(ev.x[lo:hi], ev.y[lo:hi], ev.z[lo:hi], ev.module[lo:hi], MZ,
                                   oracle.config(**CFG))
                t0, t1 = g["track_offsets"][e], g["track_offsets"][e + 1]
                assert np.array_equal(g["track_hits"][g["hit_offsets"][t0]:g["hit_offsets"][t1]] - lo,
                                      one.track_hits)
    finally:
        h.close()


def test_host_entry_large_batch_schedule_equals_device_path(sbt):
    """From 60000 events on, the host entry point uses its thirteen-chunk
    schedule; 64000 small events (one vertex, Poisson(6) tracks) go through
    it and must give the one-call device path's result."""
    ev = synth.generate(synth.Recipe(n_events=64000, pv_mode="fixed", pv_mean=1, tracks_per_pv=6.0, seed=5),
                        workers=1)
    h = sbt.sbt_create(ev.module_z, sbt.default_config(**CFG))
    try:
        g = sbt.sbt_reconstruct_batched(h, *to_dev(ev)).compact()
        pin = lambda a: torch.from_numpy(a).pin_memory()
        out = sbt.sbt_reconstruct_host(h, pin(ev.x), pin(ev.y), pin(ev.z), pin(ev.module),
                                       pin(ev.event_offsets))
        assert h.last_launch_count() == 13 * 7
    finally:
        h.close()
    assert (g["event_status"] == 0).all() and g["counts"][0] > 100000
    c = out.compact()
    for k in ("track_offsets", "hit_offsets", "track_hits", "ndof", "event_status"):
        assert np.array_equal(c[k], g[k]), k
    assert np.array_equal(c["params"].view(np.uint32), g["params"].view(np.uint32))
    assert np.array_equal(c["chi2"].view(np.uint32), g["chi2"].view(np.uint32))


def test_output_capacity_overflow_is_reported(sbt, handle):
    ev = synth.make_events(2, 10, workers=1)
    x, y, z, m, off = to_dev(ev)
    o = oracle_of(ev)
    out = sbt.TrackOutput.allocate(ev.n_events, ev.n_hits, cap_tracks=o.n_tracks - 1)
    sbt.sbt_reconstruct(handle, x, y, z, m, off, out=out)
    torch.cuda.synchronize()
    c = out.counts.cpu().numpy()
    assert c[2] == sbt.SBT_ERR_CAPACITY and c[0] == o.n_tracks and c[1] == len(o.track_hits)


def test_output_capacity_overflow_writes_the_fitting_events_only(sbt, handle):
    """With too small a track capacity, the events that fit (a prefix of the
    batch) get their tracks, hit lists and fits, identical to a run with room
    to spare, and nothing is written past them."""
    ev = synth.make_events(2, 10, workers=1)
    dev = to_dev(ev)
    full = sbt.sbt_reconstruct(handle, *dev).compact()
    per_event = np.diff(full["track_offsets"])
    assert per_event[-1] > 0
    cap = int(full["counts"][0]) - 1                       # the last event does not fit
    tw = int(full["track_offsets"][-2])                    # tracks of the events before it
    hw = int(full["hit_offsets"][tw])
    out = sbt.TrackOutput.allocate(ev.n_events, ev.n_hits, cap_tracks=cap)
    for a in (out.hit_offsets, out.track_hits, out.ndof):
        a.fill_(-7)
    for a in (out.params, out.chi2):
        a.fill_(-7.0)
    sbt.sbt_reconstruct(handle, *dev, out=out)
    torch.cuda.synchronize()
    c = out.counts.cpu().numpy()
    assert c[2] == sbt.SBT_ERR_CAPACITY and c[0] == full["counts"][0]
    ho, th = out.hit_offsets.cpu().numpy(), out.track_hits.cpu().numpy()
    par, chi, nd = out.params.cpu().numpy(), out.chi2.cpu().numpy(), out.ndof.cpu().numpy()
    assert np.array_equal(ho[:tw], full["hit_offsets"][:tw]) and (ho[tw:] == -7).all()
    assert np.array_equal(th[:hw], full["track_hits"][:hw]) and (th[hw:] == -7).all()
    assert np.array_equal(par[:4 * tw].view(np.uint32), full["params"][:tw].reshape(-1).view(np.uint32))
    assert (par[4 * tw:] == -7.0).all()
    assert np.array_equal(chi[:tw].view(np.uint32), full["chi2"][:tw].view(np.uint32)) and (chi[tw:] == -7.0).all()
    assert np.array_equal(nd[:tw], full["ndof"][:tw]) and (nd[tw:] == -7).all()


def test_repeat_runs_are_identical(sbt, handle):
    ev = synth.make_events(2, 200, workers=1)
    a = run_gpu(sbt, handle, ev, True)
    b = run_gpu(sbt, handle, ev, True)
    c = run_gpu(sbt, handle, ev, False)
    for k in a:
        assert np.array_equal(a[k], b[k]) and np.array_equal(a[k], c[k])


def test_host_entry_point_matches_device(sbt, handle):
    ev = synth.make_events(2, 150, workers=1)
    pin = lambda a: torch.from_numpy(a).pin_memory()
    out = sbt.sbt_reconstruct_host(handle, pin(ev.x), pin(ev.y), pin(ev.z), pin(ev.module),
                                   pin(ev.event_offsets))
    T, H = int(out.counts[0]), int(out.counts[1])
    o = oracle_of(ev)
    assert T == o.n_tracks and H == len(o.track_hits)
    assert np.array_equal(out.track_offsets.numpy(), o.track_offsets)
    assert np.array_equal(out.hit_offsets[:T + 1].numpy(), o.hit_offsets)
    assert np.array_equal(out.track_hits[:H].numpy(), o.track_hits)
    assert np.array_equal(out.params[:4 * T].numpy().reshape(T, 4), o.params)


def test_host_entry_point_chunked_matches_device(sbt):
    """Above 12500 events the host entry point cuts the batch into chunks of
    uneven size (uploads, reconstruction and downloads overlapped); the result
    must equal the one-call device path, hit indices and offsets global."""
    ev = synth.make_events(1, 20000, workers=1)
    h = sbt.sbt_create(ev.module_z, sbt.default_config(**CFG))
    try:
        d = sbt.sbt_reconstruct_batched(h, *to_dev(ev))
        torch.cuda.synchronize()
        g = d.compact()
        pin = lambda a: torch.from_numpy(a).pin_memory()
        out = sbt.sbt_reconstruct_host(h, pin(ev.x), pin(ev.y), pin(ev.z), pin(ev.module),
                                       pin(ev.event_offsets))
    finally:
        h.close()
    T, H = int(out.counts[0]), int(out.counts[1])
    assert T == len(g["ndof"]) and H == len(g["track_hits"])
    assert np.array_equal(out.event_status.numpy(), g["event_status"])
    assert np.array_equal(out.track_offsets.numpy(), g["track_offsets"])
    assert np.array_equal(out.hit_offsets[:T + 1].numpy(), g["hit_offsets"])
    assert np.array_equal(out.track_hits[:H].numpy(), g["track_hits"])
    assert np.array_equal(out.params[:4 * T].numpy().view(np.uint32), g["params"].reshape(-1).view(np.uint32))
    assert np.array_equal(out.chi2[:T].numpy().view(np.uint32), g["chi2"].view(np.uint32))
    assert np.array_equal(out.ndof[:T].numpy(), g["ndof"])
    # and a sample of events against the oracle
    o = oracle.reconstruct(ev.x[:ev.event_offsets[200]], ev.y[:ev.event_offsets[200]],
                           ev.z[:ev.event_offsets[200]], ev.module[:ev.event_offsets[200]],
                           ev.event_offsets[:201], ev.module_z, oracle.config(**CFG))
    assert np.array_equal(out.track_offsets.numpy()[:201], o.track_offsets)
    assert np.array_equal(out.track_hits[:len(o.track_hits)].numpy(), o.track_hits)


def test_autotune_keeps_results(sbt):
    ev = synth.make_events(2, 300, workers=1)
    h = sbt.sbt_create(MZ, sbt.default_config(**CFG))
    try:
        chosen, per_sm = sbt.sbt_autotune(h, *to_dev(ev))
        assert chosen in (64, 128, 256) and per_sm >= 1
        assert sbt.sbt_tuned_shape(h) == (chosen, per_sm)
        o = oracle_of(ev)
        assert_same(run_gpu(sbt, h, ev, True), o)
        # any launch shape gives the same tracks
        for shape in ((64, 3), (128, 1), (256, 0)):
            sbt.sbt_set_launch_shape(h, *shape)
            assert_same(run_gpu(sbt, h, ev, True), o)
        with pytest.raises(sbt.SbtError):
            sbt.sbt_set_launch_shape(h, 96, 4)
    finally:
        h.close()


@pytest.mark.parametrize("fp16", [0, 1])
def test_maximum_event_size_bit_exact(sbt, fp16):
    """An event of exactly the largest supported size (16384 hits: the sort's
    shared-memory buffers and the 16-bit hit positions of the search) between
    two ordinary events, through the plain, batched and host entry points; an
    event one hit larger is reported as SBT_ERR_CAPACITY, the others kept."""
    base = synth.make_events(2, 14, seed=4, workers=1)
    o = base.event_offsets
    big = slice(int(o[1]), int(o[1]) + 16384)          # events 1.. merged, cut at 16384 hits
    assert o[13] - o[1] > 16384
    parts = [slice(int(o[0]), int(o[1])), big, slice(int(o[13]), int(o[14]))]
    cat = lambda a: np.concatenate([a[p] for p in parts])
    sizes = [p.stop - p.start for p in parts]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    ev = synth.Events(cat(base.x), cat(base.y), cat(base.z), cat(base.module), offs,
                      cat(base.mc), 0, base.module_z)
    h = sbt.sbt_create(ev.module_z, sbt.default_config(max_hits_per_event=16384, fp16_hits=fp16, **CFG))
    try:
        ref = oracle.reconstruct(ev.x, ev.y, ev.z, ev.module, ev.event_offsets, ev.module_z,
                                 oracle.config(**CFG), fp16_hits=bool(fp16))
        assert ref.status[1] == 0 and ref.n_tracks > 0
        assert_same(run_gpu(sbt, h, ev, False), ref)
        assert_same(run_gpu(sbt, h, ev, True), ref)
        host = [torch.from_numpy(a) for a in (ev.x, ev.y, ev.z, ev.module, ev.event_offsets)]
        assert_same(sbt.sbt_reconstruct_host(h, *host).compact(), ref)
        # one more hit in the middle event: that event alone is refused
        extra = slice(big.start, big.stop + 1)
        parts2 = [parts[0], extra, parts[2]]
        cat2 = lambda a: np.concatenate([a[p] for p in parts2])
        offs2 = np.array([0, sizes[0], sizes[0] + 16385, sizes[0] + 16385 + sizes[2]], np.int32)
        ev2 = synth.Events(cat2(base.x), cat2(base.y), cat2(base.z), cat2(base.module), offs2,
                           cat2(base.mc), 0, base.module_z)
        for b in (False, True):
            g = run_gpu(sbt, h, ev2, b)
            assert list(g["event_status"]) == [0, sbt.SBT_ERR_CAPACITY, 0]
            assert g["track_offsets"][1] == g["track_offsets"][2]
            assert g["track_offsets"][1] == ref.track_offsets[1]
            assert g["track_offsets"][3] - g["track_offsets"][2] == ref.track_offsets[3] - ref.track_offsets[2]
    finally:
        h.close()


@pytest.mark.parametrize("config,n,fp16", [(2, 150, 0), (3, 60, 0), (2, 80, 1)])
def test_module_pairs_bit_exact(sbt, config, n, fp16):
    """Module-pair geometry (two one-sided planes per module, the x < 0 plane
    at module_z2): plain, batched and host entry points equal the oracle's
    pair reading, fp32 and fp16 storage."""
    ev = synth.make_events(config, n, pairs=True)
    h = sbt.sbt_create(ev.module_z, sbt.default_config(fp16_hits=fp16, **CFG), module_z2=ev.module_z2)
    try:
        o = oracle.reconstruct(ev.x, ev.y, ev.z, ev.module, ev.event_offsets, ev.module_z,
                               oracle.config(**CFG), fp16_hits=bool(fp16), module_z2=ev.module_z2)
        assert o.n_tracks > 0
        assert_same(run_gpu(sbt, h, ev, False), o)
        assert_same(run_gpu(sbt, h, ev, True), o)
        host = [torch.from_numpy(a) for a in (ev.x, ev.y, ev.z, ev.module, ev.event_offsets)]
        assert_same(sbt.sbt_reconstruct_host(h, *host).compact(), o)
        # the same hits on a single-plane handle follow the single-plane reading
        hs = sbt.sbt_create(ev.module_z, sbt.default_config(fp16_hits=fp16, **CFG))
        try:
            o1 = oracle.reconstruct(ev.x, ev.y, ev.z, ev.module, ev.event_offsets, ev.module_z,
                                    oracle.config(**CFG), fp16_hits=bool(fp16))
            assert_same(run_gpu(sbt, hs, ev, True), o1)
        finally:
            hs.close()
    finally:
        h.close()


def test_module_pairs_adjoint_is_refused(sbt):
    ev = synth.make_events(2, 4, pairs=True, workers=1)
    h = sbt.sbt_create(ev.module_z, sbt.default_config(**CFG), module_z2=ev.module_z2)
    try:
        dev = to_dev(ev)
        out = sbt.sbt_reconstruct_batched(h, *dev).compact()
        ho = torch.from_numpy(out["hit_offsets"]).cuda()
        th = torch.from_numpy(out["track_hits"]).cuda()
        align = torch.zeros(ev.module_z.shape[0], 6, dtype=torch.float64, device="cuda")
        with pytest.raises(sbt.SbtError):
            sbt.sbt_fit_adjoint(h, dev[0], dev[1], dev[2], dev[3], ho, th, align)
    finally:
        h.close()


@pytest.mark.parametrize("cfg_seed", range(4))
def test_crowded_tiny_events_bit_exact(sbt, cfg_seed):
    # the crowded tiny events of the oracle's whole-loop pin (overlapping
    # seeds, contended extensions, overlapping tracklets), 200 per batch on
    # eight planes, under four random configurations
    from tests.test_oracle_loop import random_cfg, tiny_event
    rng = np.random.default_rng(77 + cfg_seed)
    module_z = (200.0 - 20.0 * np.arange(8)).astype(np.float32)
    cfg = random_cfg(rng)
    parts = [tiny_event(rng, module_z) for _ in range(200)]
    offs = np.concatenate([[0], np.cumsum([len(p[0]) for p in parts])]).astype(np.int32)
    ev = synth.Events(*(np.concatenate([p[k] for p in parts]) for k in range(3)),
                      np.concatenate([p[3] for p in parts]).astype(np.int32), offs,
                      np.zeros(offs[-1], np.int32), 0, module_z)
    o = oracle.reconstruct(ev.x, ev.y, ev.z, ev.module, ev.event_offsets, module_z, oracle.config(**cfg))
    assert o.n_tracks > 200
    h = sbt.sbt_create(module_z, sbt.default_config(**cfg))
    try:
        for batched in (False, True):
            assert_same(run_gpu(sbt, h, ev, batched), o)
    finally:
        h.close()


def test_event_ranges_outside_the_hits_are_reported(sbt, handle):
    # events whose hit range ends past n_hits get SBT_ERR_ARG on the device
    # and no tracks; the others are reconstructed as usual.  The hit arrays
    # passed are views of the whole batch, so memory behind n_hits exists and
    # a missing check could not read outside an allocation.
    ev = synth.make_events(2, 6, workers=1)
    off = ev.event_offsets
    H = int(off[4]) + 10                       # event 4 ends past H, event 5 lies beyond it
    full = to_dev(ev)
    dev = [a[:H] for a in full[:4]] + [full[4]]
    sub = ev.subset(0, 4)
    o = oracle_of(sub)
    for fn in (sbt.sbt_reconstruct, sbt.sbt_reconstruct_batched):
        g = fn(handle, *dev).compact()
        torch.cuda.synchronize()
        assert list(g["event_status"]) == [0, 0, 0, 0, 1, 1]
        assert int(g["counts"][3]) == 2 and int(g["counts"][2]) == 0
        t4 = int(g["track_offsets"][4])
        assert t4 == o.n_tracks and int(g["track_offsets"][6]) == t4
        assert np.array_equal(g["hit_offsets"][:t4 + 1], o.hit_offsets)
        assert np.array_equal(g["track_hits"][:int(o.hit_offsets[-1])], o.track_hits)
        assert np.array_equal(g["params"][:t4].view(np.uint32), o.params.view(np.uint32))
    # the host entry point sees the offsets on the host and refuses the call
    host = [torch.from_numpy(np.ascontiguousarray(a[:H])) for a in (ev.x, ev.y, ev.z, ev.module)]
    out = sbt.TrackOutput.allocate(6, H, pin_memory=True)
    with pytest.raises(sbt.SbtError, match="non-decreasing"):
        sbt.sbt_reconstruct_host(handle, *host, torch.from_numpy(off), out=out)
