"""The whole seeding / following / claim / tracklet-filter loop of the oracle
against a second statement of it that enumerates everything (tests/brute_loop.py),
on tiny random events of at most eight modules crowded into a patch a
millimetre wide, so that seeds share hits, extensions contend for the same hit
and accepted tracklets overlap (section "Track seeding and track following",
section "Tracklet filter"; readings R3-R9)."""
import numpy as np
import pytest

import oracle
from tests import brute_loop


def tiny_event(rng, module_z=None):
    """A few straight segments (3 to M hits, random start module, small
    slopes, 20 um smearing, 10% missing hits) and a few noise hits per module,
    all within about 0.6 mm of one point of the annulus; module planes 14-26 mm
    apart in traversal order (descending z), or the given planes."""
    if module_z is None:
        M = int(rng.integers(4, 9))
        pitch = rng.uniform(14.0, 26.0, M - 1)
        module_z = (200.0 - np.concatenate([[0.0], np.cumsum(pitch)])).astype(np.float32)
    M = len(module_z)
    r0, a0 = rng.uniform(8.0, 30.0), rng.uniform(0, 2 * np.pi)
    cx, cy = r0 * np.cos(a0), r0 * np.sin(a0)
    xs, ys, ms = [], [], []
    for _ in range(int(rng.integers(2, 8))):
        m0 = int(rng.integers(0, M - 2))
        m1 = int(rng.integers(m0 + 3, M + 1))
        x0, y0 = cx + rng.uniform(-0.4, 0.4), cy + rng.uniform(-0.4, 0.4)
        tx, ty = rng.normal(0, 0.005, 2)
        for k in range(m0, m1):
            if rng.random() < 0.1:
                continue
            dz = float(module_z[m0] - module_z[k])
            xs.append(x0 + tx * dz + rng.normal(0, 0.02))
            ys.append(y0 + ty * dz + rng.normal(0, 0.02))
            ms.append(k)
    for k in range(M):
        for _ in range(int(rng.integers(0, 3))):
            xs.append(cx + rng.uniform(-0.6, 0.6))
            ys.append(cy + rng.uniform(-0.6, 0.6))
            ms.append(k)
    m = np.array(ms, np.int32)
    p = rng.permutation(len(m))
    x = np.array(xs, np.float32)[p]
    y = np.array(ys, np.float32)[p]
    m = m[p]
    return x, y, module_z[m].copy(), m, module_z


def random_cfg(rng):
    return dict(k_doublets=int(rng.choice([1, 2, 4])),
                max_scatter_seed=float(rng.choice([0.01, 0.04, 0.09])),
                max_scatter_follow=float(rng.choice([0.01, 0.04, 0.09])),
                max_chi2_tracklet=float(rng.choice([2.0, 20.0, 200.0])),
                hit_sigma=0.012)


def oracle_tracks(x, y, z, m, module_z, cfg, module_z2=None):
    r = oracle.event(x, y, z, m, module_z, oracle.config(**cfg), module_z2=module_z2)
    return [r.track_hits[r.hit_offsets[t]:r.hit_offsets[t + 1]].tolist() for t in range(r.n_tracks)]


@pytest.mark.parametrize("seed", range(60))
def test_oracle_equals_enumeration(seed):
    rng = np.random.default_rng(1000 + seed)
    x, y, z, m, module_z = tiny_event(rng)
    cfg = random_cfg(rng)
    assert oracle_tracks(x, y, z, m, module_z, cfg) == brute_loop.reconstruct(x, y, z, m, module_z, **cfg)


@pytest.mark.parametrize("seed", range(20))
def test_oracle_equals_enumeration_module_pairs(seed):
    # module pairs (R10): the second plane of each pair 3-9 mm downstream;
    # hits with x < 0 lie on it
    rng = np.random.default_rng(5000 + seed)
    x, y, z, m, module_z = tiny_event(rng)
    module_z2 = (module_z - rng.uniform(3.0, 9.0, len(module_z))).astype(np.float32)
    z = np.where(x < 0, module_z2[m], module_z[m]).astype(np.float32)
    cfg = random_cfg(rng)
    assert (oracle_tracks(x, y, z, m, module_z, cfg, module_z2)
            == brute_loop.reconstruct(x, y, z, m, module_z, module_z2=module_z2, **cfg))


def test_enumeration_events_exercise_the_conflicts():
    """The random events are crowded enough that the choices the pin is for
    arise often: extensions that lose a claim to a smaller key, and tracklets
    that pass the filter's cut but lose the claim round to an overlapping one."""
    lost_ext = lost_tl = tracks = 0
    for seed in range(60):
        rng = np.random.default_rng(1000 + seed)
        x, y, z, m, module_z = tiny_event(rng)
        cfg = random_cfg(rng)
        st = {}
        tracks += len(brute_loop.reconstruct(x, y, z, m, module_z, stats=st, **cfg))
        lost_ext += st["lost_extensions"]
        lost_tl += st["lost_tracklets"]
    assert tracks >= 100 and lost_ext >= 10 and lost_tl >= 10, (tracks, lost_ext, lost_tl)
