"""Module-pair geometry (reading R10): each module is a pair of one-sided
planes, hits with x >= 0 on the plane at module_z and hits with x < 0 on the
plane at module_z2, and every extrapolation targets the plane of the hit it is
compared with.  Pinned by exhaustive enumeration of seeding steps, by the
reduction to single planes when both planes coincide, by straight lines that
must be found whole (and are not when the planes are swapped), by the track
invariants and by the physics indicators against truth."""
import numpy as np
import pytest

import oracle
from paper_2207_03936_gb300 import synth, validation
from tests.test_oracle_invariants import CFG, check_invariants
from tests.test_oracle_seeding import circ

ZP = synth.module_z_ascending().reshape(synth.N_PAIRS, 2)[::-1].astype(np.float32)
MZ1, MZ2 = ZP[:, 0].copy(), ZP[:, 1].copy()    # x >= 0 plane, x < 0 plane; traversal order


def plane(m, x):
    return MZ2[m] if x < 0 else MZ1[m]


def brute_seeds_pairs(x, y, z, m, s, K, S, flags):
    """Every (a, c, b): candidates of a middle hit as in the single-plane
    enumeration; the extrapolation of (a, c) goes to the plane of each b."""
    n = len(x)
    ph = oracle.phi16(x, y)
    order = np.lexsort((np.arange(n), ph, m))
    sx, sy, sz, sm, sp = x[order], y[order], z[order], m[order], ph[order]
    pos = np.arange(n)
    out = []
    for c in pos[sm == s + 1]:
        if flags[c]:
            continue
        A = [a for a in pos[sm == s] if not flags[a]]
        if len(A) > K:
            dk = sorted(circ(sp[a], sp[c]) for a in A)[K - 1]
            A = [a for a in A if circ(sp[a], sp[c]) <= dk]
        best = None
        for a in A:
            for b in pos[sm == s + 2]:
                if flags[b]:
                    continue
                zi = np.float32(plane(s + 2, sx[b]))
                dz = np.float32(sz[c] - sz[a])
                tz = np.float32(np.float32(zi - sz[c]) / dz)
                xp = np.float32(sx[c] + np.float32(np.float32(sx[c] - sx[a]) * tz))
                yp = np.float32(sy[c] + np.float32(np.float32(sy[c] - sy[a]) * tz))
                dx = np.float32(sx[b] - xp)
                dy = np.float32(sy[b] - yp)
                sc = np.float32(np.float32(dx * dx) + np.float32(dy * dy))
                if sc < np.float32(S):
                    key = (float(sc), int(a), int(b))
                    if best is None or key < best:
                        best = key
        if best is not None:
            out.append((best[1], int(c), best[2]))
    return out


def tiny_pair_event(rng, s, n_per, n_lines):
    xs, ys, ms = [], [], []
    for k in range(3):
        r = np.sqrt(rng.uniform(5.1 ** 2, 42.0 ** 2, n_per))
        a = rng.uniform(0, 2 * np.pi, n_per)
        xs.append(r * np.cos(a)); ys.append(r * np.sin(a)); ms.append(np.full(n_per, s + k))
    for _ in range(n_lines):
        x0, y0 = rng.uniform(-30, 30, 2)
        tx, ty = rng.normal(0, 0.02, 2)
        for k in range(3):
            # the line's crossing of the plane on its own side (fixed point: x sign)
            zz = float(MZ1[s + k]) - float(MZ1[s])
            if x0 + tx * zz < 0:
                zz = float(MZ2[s + k]) - float(MZ1[s])
            xs.append([x0 + tx * zz + rng.normal(0, 0.05)])
            ys.append([y0 + ty * zz + rng.normal(0, 0.05)])
            ms.append([s + k])
    x = np.concatenate(xs).astype(np.float32)
    y = np.concatenate(ys).astype(np.float32)
    m = np.concatenate(ms).astype(np.int32)
    x[x == 0] = np.float32(1e-3)
    z = np.where(x < 0, MZ2[m], MZ1[m]).astype(np.float32)
    p = rng.permutation(len(x))
    return x[p], y[p], z[p], m[p]


@pytest.mark.parametrize("seed", range(10))
def test_pair_seed_step_equals_enumeration(seed):
    rng = np.random.default_rng(700 + seed)
    s = int(rng.integers(0, synth.N_PAIRS - 2))
    K = int(rng.integers(1, 6))
    S = float(rng.choice([0.04, 0.5, 5.0]))
    x, y, z, m = tiny_pair_event(rng, s, int(rng.integers(2, 12)), int(rng.integers(0, 5)))
    flags = (rng.uniform(size=len(x)) < 0.2).astype(np.uint8)
    cfg = oracle.config(k_doublets=K, max_scatter_seed=S)
    got = [tuple(int(v) for v in r)
           for r in oracle.seed_step(x, y, z, m, MZ1, s, cfg, flags, module_z2=MZ2)]
    assert got == brute_seeds_pairs(x, y, z, m, s, K, S, flags)


def test_coinciding_planes_reduce_to_single_planes():
    ev = synth.make_events(2, 60, workers=1)
    a = oracle.reconstruct(ev.x, ev.y, ev.z, ev.module, ev.event_offsets, ev.module_z,
                           oracle.config(**CFG))
    b = oracle.reconstruct(ev.x, ev.y, ev.z, ev.module, ev.event_offsets, ev.module_z,
                           oracle.config(**CFG), module_z2=ev.module_z)
    for f in ("track_offsets", "hit_offsets", "track_hits", "ndof", "status"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
    assert np.array_equal(a.params.view(np.uint32), b.params.view(np.uint32))
    assert np.array_equal(a.chi2.view(np.uint32), b.chi2.view(np.uint32))


def two_sided_lines():
    """Two straight lines through all 26 pairs, one on each side of the beam;
    each crosses only the planes of its side."""
    lines = [(20.0, 3.0, 0.02, 0.005), (-18.0, -4.0, -0.02, 0.01)]
    xs, ys, zs, ms, groups = [], [], [], [], []
    n = 0
    for (x0, y0, tx, ty) in lines:
        mods = np.arange(synth.N_PAIRS, dtype=np.int32)
        z = (MZ1 if x0 > 0 else MZ2)[mods]
        xs.append((x0 + tx * z.astype(np.float64)).astype(np.float32))
        ys.append((y0 + ty * z.astype(np.float64)).astype(np.float32))
        zs.append(z); ms.append(mods)
        groups.append(np.arange(n, n + len(mods))); n += len(mods)
    x, y, z, m = (np.concatenate(a) for a in (xs, ys, zs, ms))
    assert ((x > 0)[:26].all() and (x < 0)[26:].all())
    return x, y, z, m, groups, lines


def test_straight_lines_on_both_sides_found_whole():
    x, y, z, m, groups, lines = two_sided_lines()
    r = oracle.event(x, y, z, m, MZ1, oracle.config(**CFG), module_z2=MZ2)
    assert r.n_tracks == 2
    found = [r.track_hits[r.hit_offsets[t]:r.hit_offsets[t + 1]] for t in range(2)]
    assert sorted(map(tuple, found)) == sorted(tuple(g) for g in groups)
    for t in range(2):
        g = found[t]
        x0, y0, tx, ty = lines[0] if g[0] < 26 else lines[1]
        assert np.allclose(r.params[t], [x0, y0, tx, ty], rtol=1e-4, atol=2e-4)
        assert r.chi2[t] < 1e-2
    # the same hits with the two planes of every pair swapped: each line is
    # extrapolated to the wrong plane (0.4 mm off) and no track is found whole
    w = oracle.event(x, y, z, m, MZ2, oracle.config(**CFG), module_z2=MZ1)
    assert all(w.hit_offsets[t + 1] - w.hit_offsets[t] < 26 for t in range(w.n_tracks))


@pytest.mark.parametrize("config,n", [(1, None), (2, 120), (3, 30)])
def test_pair_invariants(config, n):
    ev = synth.make_events(config, n, workers=1, pairs=True)
    res = oracle.reconstruct(ev.x, ev.y, ev.z, ev.module, ev.event_offsets, ev.module_z,
                             oracle.config(**CFG), module_z2=ev.module_z2)
    assert (res.status == 0).all()
    check_invariants(ev, res, CFG)


@pytest.mark.parametrize("config", [1, 2])
def test_pair_physics_indicators_against_truth(config):
    # thresholds fixed once from the first oracle run on the pair workloads
    ev = synth.make_events(config, workers=1, pairs=True)
    res = oracle.reconstruct(ev.x, ev.y, ev.z, ev.module, ev.event_offsets, ev.module_z,
                             oracle.config(**CFG), module_z2=ev.module_z2)
    ind = validation.indicators(res.hit_offsets, res.track_hits, ev.mc, ev.n_particles)
    assert ind["efficiency"] >= 0.99
    assert ind["fake_fraction"] <= 0.005
    assert ind["clone_fraction"] <= 0.015
    assert ind["hit_purity"] >= 0.995
    assert ind["hit_efficiency"] >= 0.98


def test_generator_planes_match_hit_sides():
    ev = synth.make_events(2, 40, workers=1, pairs=True)
    assert ev.module_z.shape == (synth.N_PAIRS,) and ev.module.max() == synth.N_PAIRS - 1
    zt = np.where(ev.x < 0, ev.module_z2[ev.module], ev.module_z[ev.module])
    assert np.array_equal(zt, ev.z)
    assert (np.abs(ev.x) >= 1e-3).all()
