"""Exhaustive enumeration of one seeding step on tiny events (readings R3, R4 of
section "Track seeding and track following")."""
import numpy as np
import pytest

import oracle
from paper_2207_03936_gb300 import synth

MZ = synth.module_z_traversal()


def circ(u, v):
    d = (int(u) - int(v)) % 65536
    return min(d, 65536 - d)


def brute_seeds(x, y, z, m, s, K, S, flags):
    """Every (a, c, b) is enumerated; the candidate set of a middle hit is the
    set of unflagged hits on module s whose distance does not exceed the K-th
    smallest; the kept triplet minimises (scatter, a, b) under S."""
    n = len(x)
    ph = oracle.phi16(x, y)
    order = np.lexsort((np.arange(n), ph, m))
    sx, sy, sz, sm, sp = x[order], y[order], z[order], m[order], ph[order]
    fl = flags
    pos = np.arange(n)
    out = []
    zi = np.float32(MZ[s + 2])
    for c in pos[sm == s + 1]:
        if fl[c]:
            continue
        A = [a for a in pos[sm == s] if not fl[a]]
        if len(A) > K:
            dk = sorted(circ(sp[a], sp[c]) for a in A)[K - 1]
            A = [a for a in A if circ(sp[a], sp[c]) <= dk]
        best = None
        for a in A:
            dz = np.float32(sz[c] - sz[a])
            tz = np.float32(np.float32(zi - sz[c]) / dz)
            xp = np.float32(sx[c] + np.float32(np.float32(sx[c] - sx[a]) * tz))
            yp = np.float32(sy[c] + np.float32(np.float32(sy[c] - sy[a]) * tz))
            for b in pos[sm == s + 2]:
                if fl[b]:
                    continue
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


def tiny_event(rng, s, n_per, n_lines):
    xs, ys, zs, ms = [], [], [], []
    for k in range(3):
        mod = s + k
        r = np.sqrt(rng.uniform(5.1 ** 2, 42.0 ** 2, n_per))
        a = rng.uniform(0, 2 * np.pi, n_per)
        xs.append(r * np.cos(a)); ys.append(r * np.sin(a))
        zs.append(np.full(n_per, MZ[mod])); ms.append(np.full(n_per, mod))
    for _ in range(n_lines):
        x0, y0 = rng.uniform(-30, 30, 2)
        tx, ty = rng.normal(0, 0.01, 2)
        for k in range(3):
            mod = s + k
            zz = float(MZ[mod]) - float(MZ[s])
            xs.append([x0 + tx * zz + rng.normal(0, 0.05)])
            ys.append([y0 + ty * zz + rng.normal(0, 0.05)])
            zs.append([MZ[mod]]); ms.append([mod])
    x = np.concatenate(xs).astype(np.float32)
    y = np.concatenate(ys).astype(np.float32)
    z = np.concatenate(zs).astype(np.float32)
    m = np.concatenate(ms).astype(np.int32)
    p = rng.permutation(len(x))
    return x[p], y[p], z[p], m[p]


@pytest.mark.parametrize("seed", range(12))
def test_seed_step_equals_enumeration(seed):
    rng = np.random.default_rng(100 + seed)
    s = int(rng.integers(0, 49))
    K = int(rng.integers(1, 6))
    S = float(rng.choice([0.04, 0.5, 5.0]))
    x, y, z, m = tiny_event(rng, s, int(rng.integers(2, 12)), int(rng.integers(0, 5)))
    flags = (rng.uniform(size=len(x)) < 0.2).astype(np.uint8)
    cfg = oracle.config(k_doublets=K, max_scatter_seed=S)
    got = [tuple(int(v) for v in r) for r in oracle.seed_step(x, y, z, m, MZ, s, cfg, flags)]
    assert got == brute_seeds(x, y, z, m, s, K, S, flags)


def test_k_nearest_keeps_all_ties_at_boundary():
    # middle hit at phi16 ~ p; four outer hits at +-d and +-2d; K = 3: the
    # third smallest distance is 2d, so both hits at 2d are candidates and
    # the one giving the best triplet wins even though it is the fourth nearest
    # by sorted position.
    s = 20
    r = 20.0
    ang = 0.5
    dphi = 200 / 10430.378
    outer = [ang - dphi, ang + dphi, ang - 2 * dphi, ang + 2 * dphi]
    x = [r * np.cos(a) for a in outer]
    y = [r * np.sin(a) for a in outer]
    m = [s] * 4
    # middle hit
    x.append(r * np.cos(ang)); y.append(r * np.sin(ang)); m.append(s + 1)
    # third hit on the continuation of outer[2] -> middle (a straight line)
    xa, ya = x[2], y[2]
    xc, yc = x[4], y[4]
    x.append(2 * xc - xa); y.append(2 * yc - ya); m.append(s + 2)
    x = np.array(x, np.float32); y = np.array(y, np.float32)
    m = np.array(m, np.int32); z = MZ[m]
    ph = oracle.phi16(x, y)
    d = [circ(ph[i], ph[4]) for i in range(4)]
    assert d[0] == d[1] and d[2] == d[3] and d[2] > d[0]
    cfg = oracle.config(k_doublets=3, max_scatter_seed=0.04)
    got = oracle.seed_step(x, y, z, m, MZ, s, cfg)
    assert len(got) == 1
    perm, _, _ = oracle.sort_event(x, y, m, 52)
    a, c, b = (int(perm[v]) for v in got[0])
    assert (a, c, b) == (2, 4, 5)
    # with K = 2 the hit at 2d is not a candidate: no compatible triplet
    assert len(oracle.seed_step(x, y, z, m, MZ, s, oracle.config(k_doublets=2))) == 0
