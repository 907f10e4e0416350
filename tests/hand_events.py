"""Hand-built events whose reconstruction is known by construction.

Each builder returns (x, y, z, module, expected) where expected is a list of
tracks, each a list of input hit indices in traversal order.  The geometry is
the 52-plane layout of the synthetic workloads.
"""
import numpy as np

from paper_2207_03936_gb300 import synth

MZ = synth.module_z_traversal()


def line_hits(x0, y0, tx, ty, modules, jitter=None):
    """Hits of the straight line x = x0 + tx z, y = y0 + ty z on the given modules."""
    modules = np.asarray(modules, dtype=np.int32)
    z = MZ[modules].astype(np.float64)
    x = x0 + tx * z
    y = y0 + ty * z
    if jitter is not None:
        x = x + jitter[0]
        y = y + jitter[1]
    return x.astype(np.float32), y.astype(np.float32), MZ[modules].copy(), modules


def assemble(parts, shuffle_seed=None):
    """Concatenate hit groups; optionally shuffle the input order.

    Returns (x, y, z, module, groups) where groups[i] are the input indices of
    part i in its original order.
    """
    xs, ys, zs, ms, groups = [], [], [], [], []
    n = 0
    for (x, y, z, m) in parts:
        xs.append(x); ys.append(y); zs.append(z); ms.append(m)
        groups.append(np.arange(n, n + len(x)))
        n += len(x)
    x, y, z, m = (np.concatenate(a) for a in (xs, ys, zs, ms))
    if shuffle_seed is not None:
        perm = np.random.default_rng(shuffle_seed).permutation(n)
        inv = np.empty(n, np.int64)
        inv[perm] = np.arange(n)
        x, y, z, m = x[perm], y[perm], z[perm], m[perm]
        groups = [inv[g] for g in groups]
    return x, y, z, m.astype(np.int32), groups


def single_track(missing=(), shuffle_seed=1):
    mods = [k for k in range(52) if k not in set(missing)]
    # a line that stays well inside the annulus over the full length
    part = line_hits(8.0, 5.0, 0.004, -0.003, mods)
    x, y, z, m, g = assemble([part], shuffle_seed)
    return x, y, z, m, g[0]


def tracklet_conflict(equal_chi2=False, shuffle_seed=3):
    """Two 3-hit tracklets on modules 30-32 that share their first hit A at
    (10, 0): seeds do not flag hits, so both middle hits on module 31 take A
    as their outer hit, and with nothing on modules 33 and 34 both tracks end
    as tracklets, unflagged and under the chi2 cut.  Track 1 runs below the x
    axis, track 2 is its mirror image in y above it; the last hit of each is
    moved by j1 (track 1) and j2 (track 2) towards the axis.  Track 2's middle
    hit has the smaller phi16 (just above zero; track 1's is just below 2^16),
    hence the smaller sorted position and track key.

    Returns (x, y, z, module, tracks) with tracks = [track 1, track 2] as
    input indices in traversal order."""
    mods = [30, 31, 32]
    z = MZ[mods].astype(np.float64)
    dz = z - z[0]
    j1, j2 = 0.01, (0.01 if equal_chi2 else 0.02)
    t1 = ([10.0 + 0.01 * d for d in dz], [0.005 * d for d in dz])
    t1[1][2] += j1
    t2 = ([10.0 + 0.01 * d for d in dz], [-0.005 * d for d in dz])
    t2[1][2] -= j2
    x = np.array(t1[0] + t2[0][1:], np.float32)
    y = np.array(t1[1] + t2[1][1:], np.float32)
    m = np.array(mods + mods[1:], np.int32)
    x, y, zz, m, g = assemble([(x, y, MZ[m].copy(), m)], shuffle_seed)
    idx = g[0]
    return x, y, zz, m, [[int(idx[0]), int(idx[1]), int(idx[2])], [int(idx[0]), int(idx[3]), int(idx[4])]]


def following_tie(shuffle_seed=4):
    """A straight track along the +x axis (y = 0 on every hit) over modules
    5-24 whose hit on module 15 is replaced by two hits at the predicted x and
    y = +0.05 and -0.05 mm: the following step to module 15 sees both at a
    bitwise-equal scatter.  The tie goes to the smaller sorted position, the
    hit at y = +0.05 (phi16 just above zero; the other is just below 2^16).

    Returns (x, y, z, module, track) with the expected track's input indices
    in traversal order."""
    mods = list(range(5, 25))
    x, y, z, m = line_hits(9.0, 0.0, 0.002, 0.0, mods)
    k = mods.index(15)
    x = np.concatenate([x, x[k:k + 1]])
    y = np.concatenate([y, np.float32([-0.05])])
    y[k] = np.float32(0.05)
    z = np.concatenate([z, z[k:k + 1]])
    m = np.concatenate([m, m[k:k + 1]])
    x, y, z, m, g = assemble([(x, y, z, m)], shuffle_seed)
    return x, y, z, m, [int(i) for i in g[0][:len(mods)]]


def seeding_tie(shuffle_seed=5):
    """One middle hit C at (10, 0) on module 31; two outer hits A1, A2 on
    module 30 at y = +0.2 and -0.2 mm (same x), and on module 32 the two hits
    B1, B2 that continue the lines A1-C and A2-C, each moved 0.01 mm back
    towards the axis, mirror images of each other in y.  The triplets
    (A1, C, B1) and (A2, C, B2) have bitwise-equal scatter; the tie goes to
    the smaller sorted position of the outer hit, A1 (phi16 just above zero).
    A second middle-hit tie, two third hits for one doublet, is covered by
    following_tie's mirror construction.

    Returns (x, y, z, module, tracklet) with the expected tracklet's input
    indices [A1, C, B1]."""
    mods = [30, 31, 32]
    zz = MZ[mods].astype(np.float64)
    xs = [10.0 + 0.004 * (v - zz[1]) for v in zz]
    tz = (zz[2] - zz[1]) / (zz[1] - zz[0])
    yb = -0.2 * tz
    ya = [0.2, -0.2]
    x = np.array([xs[0], xs[0], xs[1], xs[2], xs[2]], np.float32)
    y = np.array([ya[0], ya[1], 0.0, yb + 0.01, 0.0], np.float32)
    y[4] = -y[3]
    m = np.array([30, 30, 31, 32, 32], np.int32)
    x, y, z, m, g = assemble([(x, y, MZ[m].copy(), m)], shuffle_seed)
    idx = g[0]
    return x, y, z, m, [int(idx[0]), int(idx[2]), int(idx[3])]


def seeding_tie_third(shuffle_seed=6):
    """Outer hit A and middle hit C on the +x axis (modules 30, 31) and two
    hits on module 32 at the predicted x and y = +0.05 and -0.05 mm: one
    doublet, two third hits at bitwise-equal scatter.  The tie goes to the
    smaller sorted position, the hit at y = +0.05.

    Returns (x, y, z, module, tracklet) with the expected [A, C, B+]."""
    mods = [30, 31, 32]
    zz = MZ[mods].astype(np.float64)
    xs = [10.0 + 0.004 * (v - zz[1]) for v in zz]
    x = np.array([xs[0], xs[1], xs[2], xs[2]], np.float32)
    y = np.array([0.0, 0.0, 0.05, -0.05], np.float32)
    m = np.array([30, 31, 32, 32], np.int32)
    x, y, z, m, g = assemble([(x, y, MZ[m].copy(), m)], shuffle_seed)
    idx = g[0]
    return x, y, z, m, [int(idx[0]), int(idx[1]), int(idx[2])]
