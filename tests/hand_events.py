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
