"""A second, deliberately different statement of the whole Search-by-triplet
loop, for tiny events (a few modules, tens of hits), used to pin the oracle.

It follows the paper's section "Track seeding and track following" and
"Tracklet filter" with the readings R3-R9 of the oracle, but computes every
choice by plain enumeration:
  - no phi windows and no binary searches: every seeding candidate is tried
    against every unflagged hit of the third module, every forming track
    against every unflagged hit of the target module;
  - the one-round claims (R6, R7) are resolved by sorting all the step's
    extensions by their key and giving each hit to its first claimant in
    that order (the oracle instead keeps a running minimum per hit);
  - tracks keep their whole hit lists (the oracle keeps them in a pool).
Only the pinned phi16 mapping comes from the oracle.  Arithmetic is fp32
with every operation rounded as written (numpy float32 scalars), like both
implementations it checks.
"""
from __future__ import annotations

import numpy as np

import oracle

F = np.float32


def _circ(u, v):
    d = (int(u) - int(v)) % 65536
    return min(d, 65536 - d)


def _extrapolate(ax, ay, az, cx, cy, cz, zt):
    dz = F(cz - az)
    tz = F(F(zt - cz) / dz)
    return F(cx + F(F(cx - ax) * tz)), F(cy + F(F(cy - ay) * tz))


def _scatter(bx, by, xp, yp):
    dx = F(bx - xp)
    dy = F(by - yp)
    return F(F(dx * dx) + F(dy * dy))


def fit_chi2(xs, ys, zs, sigma):
    """chi2 of the least-squares line through the hits, fp32 sums in hit
    order (reading R8)."""
    n = F(len(xs))
    sx = sy = sz = F(0.0)
    for x, y, z in zip(xs, ys, zs):
        sx, sy, sz = F(sx + x), F(sy + y), F(sz + z)
    xm, ym, zm = F(sx / n), F(sy / n), F(sz / n)
    szz = szx = szy = F(0.0)
    for x, y, z in zip(xs, ys, zs):
        dz = F(z - zm)
        szz = F(szz + F(dz * dz))
        szx = F(szx + F(dz * F(x - xm)))
        szy = F(szy + F(dz * F(y - ym)))
    tx, ty = F(szx / szz), F(szy / szz)
    s = F(0.0)
    for x, y, z in zip(xs, ys, zs):
        dz = F(z - zm)
        rx = F(F(x - xm) - F(tx * dz))
        ry = F(F(y - ym) - F(ty * dz))
        s = F(s + F(F(rx * rx) + F(ry * ry)))
    return F(s / F(F(sigma) * F(sigma)))


def reconstruct(x, y, z, module, module_z, k_doublets=4, max_scatter_seed=0.04,
                max_scatter_follow=0.04, max_chi2_tracklet=20.0, hit_sigma=0.012,
                module_z2=None, stats=None):
    """Track list of one event: each track a list of input hit indices in
    traversal order, tracks ordered by their smallest input index.  stats
    (a dict, optional) receives how often the claims decided something:
    extensions that lost a claim, and tracklets that passed the filter's cut
    but lost the claim round."""
    lost_ext = 0
    x, y, z = (np.asarray(a, np.float32) for a in (x, y, z))
    module = np.asarray(module, np.int32)
    module_z = np.asarray(module_z, np.float32)
    M = len(module_z)
    n = len(x)
    S_seed, S_follow, C3 = F(max_scatter_seed), F(max_scatter_follow), F(max_chi2_tracklet)
    ph = oracle.phi16(x, y)
    order = np.lexsort((np.arange(n), ph, module))       # sorted position -> input index
    sx, sy, sz, sm, sp = x[order], y[order], z[order], module[order], ph[order]
    on = [np.flatnonzero(sm == k).tolist() for k in range(M)]

    def plane_z(mod, b):
        if module_z2 is not None and sx[b] < 0:
            return F(module_z2[mod])
        return module_z[mod]

    flag = np.zeros(n, bool)
    forming, finished = [], []                 # tracks: {"hits", "skipped", "key"}
    for s in range(M - 2):
        # seeding over the middle module s+1 with the flags as they stand
        for c in on[s + 1]:
            if flag[c]:
                continue
            outer = [a for a in on[s] if not flag[a]]
            if len(outer) > k_doublets:
                dk = sorted(_circ(sp[a], sp[c]) for a in outer)[k_doublets - 1]
                outer = [a for a in outer if _circ(sp[a], sp[c]) <= dk]
            best = None
            for a in outer:
                for b in on[s + 2]:
                    if flag[b]:
                        continue
                    xp, yp = _extrapolate(sx[a], sy[a], sz[a], sx[c], sy[c], sz[c], plane_z(s + 2, b))
                    sc = _scatter(sx[b], sy[b], xp, yp)
                    if sc < S_seed and (best is None or (float(sc), a, b) < best):
                        best = (float(sc), a, b)
            if best is not None:
                forming.append({"hits": [best[1], c, best[2]], "skipped": 0, "key": c})
        if s + 3 > M - 1:
            finished += forming
            forming = []
            break
        t = s + 3
        # every extension with its key and the hits it claims
        ext = []
        for i, T in enumerate(forming):
            h = T["hits"]
            if len(h) == 3 and flag[h].any():
                continue
            best = None
            for b in on[t]:
                if flag[b]:
                    continue
                xp, yp = _extrapolate(sx[h[-2]], sy[h[-2]], sz[h[-2]], sx[h[-1]], sy[h[-1]], sz[h[-1]],
                                      plane_z(t, b))
                sc = _scatter(sx[b], sy[b], xp, yp)
                if sc < S_follow and (best is None or (float(sc), b) < best):
                    best = (float(sc), b)
            if best is not None:
                claimed = [best[1]] + (list(h) if len(h) == 3 else [])
                ext.append(((best[0], T["key"]), i, best[1], claimed))
        ext.sort()
        first = {}
        for key, _, _, claimed in ext:
            for hit in claimed:
                first.setdefault(hit, key)
        won = {i: (b, claimed) for key, i, b, claimed in ext if all(first[hh] == key for hh in claimed)}
        lost_ext += len(ext) - len(won)
        alive = []
        for i, T in enumerate(forming):
            if i in won:
                b, claimed = won[i]
                flag[claimed] = True
                T["hits"].append(b)
                T["skipped"] = 0
                alive.append(T)
            else:
                T["skipped"] += 1
                (finished if T["skipped"] == 2 else alive).append(T)
        forming = alive
    tracks = [T["hits"] for T in finished if len(T["hits"]) >= 4]
    # tracklet filter: unflagged hits and chi2 under the cut, then claims in key order
    cand = []
    for T in finished:
        h = T["hits"]
        if len(h) != 3 or flag[h].any():
            continue
        q = fit_chi2(sx[h], sy[h], sz[h], hit_sigma)
        if q < C3:
            cand.append(((float(q), T["key"]), h))
    cand.sort()
    first = {}
    for key, h in cand:
        for hit in h:
            first.setdefault(hit, key)
    kept = [h for key, h in cand if all(first[hh] == key for hh in h)]
    tracks += kept
    if stats is not None:
        stats["lost_extensions"] = lost_ext
        stats["lost_tracklets"] = len(cand) - len(kept)
    out = [[int(order[p]) for p in h] for h in tracks]
    return sorted(out, key=min)
