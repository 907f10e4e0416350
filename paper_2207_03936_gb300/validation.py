"""Physics performance indicators of reconstructed tracks against generator truth.

The five indicators of the paper's introduction (after Schiller et al.):
reconstruction efficiency, fake (ghost) fraction, clone fraction, hit purity
and hit efficiency.  A track is associated with a particle when at least 70%
of its hits come from that particle; a particle is reconstructible when it
left at least 3 hits.  Input is the CSR track output and the per-hit truth
(particle id, -1 for noise).
"""
from __future__ import annotations

import numpy as np


def indicators(hit_offsets, track_hits, mc, n_particles: int, min_hits: int = 3,
               assoc_frac: float = 0.7) -> dict:
    hit_offsets = np.asarray(hit_offsets, dtype=np.int64)
    track_hits = np.asarray(track_hits, dtype=np.int64)
    mc = np.asarray(mc, dtype=np.int64)
    n_tracks = hit_offsets.shape[0] - 1
    part_hits = np.bincount(mc[mc >= 0], minlength=n_particles)
    reconstructible = part_hits >= min_hits
    lens = np.diff(hit_offsets)
    assoc = np.full(n_tracks, -1, dtype=np.int64)
    n_match = np.zeros(n_tracks, dtype=np.int64)
    if n_tracks:
        trk_of_hit = np.repeat(np.arange(n_tracks), lens)
        pid = mc[track_hits]
        ok = pid >= 0
        # most frequent particle per track
        key = trk_of_hit[ok] * (n_particles + 1) + pid[ok]
        uk, cnt = np.unique(key, return_counts=True)
        t_of = uk // (n_particles + 1)
        p_of = uk % (n_particles + 1)
        order = np.lexsort((-cnt, t_of))
        t_sorted = t_of[order]
        first = np.ones(t_sorted.shape[0], dtype=bool)
        first[1:] = t_sorted[1:] != t_sorted[:-1]
        best_t = t_sorted[first]
        best_p = p_of[order][first]
        best_c = cnt[order][first]
        good = best_c >= assoc_frac * lens[best_t]
        assoc[best_t[good]] = best_p[good]
        n_match[best_t] = best_c
    matched = assoc >= 0
    n_fake = int((~matched).sum())
    per_part = np.bincount(assoc[matched], minlength=n_particles)
    found = (per_part > 0) & reconstructible
    n_reco_tracks_of_recble = per_part[reconstructible]
    clones = int(np.maximum(per_part - 1, 0).sum())
    purity = float((n_match[matched] / lens[matched]).mean()) if matched.any() else float("nan")
    hit_eff = (float((n_match[matched] / part_hits[assoc[matched]]).mean())
               if matched.any() else float("nan"))
    return {
        "n_tracks": int(n_tracks),
        "n_reconstructible": int(reconstructible.sum()),
        "efficiency": float(found.sum() / max(int(reconstructible.sum()), 1)),
        "fake_fraction": float(n_fake / max(n_tracks, 1)),
        "clone_fraction": float(clones / max(n_tracks, 1)),
        "hit_purity": purity,
        "hit_efficiency": hit_eff,
        "reconstructed_reconstructible": int((n_reco_tracks_of_recble > 0).sum()),
    }
