"""Writes oracle_digests.json: the oracle's results on fixed synthetic inputs.

Calls only the oracle and the seeded input generator (no CUDA)."""
import hashlib
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2207_03936_gb300 import synth  # noqa: E402

CFG = dict(k_doublets=4, max_scatter_seed=0.04, max_scatter_follow=0.04, max_chi2_tracklet=20.0,
           hit_sigma=0.012)

# (name, workload config, events, seed, module pairs, fp16 hit storage)
CASES = [
    ("small", 1, None, 0, False, False),
    ("upgrade_60", 2, 60, 0, False, False),
    ("uneven_20", 3, 20, 5, False, False),
    ("upgrade_60_pairs", 2, 60, 0, True, False),
    ("upgrade_60_fp16", 2, 60, 0, False, True),
]


def digest(res) -> str:
    m = hashlib.sha256()
    for a in (res.track_offsets, res.hit_offsets, res.track_hits, res.ndof, res.status):
        m.update(np.ascontiguousarray(a, dtype=np.int32).tobytes())
    for a in (res.params, res.chi2):
        m.update(np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).tobytes())
    return m.hexdigest()


def run(case):
    name, config, n, seed, pairs, fp16 = case
    ev = synth.make_events(config, n, seed=seed, workers=1, pairs=pairs)
    res = oracle.reconstruct(ev.x, ev.y, ev.z, ev.module, ev.event_offsets, ev.module_z,
                             oracle.config(**CFG), n_threads=4, fp16_hits=fp16,
                             module_z2=ev.module_z2)
    return {"name": name, "workload_config": config, "events": ev.n_events, "seed": seed,
            "pairs": pairs, "fp16_hits": fp16, "hits": ev.n_hits, "tracks": res.n_tracks,
            "track_hits": int(res.hit_offsets[-1]), "sha256": digest(res)}


def main():
    out = {"config": CFG, "cases": [run(c) for c in CASES]}
    with open(os.path.join(HERE, "oracle_digests.json"), "w") as f:
        json.dump(out, f, indent=2)
        f.write("\n")


if __name__ == "__main__":
    main()
