"""The fp16 hit-storage mode of the oracle: coordinates rounded to IEEE
binary16 (round to nearest, ties to even) before the unchanged algorithm."""
import numpy as np

import oracle
from paper_2207_03936_gb300 import synth, validation

CFG = dict(k_doublets=4, max_scatter_seed=0.04, max_scatter_follow=0.04,
           max_chi2_tracklet=20.0, hit_sigma=0.012)


def test_binary16_rounding_facts():
    # binary16 has an 11-bit significand: spacing 2^-10 in [1, 2), 2 in [2048, 4096)
    v = np.array([1.0, 1 + 2.0**-11, 1 + 3 * 2.0**-11, 2049.0, 2051.0, 65504.0, -3.0], np.float32)
    want = np.array([1.0, 1.0, 1 + 2.0**-9, 2048.0, 2052.0, 65504.0, -3.0], np.float32)
    assert np.array_equal(oracle.round_fp16(v), want)
    # 0.1 is 0x2E66 in binary16: 1638 * 2^-14
    assert oracle.round_fp16(np.float32(0.1)) == np.float32(1638 * 2.0**-14)


def test_rounding_error_bound_and_idempotence():
    rng = np.random.default_rng(3)
    v = rng.uniform(-750.0, 750.0, 100000).astype(np.float32)
    r = oracle.round_fp16(v)
    # half a unit in the last place of binary16: 2^(e - 11) for |v| in [2^e, 2^(e+1))
    e = np.floor(np.log2(np.abs(v.astype(np.float64))))
    assert (np.abs(r.astype(np.float64) - v) <= 2.0 ** (e - 11)).all()
    assert np.array_equal(oracle.round_fp16(r), r)


def test_fp16_mode_rounds_before_reconstruction():
    ev = synth.make_events(2, 20, workers=1)
    a = oracle.reconstruct(ev.x, ev.y, ev.z, ev.module, ev.event_offsets, ev.module_z,
                           oracle.config(**CFG), fp16_hits=True)
    b = oracle.reconstruct(oracle.round_fp16(ev.x), oracle.round_fp16(ev.y), oracle.round_fp16(ev.z),
                           ev.module, ev.event_offsets, ev.module_z, oracle.config(**CFG))
    assert np.array_equal(a.track_hits, b.track_hits) and np.array_equal(a.params, b.params)


def test_fp16_mode_physics():
    # same thresholds as the fp32 storage
    ev = synth.make_events(2, workers=1)
    res = oracle.reconstruct(ev.x, ev.y, ev.z, ev.module, ev.event_offsets, ev.module_z,
                             oracle.config(**CFG), fp16_hits=True)
    ind = validation.indicators(res.hit_offsets, res.track_hits, ev.mc, ev.n_particles)
    assert ind["efficiency"] >= 0.995
    assert ind["fake_fraction"] <= 0.005
    assert ind["clone_fraction"] <= 0.015
    assert ind["hit_purity"] >= 0.995
    assert ind["hit_efficiency"] >= 0.98
