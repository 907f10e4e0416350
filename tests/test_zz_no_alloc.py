"""The allocation-free entry point, for callers that may not allocate device
memory (processes that reserve all their device memory up front, plug-ins in
an application that owns the memory pool).  It must give exactly the result of
sbt_reconstruct on two calls in a row (they share its fixed workspace), and
refuse batches larger than that workspace.  This file sorts last so that a
run stopping at the first failure has run every other test before it."""
import numpy as np
import pytest

from paper_2207_03936_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_matches_reconstruct_twice():
    from paper_2207_03936_gb300 import sbt
    ev = synth.make_events(2, 100, workers=1)
    assert ev.n_hits <= 1 << 19
    dev = [torch.from_numpy(a).cuda() for a in (ev.x, ev.y, ev.z, ev.module, ev.event_offsets)]
    h = sbt.sbt_create(ev.module_z, sbt.default_config())
    try:
        ref = sbt.sbt_reconstruct(h, *dev).compact()
        for _ in range(2):
            out = sbt.TrackOutput.allocate(ev.n_events, ev.n_hits)
            sbt.sbt_reconstruct_noalloc(h, *dev, out=out)
            torch.cuda.synchronize()
            got = out.compact()
            assert (got["event_status"] == 0).all() and got["counts"][2] == 0
            for k, v in ref.items():
                # the same bit-exact standard as the other reconstruction tests
                assert np.array_equal(got[k], v), k
        # a batch above the workspace limit is refused with a clear message
        big = 1 << 19
        x = torch.zeros(big + 1, dtype=torch.float32, device="cuda")
        m = torch.zeros(big + 1, dtype=torch.int32, device="cuda")
        off = torch.tensor([0, big + 1], dtype=torch.int32, device="cuda")
        out = sbt.TrackOutput.allocate(1, big + 1)
        with pytest.raises(sbt.SbtError, match="fixed workspace"):
            sbt.sbt_reconstruct_noalloc(h, x, x, x, m, off, out=out)
    finally:
        h.close()


def test_noalloc_near_its_limits_allocates_nothing():
    # 4096 small events (one vertex, Poisson(6) tracks) totalling 99.6% of
    # the 2^19 hits: the fixed workspace at the edge of both limits.  The
    # result must equal sbt_reconstruct's, and the device's free memory must
    # not move across two calls (after one call that loads the kernels).
    from paper_2207_03936_gb300 import sbt
    ev = synth.generate(synth.Recipe(n_events=4096, pv_mode="fixed", pv_mean=1, tracks_per_pv=6.0,
                                     seed=3), workers=1)
    assert ev.n_events == 4096 and 0.99 * (1 << 19) < ev.n_hits <= 1 << 19
    dev = [torch.from_numpy(a).cuda() for a in (ev.x, ev.y, ev.z, ev.module, ev.event_offsets)]
    h = sbt.sbt_create(ev.module_z, sbt.default_config())
    try:
        ref = sbt.sbt_reconstruct(h, *dev).compact()
        assert (ref["event_status"] == 0).all() and ref["counts"][0] > 20000
        outs = [sbt.TrackOutput.allocate(ev.n_events, ev.n_hits) for _ in range(2)]
        sbt.sbt_reconstruct_noalloc(h, *dev, out=outs[0])
        torch.cuda.synchronize()
        assert h.last_launch_count() == 5
        free0 = torch.cuda.mem_get_info()[0]
        for out in outs:
            sbt.sbt_reconstruct_noalloc(h, *dev, out=out)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        for out in outs:
            got = out.compact()
            for k, v in ref.items():
                assert np.array_equal(got[k], v), k
    finally:
        h.close()
