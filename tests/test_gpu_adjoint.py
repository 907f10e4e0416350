"""GPU adjoint of the alignment objective against the fp64 oracle and central
differences, and its torch.autograd wrapper."""
import numpy as np
import pytest

import oracle
from paper_2207_03936_gb300 import synth
from tests.test_oracle_alignment import central_differences, truth_tracks

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# the library stores hit_sigma as fp32; the oracle gets the same value
SIGMA = float(np.float32(0.012))


@pytest.fixture(scope="module")
def setup():
    from paper_2207_03936_gb300 import sbt
    ev = synth.make_events(5, 40, workers=1)
    ho, th = truth_tracks(ev)
    h = sbt.sbt_create(ev.module_z, sbt.default_config(hit_sigma=SIGMA))
    d = {k: torch.from_numpy(v).cuda() for k, v in
         dict(x=ev.x, y=ev.y, z=ev.z, m=ev.module, ho=ho, th=th).items()}
    yield sbt, h, ev, ho, th, d
    h.close()


def test_adjoint_matches_oracle_gradient(setup):
    sbt, h, ev, ho, th, d = setup
    rng = np.random.default_rng(8)
    align = np.concatenate([rng.normal(0, 0.005, (52, 3)), rng.normal(0, 5e-5, (52, 3))], 1)
    c, g = sbt.sbt_fit_adjoint(h, d["x"], d["y"], d["z"], d["m"], d["ho"], d["th"],
                               torch.from_numpy(align).cuda())
    torch.cuda.synchronize()
    v, go = oracle.align_chi2(ev.x, ev.y, ev.z, ev.module, ho, th, ev.module_z, align, SIGMA)
    assert abs(float(c.item()) - v) <= 1e-12 * v
    g = g.cpu().numpy()
    scale = np.abs(go).max()
    assert (np.abs(g - go) <= 1e-9 * np.maximum(np.abs(go), 1e-3 * scale)).all()


def test_adjoint_against_central_differences(setup):
    # 12 events keep the objective small enough (~3e6) for fp64 differences
    # to resolve every gradient entry to better than 1e-6
    sbt, h, _, _, _, _ = setup
    ev = synth.make_events(5, 12, workers=1)
    ho, th = truth_tracks(ev)
    d = [torch.from_numpy(a).cuda() for a in (ev.x, ev.y, ev.z, ev.module, ho, th)]
    rng = np.random.default_rng(9)
    align = np.concatenate([rng.normal(0, 0.005, (52, 3)), rng.normal(0, 5e-5, (52, 3))], 1)
    _, g = sbt.sbt_fit_adjoint(h, *d, torch.from_numpy(align).cuda())
    g = g.cpu().numpy()
    fd = central_differences(
        lambda a: oracle.align_chi2(ev.x, ev.y, ev.z, ev.module, ho, th, ev.module_z, a, SIGMA,
                                    False)[0], align)
    scale = np.abs(fd).max()
    assert (np.abs(g - fd) <= 1e-6 * np.maximum(np.abs(fd), 1e-3 * scale)).all()


def test_adjoint_is_bitwise_reproducible(setup):
    sbt, h, ev, ho, th, d = setup
    a = torch.zeros(52, 6, dtype=torch.float64, device="cuda")
    c1, g1 = sbt.sbt_fit_adjoint(h, d["x"], d["y"], d["z"], d["m"], d["ho"], d["th"], a)
    c2, g2 = sbt.sbt_fit_adjoint(h, d["x"], d["y"], d["z"], d["m"], d["ho"], d["th"], a)
    assert torch.equal(c1, c2) and torch.equal(g1, g2)


def test_autograd_function(setup):
    sbt, h, ev, ho, th, d = setup
    a = torch.zeros(52, 6, dtype=torch.float64, device="cuda", requires_grad=True)
    loss = sbt.alignment_chi2(h, d["x"], d["y"], d["z"], d["m"], d["ho"], d["th"], a)
    (2.0 * loss).backward()
    _, g = sbt.sbt_fit_adjoint(h, d["x"], d["y"], d["z"], d["m"], d["ho"], d["th"], a.detach())
    assert torch.allclose(a.grad, 2.0 * g, rtol=0, atol=0)
    # a small step along -grad lowers the objective by about eta * |grad|^2
    with torch.no_grad():
        f0 = float(loss.detach())
        eta = 1e-4 * f0 / float((g * g).sum())
        l2 = sbt.alignment_chi2(h, d["x"], d["y"], d["z"], d["m"], d["ho"], d["th"], a - eta * g)
    assert f0 - float(l2) > 0.5e-4 * f0


def test_adjoint_on_reconstructed_tracks(setup):
    sbt, h, ev, ho, th, d = setup
    out = sbt.sbt_reconstruct_batched(h, d["x"], d["y"], d["z"], d["m"],
                                      torch.from_numpy(ev.event_offsets).cuda())
    r = out.compact()
    a = np.zeros((52, 6))
    c, g = sbt.sbt_fit_adjoint(h, d["x"], d["y"], d["z"], d["m"],
                               torch.from_numpy(r["hit_offsets"]).cuda(),
                               torch.from_numpy(r["track_hits"]).cuda(), torch.from_numpy(a).cuda())
    v, go = oracle.align_chi2(ev.x, ev.y, ev.z, ev.module, r["hit_offsets"], r["track_hits"],
                              ev.module_z, a, SIGMA)
    assert abs(float(c.item()) - v) <= 1e-12 * v
    # the fp64 objective at zero alignment equals the sum of the fp32 fits
    assert abs(v - float(r["chi2"].astype(np.float64).sum())) <= 1e-3 * v


def test_adjoint_on_long_repeated_and_invalid_tracks(setup):
    # tracks of 104 hits (two per module), a repeated module, and tracks
    # without a line fit or with indices out of range (skipped and counted):
    # the same value, gradient and count as the oracle's
    sbt, h, _, _, _, _ = setup
    from tests.hand_events import MZ
    from tests.test_oracle_alignment import _odd_tracks
    x, y, z, m, good = _odd_tracks()
    x, y, z = (np.append(a, np.float32(a[0])) for a in (x, y, z))
    m = np.append(m, np.int32(52))
    bad = [np.array([11]), np.array([], np.int64), np.array([5, 5 + 52]), np.array([1, 2, 105]),
           np.array([58, 59, 104, 61])]
    allt = [good[0], bad[0], good[1], bad[1], bad[2], good[2], bad[3], bad[4]] * 40
    th = np.concatenate(allt).astype(np.int32)
    ho = np.concatenate([[0], np.cumsum([len(t) for t in allt])]).astype(np.int32)
    rng = np.random.default_rng(21)
    align = np.concatenate([rng.normal(0, 0.005, (52, 3)), rng.normal(0, 5e-5, (52, 3))], 1)
    d = [torch.from_numpy(a).cuda() for a in (x, y, z, m, ho, th)]
    c, g, sk = sbt.sbt_fit_adjoint(h, *d, torch.from_numpy(align).cuda(), with_skipped=True)
    torch.cuda.synchronize()
    v, go, so = oracle.align_chi2(x, y, z, m, ho, th, MZ, align, SIGMA, count_skipped=True)
    assert int(sk.item()) == so == 5 * 40
    assert abs(float(c.item()) - v) <= 1e-12 * v
    g = g.cpu().numpy()
    scale = np.abs(go).max()
    assert (np.abs(g - go) <= 1e-9 * np.maximum(np.abs(go), 1e-3 * scale)).all()
    # reproducible to the bit with the repeated-module path taken
    c2, g2, _ = sbt.sbt_fit_adjoint(h, *d, torch.from_numpy(align).cuda(), with_skipped=True)
    assert torch.equal(c.cpu(), c2.cpu()) and np.array_equal(g, g2.cpu().numpy())
