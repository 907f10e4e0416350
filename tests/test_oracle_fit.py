"""Pins of the least-squares straight-line fit (tracklet filter; consolidation)."""
import numpy as np

import oracle
from paper_2207_03936_gb300 import synth

MZ = synth.module_z_traversal()


def test_fit_exact_on_collinear_hits():
    z = MZ[10:30]
    x = (1.5 + 0.01 * z.astype(np.float64)).astype(np.float32)
    y = (-2.0 - 0.02 * z.astype(np.float64)).astype(np.float32)
    p, chi2 = oracle.fit(x, y, z, 0.012)
    np.testing.assert_allclose(p, [1.5, -2.0, 0.01, -0.02], rtol=0, atol=2e-5)
    assert chi2 < 1e-2  # only fp32 representation error of the inputs


def test_fit_matches_numpy_lstsq():
    rng = np.random.default_rng(11)
    for n in (3, 4, 7, 20, 52):
        mods = np.sort(rng.choice(52, n, replace=False))
        z = MZ[mods]
        x = (3.0 + 0.005 * z + rng.normal(0, 0.012, n)).astype(np.float32)
        y = (-4.0 + 0.007 * z + rng.normal(0, 0.012, n)).astype(np.float32)
        p, chi2 = oracle.fit(x, y, z, 0.012)
        A = np.stack([np.ones(n), z.astype(np.float64)], 1)
        (x0, tx), rx, *_ = np.linalg.lstsq(A, x.astype(np.float64), rcond=None)
        (y0, ty), ry, *_ = np.linalg.lstsq(A, y.astype(np.float64), rcond=None)
        np.testing.assert_allclose(p[2:], [tx, ty], rtol=1e-4, atol=1e-7)
        np.testing.assert_allclose(p[:2], [x0, y0], rtol=1e-4, atol=2e-4)
        exact = (float(rx.sum()) + float(ry.sum())) / 0.012 ** 2 if n > 2 else 0.0
        assert abs(float(chi2) - exact) <= 2e-3 * exact + 0.05


def test_three_point_closed_form():
    # three equally spaced points: residual sum = |second difference|^2 / 6
    z = MZ[[20, 21, 22]]
    d = np.array([0.03, -0.02])
    x = np.array([1.0, 1.2, 1.4 + d[0]], np.float64)
    y = np.array([2.0, 2.1, 2.2 + d[1]], np.float64)
    p, chi2 = oracle.fit(x.astype(np.float32), y.astype(np.float32), z, 0.01)
    expect = float(d @ d) / 6.0 / 0.01 ** 2
    assert abs(float(chi2) - expect) <= 1e-3 * expect
