"""Pins of the phi computation and phi16 mapping (section "Sort by phi")."""
import math

import numpy as np
import pytest

import oracle

# The degree-9 polynomial (Hastings form, Abramowitz & Stegun 4.4.49) with the
# coefficients of the reading R1 deviates from atan on [0, 1] by at most
# 1.15e-5 rad in exact arithmetic (test_polynomial_error_in_fp64); the fp32
# evaluation and octant reconstruction add at most a few ulp of pi.
POLY_BOUND = 1.15e-5
ATAN_BOUND = 1.2e-5 + 4.0 * 2.0 ** -22


def test_polynomial_error_in_fp64():
    a = [0.9998660, -0.3302995, 0.1801410, -0.0851330, 0.0208351]
    t = np.linspace(0.0, 1.0, 400001)
    p = np.polynomial.polynomial.polyval(t * t, a) * t
    assert np.abs(p - np.arctan(t)).max() <= POLY_BOUND


def test_atan2_error_bound_dense_grid():
    ang = np.linspace(-math.pi, math.pi, 20001)
    worst = 0.0
    for r in (5.1, 17.3, 42.0, 1e-3, 1e3):
        for a in ang:
            x, y = np.float32(r * math.cos(a)), np.float32(r * math.sin(a))
            got = oracle.atan2(float(y), float(x))
            exact = math.atan2(float(y), float(x))
            d = abs(got - exact)
            d = min(d, 2 * math.pi - d)  # +pi and -pi are the same angle
            worst = max(worst, d)
    assert worst <= ATAN_BOUND, worst


def test_atan2_special_points():
    assert oracle.atan2(0.0, 0.0) == 0.0
    assert oracle.atan2(0.0, 1.0) == 0.0
    assert abs(oracle.atan2(1.0, 0.0) - math.pi / 2) <= ATAN_BOUND
    assert abs(oracle.atan2(-1.0, 0.0) + math.pi / 2) <= ATAN_BOUND
    assert abs(oracle.atan2(0.0, -1.0) - math.pi) <= ATAN_BOUND
    assert abs(oracle.atan2(1.0, 1.0) - math.pi / 4) <= ATAN_BOUND
    # odd in y, and x-reflection gives pi - a
    for (y, x) in ((0.3, 2.0), (5.0, 1.0), (7.0, -3.0)):
        assert oracle.atan2(-y, x) == -oracle.atan2(y, x)


def _phi16_exact(x, y):
    return int(round(math.atan2(y, x) * 32768.0 / math.pi)) % 65536


def test_phi16_matches_closed_form_within_one_unit():
    rng = np.random.default_rng(3)
    x = rng.uniform(-42, 42, 50000).astype(np.float32)
    y = rng.uniform(-42, 42, 50000).astype(np.float32)
    got = oracle.phi16(x, y).astype(np.int64)
    exact = np.array([_phi16_exact(float(a), float(b)) for a, b in zip(x, y)])
    d = np.minimum((got - exact) % 65536, (exact - got) % 65536)
    # 1.2e-5 rad is 0.13 units; rounding can move at most one unit
    assert d.max() <= 1


def test_phi16_wraps_around_pi_and_zero():
    # just above and below the negative x axis: both near 32768
    a = oracle.phi16(np.array([-10.0, -10.0], np.float32), np.array([1e-3, -1e-3], np.float32))
    assert abs(int(a[0]) - 32768) <= 2 and abs(int(a[1]) - 32768) <= 2
    # just above and below the positive x axis: 0+ and 65535-
    b = oracle.phi16(np.array([10.0, 10.0], np.float32), np.array([2e-3, -2e-3], np.float32))
    assert 0 < int(b[0]) <= 3 and 65533 <= int(b[1]) <= 65535
    assert oracle.phi_distance(int(b[0]), int(b[1])) <= 6


@pytest.mark.parametrize("u,v,d", [(0, 65535, 1), (100, 200, 100), (0, 32768, 32768),
                                   (65000, 500, 1036), (7, 7, 0), (32767, 65535, 32768)])
def test_circular_distance(u, v, d):
    assert oracle.phi_distance(u, v) == d
    assert oracle.phi_distance(v, u) == d
