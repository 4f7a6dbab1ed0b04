"""Pins of the oracle's geometry: Eq. 1 and Eq. 2 (Sec. 2).

The reference values come from plain ray geometry (the event generator traces
the emission line to the strip planes and measures Euclidean distances), not
from the oracle's formulas.
"""
import numpy as np
import pytest

import oracle
from oracle import Setup
from synth.events import _trace

ST = Setup(R=350.0, L=500.0, ny=140, nz=100, sigma_z=10.0, sigma_dl=42.0)


def _truth(n, seed, theta_max=1.2):
    rng = np.random.default_rng(seed)
    y = rng.uniform(-340.0, 340.0, n)
    z = rng.uniform(-240.0, 240.0, n)
    th = rng.uniform(-theta_max, theta_max, n)
    return y, z, th


def test_direct_reconstruction_roundtrip():
    """Eq. 2 (first forms) inverts noise-free measurements exactly."""
    y, z, th = _truth(3000, 11)
    zu, zd, dl = _trace(y, z, th, ST.R)
    for k in range(y.size):
        ey, ez, t = oracle.direct(ST, zu[k], zd[k], dl[k])
        assert abs(ey - y[k]) <= 1e-12 * 400.0
        assert abs(ez - z[k]) <= 1e-12 * 2000.0
        assert abs(t - np.tan(th[k])) <= 1e-12 * (1.0 + abs(np.tan(th[k])))


def test_eq1_matches_ray_geometry():
    """Eq. 1 gives the traced path-length difference, which is -2y/cos(theta)."""
    y, z, th = _truth(500, 12)
    zu, zd, dl = _trace(y, z, th, ST.R)
    for k in range(y.size):
        v = oracle.delta_l(ST, y[k], z[k], zu[k], zd[k])
        assert v == pytest.approx(dl[k], rel=1e-12, abs=1e-9)
        assert v == pytest.approx(-2.0 * y[k] / np.cos(th[k]), rel=1e-12, abs=1e-9)


def test_direct_special_case_perpendicular():
    """theta = 0: both hits at z, delta_l = -2y, so the event maps back to (y, z, 0)."""
    for y, z in [(0.0, 0.0), (123.5, -77.0), (-300.0, 240.0)]:
        ey, ez, t = oracle.direct(ST, z, z, -2.0 * y)
        assert (ey, ez, t) == pytest.approx((y, z, 0.0), abs=1e-12)


def test_printed_second_forms_do_not_invert():
    """Reading R1: the second forms printed in Eq. 2 are garbled (no square on
    z_u - z_d, a factor 2R instead of -1/2).  Taken literally they miss the
    emission point that the first forms recover."""
    y, z, th = 100.0, 0.0, 0.3
    zu, zd, dl = _trace(np.array([y]), np.array([z]), np.array([th]), ST.R)
    zu, zd, dl = float(zu[0]), float(zd[0]), float(dl[0])
    R = ST.R
    y_printed = 2 * R * dl / np.sqrt(zu - zd + 4 * R * R)
    z_printed = 0.5 * (zu + zd + (zu - zd) * dl / np.sqrt(zu - zd + 4 * R * R))
    ey, ez, _ = oracle.direct(ST, zu, zd, dl)
    assert (ey, ez) == pytest.approx((y, z), abs=1e-9)
    assert abs(y_printed - y) > 100.0 and abs(z_printed - z) > 10.0


def test_direct_image_is_the_histogram_of_the_emission_points():
    """The direct image of noise-free events is the 2-D histogram of their
    emission points (points kept at least a quarter pixel from pixel edges, so
    that the exact inversion decides every bin), and points beyond the grid
    (|y| > R is impossible; |z| > L/2 here) are not counted."""
    rng = np.random.default_rng(21)
    n = 20000
    iy = rng.integers(0, ST.ny, n)
    iz = rng.integers(-3, ST.nz + 3, n)          # some columns beyond the grid
    fy = rng.uniform(0.25, 0.75, n)
    fz = rng.uniform(0.25, 0.75, n)
    y = -ST.R + (iy + fy) * ST.dy
    z = -0.5 * ST.L + (iz + fz) * ST.dz
    th = rng.uniform(-0.6, 0.6, n)
    zu, zd, dl = _trace(y, z, th, ST.R)
    img = oracle.direct_image(ST, (zu, zd, dl))
    inside = (iz >= 0) & (iz < ST.nz)
    ref = np.zeros((ST.ny, ST.nz))
    np.add.at(ref, (iy[inside], iz[inside]), 1.0)
    np.testing.assert_array_equal(img, ref)
    assert img.sum() == inside.sum() < n
