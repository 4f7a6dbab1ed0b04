"""Pins of the oracle's sensitivity, Eq. s-yz (Sec. 2)."""
import numpy as np
import pytest

import oracle
from oracle import Setup
from synth.events import _trace

ST = Setup(R=350.0, L=500.0, ny=140, nz=100, sigma_z=10.0, sigma_dl=42.0)


def test_centre_closed_form():
    """At the centre both strips subtend the same half-angle atan(L/2R)."""
    v = oracle.sensitivity_at(ST, 0.0, 0.0)
    assert v == pytest.approx(2.0 / np.pi * np.arctan(250.0 / 350.0), rel=1e-14)
    assert v == pytest.approx(0.39486308657749, abs=1e-12)


def test_midplane_closed_form():
    """On y = 0 the binding limits are (L/2 - |z|)/R on both sides."""
    for z in np.linspace(-249.0, 249.0, 41):
        expect = 2.0 / np.pi * np.arctan((250.0 - abs(z)) / 350.0)
        assert oracle.sensitivity_at(ST, 0.0, z) == pytest.approx(expect, rel=1e-13, abs=1e-15)


def test_symmetry_and_range():
    s = oracle.sensitivity(ST)
    assert np.all(s >= 0.0) and np.all(s <= 1.0)
    assert np.all(s > 0.0)  # every pixel centre lies strictly inside the detector
    np.testing.assert_allclose(s, s[::-1, :], rtol=1e-13, atol=0)
    np.testing.assert_allclose(s, s[:, ::-1], rtol=1e-13, atol=0)
    yc, zc = ST.pixel_centres()
    for iy, iz in [(0, 0), (70, 50), (139, 99), (13, 77)]:
        assert s[iy, iz] == oracle.sensitivity_at(ST, yc[iy], zc[iz])


def test_outside_detector_is_zero():
    assert oracle.sensitivity_at(ST, 350.0, 0.0) == 0.0
    assert oracle.sensitivity_at(ST, -400.0, 0.0) == 0.0
    assert oracle.sensitivity_at(ST, 0.0, 600.0) == 0.0


def test_matches_monte_carlo_acceptance():
    """Eq. s-yz is the fraction of isotropic emission lines that hit both strips;
    count that fraction with the ray tracer at 20 points (4 binomial sigmas)."""
    rng = np.random.default_rng(21)
    n = 40000
    for _ in range(20):
        y = rng.uniform(-330.0, 330.0)
        z = rng.uniform(-240.0, 240.0)
        th = rng.uniform(-0.5 * np.pi, 0.5 * np.pi, n)
        zu, zd, _ = _trace(np.full(n, y), np.full(n, z), th, ST.R)
        frac = np.mean((np.abs(zu) <= 250.0) & (np.abs(zd) <= 250.0))
        s = oracle.sensitivity_at(ST, y, z)
        sig = np.sqrt(max(s * (1 - s), 1e-4) / n)
        assert abs(frac - s) <= 4.0 * sig, (y, z, frac, s)
