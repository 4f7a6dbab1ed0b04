"""Pins of the oracle's 3-sigma window and its bounding box (Sec. 3, App. B)."""
import numpy as np
import pytest

import oracle
from oracle import Setup, bruteforce
from synth import make_workload

ST = Setup(R=350.0, L=500.0, ny=140, nz=100, sigma_z=10.0, sigma_dl=42.0)


def test_bbox_is_tight_on_the_ellipse():
    """Points on b C^-1 b = 9 (parametrised from the quadratic form's own axes)
    reach exactly the App. B half-extents and never exceed them."""
    iz, il = ST.sigma_z ** -2, ST.sigma_dl ** -2
    phi = np.linspace(0.0, 2 * np.pi, 20001)
    for t in (0.0, 0.3, -0.55, 0.71, 1.5):
        c2i = 1.0 + t * t
        u = 3.0 / np.sqrt(2 * iz) * np.cos(phi)           # u = dz - t dy
        dy = 3.0 / (2.0 * np.sqrt(il * c2i)) * np.sin(phi)
        dz = u + t * dy
        ey, ez = 40.0, -30.0
        for k in range(0, phi.size, 1000):
            _, bq = oracle.kernel(ST, ey, ez, t, ey + dy[k], ez + dz[k])
            assert bq == pytest.approx(9.0, rel=1e-10)
        hy, hz = oracle.bbox(ST, t)
        assert np.max(np.abs(dy)) == pytest.approx(hy, rel=1e-7)
        assert np.max(np.abs(dz)) == pytest.approx(hz, rel=1e-7)


def test_every_in_window_pixel_is_in_the_bbox():
    rng = np.random.default_rng(41)
    yc, zc = ST.pixel_centres()
    Y, Z = np.meshgrid(yc, zc, indexing="ij")
    for _ in range(60):
        ey, ez, t = rng.uniform(-330, 330), rng.uniform(-240, 240), rng.uniform(-1.0, 1.0)
        _, bq = oracle.kernel_batch(ST, ey, ez, t, Y, Z)
        inside = bq <= 9.0
        hy, hz = oracle.bbox(ST, t)
        assert np.all(np.abs(Y[inside] - ey) <= hy * (1 + 1e-12))
        assert np.all(np.abs(Z[inside] - ez) <= hz * (1 + 1e-12))


def test_unbounded_window_equals_brute_force():
    """With an infinite cut every pixel is in every window: the C oracle's
    bounding-box loop then covers the whole grid and must equal the dense
    brute force exactly."""
    w = make_workload("small_5mm")
    ev = [e[:40].astype(np.float64) for e in w.events()]
    st = Setup.from_workload(w, cut=1e6)
    s = oracle.sensitivity(st)
    rho_o, stats = oracle.mlem(st, ev, 2, s=s)
    rho_b = bruteforce.mlem(st, ev, 2, s)
    np.testing.assert_allclose(rho_o, rho_b, rtol=1e-11, atol=1e-300)
    assert stats.n_window == 40 * st.ny * st.nz


@pytest.mark.parametrize("cut", [3.0, 2.0])
def test_windowed_equals_brute_force(cut):
    w = make_workload("small_5mm")
    ev = [e[:300].astype(np.float64) for e in w.events()]
    st = Setup.from_workload(w, cut=cut)
    s = oracle.sensitivity(st)
    rho_o, _ = oracle.mlem(st, ev, 3, s=s)
    rho_b = bruteforce.mlem(st, ev, 3, s)
    np.testing.assert_allclose(rho_o, rho_b, rtol=1e-11, atol=1e-300)


def test_tiny_grid_equals_brute_force():
    """8 x 6 pixels of 5 mm on a 20 mm / 30 mm detector, 50 events."""
    st = Setup(R=20.0, L=30.0, ny=8, nz=6, sigma_z=3.0, sigma_dl=8.0)
    rng = np.random.default_rng(7)
    zu = rng.uniform(-15, 15, 50)
    zd = rng.uniform(-15, 15, 50)
    dl = rng.uniform(-30, 30, 50)
    s = oracle.sensitivity(st)
    rho_o, _ = oracle.mlem(st, (zu, zd, dl), 4, s=s)
    rho_b = bruteforce.mlem(st, (zu, zd, dl), 4, s)
    np.testing.assert_allclose(rho_o, rho_b, rtol=1e-11, atol=1e-300)
