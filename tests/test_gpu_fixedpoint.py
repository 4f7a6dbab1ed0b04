"""The MLEM tile pass sums each work item's terms x = P rho' / D (in [0, 1],
Eq. iter) in two-word fixed point, H = floor(x 2^12) and L = round of the
remainder at 2^-20, with the words' sums exact while an item holds at most
4000 events (the layout constants of the device header state the split and
its bounds).  These tests drive the accumulator to its bounds and check the
result against the FP64 oracle at the parity bar (max relative error <= 1e-4
on pixels above 1% of the maximum):

- a point source whose events fill work items to the 4000-event cap, started
  from a spike image, so that every event of an item puts x ~ 1 on one pixel
  and the H word's sum comes within 5% of its 2^24 limit;
- an image with zero pixels: the update keeps them at 0, and the
  back-projection reports the oracle's A = sum_j P/D where rho' > 0 and
  nothing from the tile pass where rho' = 0 (the update rho A is 0 there
  either way).
"""
from dataclasses import replace

import numpy as np
import pytest

import oracle
from oracle import Setup
from synth import make_workload
from synth.phantom import Ellipse, Phantom

pytestmark = pytest.mark.gpu

TOL = 1e-4


def rel_err(gpu, ref, mask):
    gpu = np.asarray(gpu, dtype=np.float64).reshape(ref.shape)
    return float(np.max(np.abs(gpu[mask] - ref[mask]) / ref[mask]))


def _point_workload(n_events):
    """small_5mm's grid and resolution; the tracer a 4 mm disc at (y, z) = (-30, 20)."""
    src = Phantom((Ellipse(20.0, -30.0, 2.0, 2.0, 0.0, 1.0),))
    return replace(make_workload("small_5mm"), n_events=n_events, phantom_fn=lambda: src)


def test_point_source_full_items_spike_start():
    from paper_1502_07478_gb300 import Recon
    w = _point_workload(600_000)
    ev = w.events()
    st = Setup.from_workload(w)
    # spike start: the source pixel 1e3, every other pixel 1e-6
    rho0 = np.full((w.ny, w.nz), 1e-6, np.float32)
    iy = int((-30.0 + w.R) / w.dy)
    iz = int((20.0 + w.L / 2) / w.dz)
    rho0[iy, iz] = 1e3
    r = Recon.from_workload(w)
    r.upload_events(*ev)
    # one item per SM and bin: items reach the 4000-event cap
    r.set_schedule(ty_cap=128, items_per_sm=1, order=0)
    r.set_image(rho0)
    imgs = []
    for _ in range(3):
        r.iterate(1)
        imgs.append(r.read_image().cpu().numpy())
    stats = r.stats()
    r.close()
    assert stats["n_outliers"] == 0 and stats["n_clipped"] == 0
    ref1, rs = oracle.mlem(st, ev, 1, rho0=rho0)
    ref3, _ = oracle.mlem(st, ev, 3, rho0=rho0)
    assert rs.n_used == stats["n_used"]
    for img, ref in ((imgs[0], ref1), (imgs[2], ref3)):
        assert rel_err(img, ref, ref > 0.01 * ref.max()) <= TOL
    # the spike holds nearly every event's whole responsibility: x ~ 1 there
    s = oracle.sensitivity(st)
    assert s[iy, iz] * ref1[iy, iz] > 0.9 * rs.n_used
    # the background in aggregate: count conservation sum_l s_l rho_l = N_used
    for img in imgs:
        assert float((s * img).sum()) == pytest.approx(rs.n_used, rel=1e-6)


def test_zero_pixels_and_backprojection():
    from paper_1502_07478_gb300 import Recon
    w = make_workload("small_5mm")
    ev = w.events()
    st = Setup.from_workload(w)
    rng = np.random.Generator(np.random.PCG64(17))
    rho = rng.uniform(0.5, 2.0, size=(w.ny, w.nz)).astype(np.float32)
    rho[40:70, 30:60] = 0.0                     # a zero block inside the field of view
    r = Recon.from_workload(w)
    r.upload_events(*ev)
    r.set_image(rho)
    A = r.backproject().cpu().numpy().astype(np.float64)
    stats = r.stats()
    r.iterate(2)
    img = r.read_image().cpu().numpy()
    r.close()
    # oracle A = 1 + g_rho / s (dlogL/drho_l = s_l (A_l - 1), Eq. iter)
    s = oracle.sensitivity(st)
    _, g, _ = oracle.loglik_grad(st, ev, rho, want_sigma=False)
    pos = (s > 0) & (rho > 0)
    A_ref = np.zeros_like(s)
    A_ref[pos] = 1.0 + g.reshape(s.shape)[pos] / s[pos]
    assert rel_err(A, A_ref, pos & (A_ref > 0.01 * A_ref.max())) <= TOL
    if stats["n_outliers"] == 0:
        assert np.all(A[rho == 0] == 0.0)
    assert np.all(img[rho == 0] == 0.0)
    ref, _ = oracle.mlem(st, ev, 2, rho0=rho)
    assert rel_err(img, ref, ref > 0.01 * ref.max()) <= TOL
