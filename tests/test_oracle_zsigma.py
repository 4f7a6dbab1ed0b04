"""Pins of the z-dependent resolution of the oracle (Sec. 3; reading R15).

Sec. 3 says that the z resolution degrades by about 10% from the centre of the
strips to their ends and gives no functional form.  The reading implemented is
sigma_z(z~) = sigma_z (1 + kappa_z min(1, (2 z~/L)^2)) for an event reconstructed
at z~: its kernel, window and bounding box use that sigma_z.  These tests pin the
reading's profile, the kernel against the exact theta-quadrature of the Gaussian
with the event's own sigma_z, the App. B box, and the gradient with respect to
the base sigma_z against differences of the log-likelihood.
"""
import numpy as np
import pytest

import oracle
from oracle import Setup
from synth import make_workload
from test_oracle_kernel import _exact

KAPPA = 0.1


def _setup(**kw):
    return Setup(R=350.0, L=500.0, ny=140, nz=100, sigma_z=10.0, sigma_dl=42.0, **kw)


@pytest.mark.parametrize("ez, f", [(0.0, 1.0), (62.5, 1.00625), (-125.0, 1.025),
                                   (250.0, 1.1), (-280.0, 1.1)])
def test_profile_of_the_reading(ez, f):
    """The kernel of an event at z~ equals the constant-sigma kernel with
    sigma_z f, f = 1 + kappa min(1, (2 z~/L)^2): 1 at the centre, 1 + kappa at
    the strip ends and beyond."""
    stk = _setup(kappa_z=KAPPA)
    stf = _setup()
    stf.sigma_z = 10.0 * f
    for ey, t, dy, dz in [(40.0, 0.2, 3.0, 4.0), (-120.0, -0.5, -6.0, 2.0),
                          (200.0, 0.7, 1.0, -9.0)]:
        Pk, bqk = oracle.kernel(stk, ey, ez, t, ey + dy, ez + dz)
        Pf, bqf = oracle.kernel(stf, ey, ez, t, ey + dy, ez + dz)
        assert Pk == pytest.approx(Pf, rel=1e-14)
        assert bqk == pytest.approx(bqf, rel=1e-14)


def test_kernel_with_kappa_matches_exact_quadrature():
    """Against the exact theta-integral of the Gaussian with the event's own
    sigma_z the Laplace kernel is as close as at constant sigma, while the z
    dependence moves it by far more than that error near the strip ends."""
    stk = _setup(kappa_z=0.3)
    st0 = _setup()
    rng = np.random.default_rng(43)
    errs, shifts = [], []
    while len(errs) < 60:
        py = rng.uniform(-300.0, 300.0)
        pz = rng.uniform(-240.0, 240.0)
        th = rng.uniform(-0.4, 0.4)
        ev = (pz + (stk.R - py) * np.tan(th) + rng.normal() * stk.sigma_z,
              pz - (stk.R + py) * np.tan(th) + rng.normal() * stk.sigma_z,
              -2.0 * py / np.cos(th) + rng.normal() * stk.sigma_dl)
        ey, ez, t = oracle.direct(stk, *ev)
        if abs(2.0 * ez / stk.L) < 0.5:
            continue
        P, bq = oracle.kernel(stk, ey, ez, t, py, pz)
        if bq > stk.cut ** 2:
            continue
        f = 1.0 + 0.3 * min(1.0, (2.0 * ez / stk.L) ** 2)
        stf = _setup()
        stf.sigma_z = 10.0 * f
        errs.append(abs(P / _exact(stf, ev, py, pz) - 1.0))
        shifts.append(abs(P / oracle.kernel(st0, ey, ez, t, py, pz)[0] - 1.0))
    errs, shifts = np.array(errs), np.array(shifts)
    assert errs.mean() < 0.01 and np.percentile(errs, 90) < 0.025
    assert np.median(shifts) > 5 * np.median(errs)


def test_bbox_is_tight_on_the_ellipse_with_kappa():
    """App. B box of an event at z~ = 200 mm: the extreme points of the cut
    ellipse bC^-1b = 9 with sigma_z (1 + kappa (2 z~/L)^2)."""
    st = _setup(kappa_z=KAPPA)
    ey, ez = 40.0, 200.0
    f = 1.0 + KAPPA * (2.0 * ez / st.L) ** 2
    iz, il = (st.sigma_z * f) ** -2, st.sigma_dl ** -2
    phi = np.linspace(0.0, 2 * np.pi, 200001)
    for t in (0.0, 0.3, -0.8):
        c2i = 1.0 + t * t
        # b C^-1 b = 2 iz u^2 + 4 il dy^2 c2i = 9 on the ellipse
        u = 3.0 / np.sqrt(2.0 * iz) * np.cos(phi)
        dy = 3.0 / (2.0 * np.sqrt(il * c2i)) * np.sin(phi)
        dz = u + t * dy
        for k in range(0, phi.size, 2000):
            _, bq = oracle.kernel(st, ey, ez, t, ey + dy[k], ez + dz[k])
            assert bq == pytest.approx(9.0, rel=1e-9)
        hy, hz = oracle.bbox(st, t, ez)
        assert np.max(np.abs(dy)) == pytest.approx(hy, rel=1e-7)
        assert np.max(np.abs(dz)) == pytest.approx(hz, rel=1e-7)


def test_every_in_window_pixel_is_in_the_bbox_with_kappa():
    st = _setup(kappa_z=0.5)
    rng = np.random.default_rng(47)
    yc, zc = st.pixel_centres()
    Y, Z = np.meshgrid(yc, zc, indexing="ij")
    for _ in range(60):
        ey, ez, t = rng.uniform(-330, 330), rng.uniform(-260, 260), rng.uniform(-1.0, 1.0)
        _, bq = oracle.kernel_batch(st, ey, ez, t, Y, Z)
        inside = bq <= 9.0
        hy, hz = oracle.bbox(st, t, ez)
        assert np.all(np.abs(Y[inside] - ey) <= hy * (1 + 1e-12))
        assert np.all(np.abs(Z[inside] - ez) <= hz * (1 + 1e-12))


def test_sigma_gradient_with_kappa_matches_differences():
    """d L / d sigma_z with respect to the base sigma_z (each event's own
    sigma_z scales with it), windows frozen, against Richardson-extrapolated
    central differences of L."""
    w = make_workload("adjoint_2mm", n_events=3000)
    ev = [e.astype(np.float64) for e in w.events()]
    base = Setup.from_workload(w, ny=70, nz=50)
    st = Setup(**{**base.__dict__, "sigma_z": 14.0, "sigma_dl": 55.0,
                  "wsigma_z": 14.0, "wsigma_dl": 55.0, "kappa_z": 0.2})
    s = oracle.sensitivity(st)
    rho, _ = oracle.mlem(Setup(**{**base.__dict__, "kappa_z": 0.2}), ev, 3, s=s)
    _, _, gs = oracle.loglik_grad(st, ev, rho, s=s, want_rho=False)
    _, _, gs0 = oracle.loglik_grad(Setup(**{**st.__dict__, "kappa_z": 0.0}), ev, rho, s=s,
                                   want_rho=False)
    for k, name in enumerate(("sigma_z", "sigma_dl")):
        v = getattr(st, name)

        def fd(h):
            sp = Setup(**{**st.__dict__, name: v + h})
            sm = Setup(**{**st.__dict__, name: v - h})
            Lp = oracle.loglik_grad(sp, ev, rho, s=s, want_rho=False, want_sigma=False)[0]
            Lm = oracle.loglik_grad(sm, ev, rho, s=s, want_rho=False, want_sigma=False)[0]
            return (Lp - Lm) / (2 * h)
        h = 1e-3 * v
        est = (4.0 * fd(0.5 * h) - fd(h)) / 3.0
        assert gs[k] == pytest.approx(est, rel=1e-7)
        assert abs(gs[k]) > 1.0
    # the z dependence changes the sigma_z gradient (the check is not vacuous)
    assert abs(gs[0] - gs0[0]) > 1e-3 * abs(gs0[0])
