"""Pins of the oracle's event kernel (Eq. kernel, Sec. 3).

The kernel is a Laplace approximation of the exact detection density
    P_exact(e|i) = (1/pi) int dtheta N(e; e_i(theta), C),
e_i(theta) = (z + (R - y) tan, z - (R + y) tan, -2 y sec) (Eq. 1 geometry).
That integral is computed here by adaptive quadrature, independently of the
vectors o, a, b.  The normalisation is checked by integrating P over the
measurement space through the change of variables given by Eq. 2.
"""
import numpy as np
import pytest
from scipy.integrate import quad

import oracle
from oracle import Setup


def _setup(scale=1.0, **kw):
    return Setup(R=350.0, L=500.0, ny=140, nz=100, sigma_z=10.0 * scale,
                 sigma_dl=42.0 * scale, **kw)


def _cinv(st):
    iz, il, g = st.sigma_z ** -2, st.sigma_dl ** -2, st.gamma
    return np.array([[iz, 0.0, g], [0.0, iz, -g], [g, -g, il]])


def _exact(st, ev, py, pz):
    Ci = _cinv(st)
    norm = np.sqrt(np.linalg.det(Ci)) / (2 * np.pi) ** 1.5 / np.pi
    R = st.R
    e_meas = np.asarray(ev)

    def f(th):
        e = np.array([pz + (R - py) * np.tan(th), pz - (R + py) * np.tan(th),
                      -2.0 * py / np.cos(th)])
        d = e - e_meas
        return norm * np.exp(-0.5 * d @ Ci @ d)

    _, _, t = oracle.direct(st, *ev)
    v, _ = quad(f, -0.5 * np.pi, 0.5 * np.pi, points=[np.arctan(t)], limit=400,
                epsabs=0.0, epsrel=1e-11)
    return v


def _laplace_errors(st, n=160, seed=31):
    rng = np.random.default_rng(seed)
    errs = []
    while len(errs) < n:
        py = rng.uniform(-300.0, 300.0)
        pz = rng.uniform(-200.0, 200.0)
        th = rng.uniform(-0.6, 0.6)
        ev = (pz + (st.R - py) * np.tan(th) + rng.normal() * st.sigma_z,
              pz - (st.R + py) * np.tan(th) + rng.normal() * st.sigma_z,
              -2.0 * py / np.cos(th) + rng.normal() * st.sigma_dl)
        ey, ez, t = oracle.direct(st, *ev)
        P, bq = oracle.kernel(st, ey, ez, t, py, pz)
        if bq > st.cut ** 2:
            continue
        errs.append(P / _exact(st, ev, py, pz) - 1.0)
    return np.abs(np.array(errs))


@pytest.fixture(scope="module")
def laplace_err():
    return {(sc, a3p): _laplace_errors(_setup(sc, a3_printed=a3p))
            for sc in (1.0, 0.5, 0.25) for a3p in (False, True)}


def test_kernel_matches_exact_quadrature(laplace_err):
    """Inside the 3-sigma windows the Laplace kernel is within a few percent of the
    exact integral at the paper's resolution (mean under 1%, worst at the window
    edge under 10%)."""
    e = laplace_err[(1.0, False)]
    assert e.mean() < 0.01 and np.percentile(e, 90) < 0.025 and e.max() < 0.10


def test_kernel_error_shrinks_with_sigma(laplace_err):
    """The Laplace error vanishes in proportion to sigma as the resolution sharpens."""
    e1, e2, e4 = (laplace_err[(sc, False)] for sc in (1.0, 0.5, 0.25))
    assert e2.mean() < 0.6 * e1.mean() and e4.mean() < 0.6 * e2.mean()
    assert e4.max() < 0.5 * e1.max()


def test_derived_a3_beats_printed(laplace_err):
    """Reading R3: with a_3 = -2 y tan sec (the derivative of -2 y sec) the kernel
    converges to the exact integral as sigma shrinks; with the printed -y tan sec
    an error of about half a percent remains."""
    for sc in (1.0, 0.5, 0.25):
        assert laplace_err[(sc, False)].mean() < laplace_err[(sc, True)].mean()
    assert laplace_err[(0.25, False)].mean() < 0.4 * laplace_err[(0.25, True)].mean()
    assert laplace_err[(0.25, True)].mean() > 0.6 * laplace_err[(0.5, True)].mean()


def _integral_over_measurements(st, py, pz, th_max=1.2, n=(61, 61, 121)):
    """int P(e|i) de over the events reconstructed with |theta~| <= th_max, using
    the Eq. 2 map (y~, z~, tan theta~) -> (z_u, z_d, delta_l) and its Jacobian."""
    R = st.R
    th = np.linspace(-th_max, th_max, n[2])
    sy, su = st.sigma_dl / 2.0, st.sigma_z / np.sqrt(2.0)
    dY = np.linspace(-8 * sy, 8 * sy, n[0])
    U = np.linspace(-8 * su, 8 * su, n[1])
    DY, UU, TH = np.meshgrid(dY, U, th, indexing="ij")
    T = np.tan(TH)
    ey = py - DY
    ez = pz - (UU + T * DY)
    P, _ = oracle.kernel_batch(st, ey, ez, T, py, pz)
    sec = np.sqrt(1.0 + T * T)
    J = np.empty(DY.shape + (3, 3))
    J[..., 0, :] = np.stack([-T, np.ones_like(T), R - ey], -1)
    J[..., 1, :] = np.stack([-T, np.ones_like(T), -(R + ey)], -1)
    J[..., 2, :] = np.stack([-2.0 * sec, np.zeros_like(T), -2.0 * ey * T / sec], -1)
    f = P * np.abs(np.linalg.det(J)) * sec ** 2   # d tan = sec^2 d theta
    return np.trapezoid(np.trapezoid(np.trapezoid(f, th, axis=2), U, axis=1), dY, axis=0)


@pytest.mark.parametrize("py,pz", [(0.0, 0.0), (100.0, 50.0), (-200.0, -100.0),
                                   (300.0, 200.0)])
def test_kernel_normalisation(py, pz):
    """Reading R4: with det^(1/2)(C^-1)/(2 pi^2) the kernel is a probability
    density over the measurements; events with |theta~| <= 1.2 carry mass 2.4/pi.
    The small deficit away from the centre is the Laplace error and falls as
    sigma^2."""
    devs = []
    for sc in (1.0, 0.5):
        st = _setup(sc, cut=1e6)
        devs.append(abs(_integral_over_measurements(st, py, pz) / (2.4 / np.pi) - 1.0))
    assert devs[0] < 1e-3
    assert devs[1] <= 0.3 * devs[0] + 1e-12


def test_window_quantity_ignores_gamma_and_cut():
    """b has equal first two components, so the gamma terms of C^-1 cancel in
    b C^-1 b; the cut changes only membership, never the kernel's value."""
    st0 = _setup()
    st1 = _setup(gamma=1e-3)
    st2 = _setup(cut=5.0)
    for args in [(10.0, 5.0, 0.2, 40.0, 20.0), (-100.0, 30.0, -0.5, -80.0, 0.0)]:
        P0, b0 = oracle.kernel(st0, *args)
        _, b1 = oracle.kernel(st1, *args)
        P2, _ = oracle.kernel(st2, *args)
        assert b1 == pytest.approx(b0, rel=1e-13)
        assert P2 == P0


def test_q_positive_inside_windows():
    """Reading R5's guard never fires at the workloads' resolution."""
    st = _setup()
    rng = np.random.default_rng(5)
    ey = rng.uniform(-340, 340, 20000)
    ez = rng.uniform(-250, 250, 20000)
    t = rng.uniform(-0.8, 0.8, 20000)
    py = ey + rng.uniform(-63, 63, 20000)
    pz = ez + rng.uniform(-45, 45, 20000)
    P, bq = oracle.kernel_batch(st, ey, ez, t, py, pz)
    inside = bq <= 9.0
    assert inside.sum() > 1000
    assert np.all(P[inside] > 0.0)


def test_dlog_sigma_matches_finite_differences():
    st = _setup(1.0)
    h = 1e-4
    for args in [(10.0, 5.0, 0.2, 40.0, 20.0), (-100.0, 30.0, -0.5, -80.0, 0.0),
                 (250.0, -100.0, 0.6, 270.0, -60.0)]:
        g = oracle.kernel_dlog(st, *args)
        for k, name in enumerate(("sigma_z", "sigma_dl")):
            sp = _setup(1.0)
            sm = _setup(1.0)
            setattr(sp, name, getattr(st, name) * (1 + h))
            setattr(sm, name, getattr(st, name) * (1 - h))
            fd = (np.log(oracle.kernel(sp, *args)[0]) - np.log(oracle.kernel(sm, *args)[0])) \
                / (2 * h * getattr(st, name))
            assert g[k] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_kernel_with_gamma_matches_exact_quadrature():
    """With the cross term gamma of C^-1 (Sec. 3) the Laplace kernel follows the
    exact theta-integral of the correlated Gaussian as closely as the diagonal
    kernel does, while differing from the diagonal kernel by far more (so the
    gamma terms of aC^-1a, oC^-1b and aC^-1b are exercised)."""
    st0 = _setup()
    g = 0.5 * np.sqrt(st0.sigma_z ** -2 * st0.sigma_dl ** -2 / 2.0)   # det(C^-1) > 0
    st = _setup(gamma=g)
    rng = np.random.default_rng(41)
    errs, shifts = [], []
    while len(errs) < 60:
        py = rng.uniform(-300.0, 300.0)
        pz = rng.uniform(-200.0, 200.0)
        th = rng.uniform(-0.6, 0.6)
        ev = (pz + (st.R - py) * np.tan(th) + rng.normal() * st.sigma_z,
              pz - (st.R + py) * np.tan(th) + rng.normal() * st.sigma_z,
              -2.0 * py / np.cos(th) + rng.normal() * st.sigma_dl)
        ey, ez, t = oracle.direct(st, *ev)
        P, bq = oracle.kernel(st, ey, ez, t, py, pz)
        if bq > st.cut ** 2:
            continue
        P0, _ = oracle.kernel(st0, ey, ez, t, py, pz)
        errs.append(abs(P / _exact(st, ev, py, pz) - 1.0))
        shifts.append(abs(P / P0 - 1.0))
    errs, shifts = np.array(errs), np.array(shifts)
    assert errs.mean() < 0.01 and np.percentile(errs, 90) < 0.025
    assert np.median(shifts) > 5 * np.median(errs)
