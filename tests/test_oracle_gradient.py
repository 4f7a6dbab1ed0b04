"""Pins of the oracle's log-likelihood gradient against FP64 central differences.

L(rho, sigma) = sum_j log D_j - sum_i s_i rho_i, the list-mode Poisson
log-likelihood whose EM step is Eq. iter.  Windows are frozen at the base sigma
(reading R14) for both the analytic gradient and the differences.
"""
import numpy as np
import pytest

import oracle
from oracle import Setup
from synth import make_workload


@pytest.fixture(scope="module")
def prob():
    w = make_workload("adjoint_2mm", n_events=3000)
    ev = [e.astype(np.float64) for e in w.events()]
    base = Setup.from_workload(w, ny=70, nz=50)      # 10 mm pixels keep this fast
    st = Setup(**{**base.__dict__, "sigma_z": 14.0, "sigma_dl": 55.0,
                  "wsigma_z": 14.0, "wsigma_dl": 55.0})
    s = oracle.sensitivity(st)
    rho, _ = oracle.mlem(Setup.from_workload(w, ny=70, nz=50), ev, 3, s=s)
    return st, ev, s, rho


def test_rho_gradient_matches_differences(prob):
    st, ev, s, rho = prob
    _, g, _ = oracle.loglik_grad(st, ev, rho, s=s, want_sigma=False)
    flat = rho.ravel()
    support = np.nonzero(flat > 1e-2 * flat.max())[0]
    for l in support[np.linspace(0, support.size - 1, 6).astype(int)]:
        # Central differences at steps h and h/2 combined by Richardson
        # extrapolation: a step of a few percent keeps the rounding of L (about
        # 4e4 here) small, the extrapolation removes the h^2 truncation term.
        def fd(h):
            rp = flat.copy(); rp[l] += h
            rm = flat.copy(); rm[l] -= h
            Lp = oracle.loglik_grad(st, ev, rp, s=s, want_rho=False, want_sigma=False)[0]
            Lm = oracle.loglik_grad(st, ev, rm, s=s, want_rho=False, want_sigma=False)[0]
            return (Lp - Lm) / (2 * h)
        h = 0.1 * flat[l]
        est = (4.0 * fd(0.5 * h) - fd(h)) / 3.0
        assert g.ravel()[l] == pytest.approx(est, rel=1e-6)


def test_sigma_gradient_matches_differences(prob):
    st, ev, s, rho = prob
    _, _, gs = oracle.loglik_grad(st, ev, rho, s=s, want_rho=False)
    for k, name in enumerate(("sigma_z", "sigma_dl")):
        v = getattr(st, name)

        def fd(h):
            sp = Setup(**{**st.__dict__, name: v + h})
            sm = Setup(**{**st.__dict__, name: v - h})
            Lp = oracle.loglik_grad(sp, ev, rho, s=s, want_rho=False, want_sigma=False)[0]
            Lm = oracle.loglik_grad(sm, ev, rho, s=s, want_rho=False, want_sigma=False)[0]
            return (Lp - Lm) / (2 * h)
        # h = 1e-3 relative, plus Richardson extrapolation with h/2 to remove the
        # h^2 term (about 1e-6 relative on its own)
        h = 1e-3 * v
        est = (4.0 * fd(0.5 * h) - fd(h)) / 3.0
        assert gs[k] == pytest.approx(est, rel=1e-7)
        assert gs[k] == pytest.approx(fd(h), rel=1e-5)
        assert abs(gs[k]) > 1.0  # far from the optimum, the check is not vacuous


def test_rho_gradient_is_s_times_backprojection_minus_one(prob):
    """dL/drho = s (A - 1) with A the MLEM back-projection: at a fixed point of
    Eq. iter, rho_l (A_l - 1) = 0."""
    st, ev, s, rho = prob
    st0 = Setup(**{**st.__dict__, "sigma_z": st.wsigma_z, "sigma_dl": st.wsigma_dl})
    _, g, _ = oracle.loglik_grad(st0, ev, rho, s=s, want_sigma=False)
    rho1, _ = oracle.mlem(st0, ev, 1, rho0=rho, s=s)
    A = np.where(rho > 0, rho1 / np.where(rho > 0, rho, 1.0), 0.0)
    mask = rho > 1e-6 * rho.max()
    np.testing.assert_allclose(g[mask], (s * (A - 1.0))[mask], rtol=1e-9, atol=1e-9)
