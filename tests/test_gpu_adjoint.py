"""GPU parity of the adjoint (log-likelihood gradient) pass against the FP64
oracle, the finite-difference check, the autograd binding and the sigma fit.

Bar (adjoint workload): ||dg_rho|| / ||g_rho|| <= 1e-4 and
g_sigma within 1e-3 relative at sigma = (14, 55) mm; an Adam fit of sigma from
(14, 55) lands within 0.5% of the FP64 oracle's maximum-likelihood sigma on
the same data, and within 2% of the true (10, 42).
"""
import numpy as np
import pytest

import oracle
from oracle import Setup
from synth import make_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def prob():
    from paper_1502_07478_gb300 import Recon
    w = make_workload("adjoint_2mm", n_events=200_000)
    ev = w.events()
    r = Recon.from_workload(w)
    r.upload_events(*ev)
    r.iterate(5)
    rho = r.read_image().cpu().numpy().astype(np.float64)
    return w, ev, r, rho


def test_gradient_matches_oracle(prob):
    w, ev, r, rho = prob
    r.set_sigma(14.0, 55.0)
    r.set_image(rho.astype(np.float32))
    L, g, gs = r.loglik_grad()
    st = Setup.from_workload(w, sigma_z=14.0, sigma_dl=55.0)
    Lref, gref, gsref = oracle.loglik_grad(st, ev, rho)
    g = g.cpu().numpy().astype(np.float64)
    assert L == pytest.approx(Lref, rel=1e-6)
    assert np.linalg.norm(g - gref) / np.linalg.norm(gref) <= 1e-4
    np.testing.assert_allclose(gs, gsref, rtol=1e-3)
    r.set_sigma(w.sigma_z, w.sigma_dl)


def test_gradient_with_gamma_matches_oracle(prob):
    """The adjoint pass with the cross term gamma of C^-1 (the log-determinant
    term of d log P / d sigma changes; Q and aC^-1b gain gamma terms)."""
    from paper_1502_07478_gb300 import Recon
    w, ev, _, rho = prob
    gm = 5e-4
    r = Recon.from_workload(w, gamma=gm)
    r.upload_events(*ev)
    r.set_sigma(14.0, 55.0)
    r.set_image(rho.astype(np.float32))
    L, g, gs = r.loglik_grad()
    r.close()
    st = Setup.from_workload(w, sigma_z=14.0, sigma_dl=55.0, gamma=gm)
    Lref, gref, gsref = oracle.loglik_grad(st, ev, rho)
    g = g.cpu().numpy().astype(np.float64).ravel()
    gref = np.asarray(gref).ravel()
    assert L == pytest.approx(Lref, rel=1e-6)
    assert np.linalg.norm(g - gref) / np.linalg.norm(gref) <= 1e-4
    np.testing.assert_allclose(gs, gsref, rtol=1e-3)


def test_gradient_with_kappa_matches_oracle(prob):
    """The adjoint pass with sigma_z growing towards the strip ends (Sec. 3,
    kappa_z = 1, the largest accepted): every event's log-determinant terms
    follow its own sigma_z, and g_sigma is with respect to the base sigma_z.
    The events of this workload lie mostly within the middle half of the
    strips, so the profile moves L and g_sigma by a few 1e-4 to 1e-3 relative:
    the change itself is compared with the oracle's."""
    from paper_1502_07478_gb300 import Recon
    w, ev, r0, rho = prob
    kz = 1.0
    r = Recon.from_workload(w, kappa_z=kz)
    r.upload_events(*ev)
    r.set_sigma(14.0, 55.0)
    r.set_image(rho.astype(np.float32))
    L, g, gs = r.loglik_grad()
    r.close()
    r0.set_sigma(14.0, 55.0)
    r0.set_image(rho.astype(np.float32))
    L0, _, gs0 = r0.loglik_grad(want_rho=False)
    r0.set_sigma(w.sigma_z, w.sigma_dl)
    st = Setup.from_workload(w, sigma_z=14.0, sigma_dl=55.0, kappa_z=kz)
    Lref, gref, gsref = oracle.loglik_grad(st, ev, rho)
    Lref0, gref0, gsref0 = oracle.loglik_grad(
        Setup.from_workload(w, sigma_z=14.0, sigma_dl=55.0), ev, rho)
    g = g.cpu().numpy().astype(np.float64).ravel()
    gref, gref0 = np.asarray(gref).ravel(), np.asarray(gref0).ravel()
    assert L == pytest.approx(Lref, rel=1e-6)
    assert np.linalg.norm(g - gref) / np.linalg.norm(gref) <= 1e-4
    np.testing.assert_allclose(gs, gsref, rtol=1e-3)
    # the profile's effect, well above the tolerances above ...
    assert abs(Lref - Lref0) > 10 * 1e-6 * abs(Lref0)
    assert np.linalg.norm(gref - gref0) > 10 * 1e-4 * np.linalg.norm(gref0)
    # ... and reproduced: the GPU's change of L and g_sigma follows the oracle's
    assert (L - L0) == pytest.approx(Lref - Lref0, rel=0.05)
    np.testing.assert_allclose(np.asarray(gs) - np.asarray(gs0),
                               np.asarray(gsref) - np.asarray(gsref0), rtol=0.1,
                               atol=2e-5 * np.abs(gsref0).max())


def test_sigma_gradient_matches_fp64_differences(prob):
    """GPU g_sigma against FP64 central differences of the oracle's L (h = 1e-3
    relative, windows frozen at the base sigma)."""
    w, ev, r, rho = prob
    r.set_sigma(14.0, 55.0)
    r.set_image(rho.astype(np.float32))
    _, _, gs = r.loglik_grad(want_rho=False)
    base = dict(sigma_z=14.0, sigma_dl=55.0, wsigma_z=14.0, wsigma_dl=55.0)
    for k, name in enumerate(("sigma_z", "sigma_dl")):
        v = base[name]
        h = 1e-3 * v
        Lp = oracle.loglik_grad(Setup.from_workload(w, **{**base, name: v + h}), ev, rho,
                                want_rho=False, want_sigma=False)[0]
        Lm = oracle.loglik_grad(Setup.from_workload(w, **{**base, name: v - h}), ev, rho,
                                want_rho=False, want_sigma=False)[0]
        assert gs[k] == pytest.approx((Lp - Lm) / (2 * h), rel=1e-3)
    r.set_sigma(w.sigma_z, w.sigma_dl)


def test_autograd_function(prob):
    import torch
    from paper_1502_07478_gb300 import LogLik
    w, ev, r, rho = prob
    rho_t = torch.tensor(rho, dtype=torch.float32, device="cuda", requires_grad=True)
    sig = torch.tensor([14.0, 55.0], dtype=torch.float64, requires_grad=True)
    L = LogLik.apply(r, rho_t, sig)
    L.backward()
    r.set_image(rho.astype(np.float32))
    L2, g, gs = r.loglik_grad()
    assert float(L.detach()) == pytest.approx(L2, rel=1e-9)
    torch.testing.assert_close(rho_t.grad, g, rtol=1e-6, atol=1e-6 * float(g.abs().max()))
    np.testing.assert_allclose(sig.grad.numpy(), gs, rtol=1e-9)
    r.set_sigma(w.sigma_z, w.sigma_dl)


def _mle_module():
    import importlib.util
    import os
    spec = importlib.util.spec_from_file_location(
        "sigma_mle", os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                  "sigma_mle.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _adam_fit(w, ev, rho_np, steps=500):
    """Adam on -L/N over (log sigma_z, log sigma_dl) from (14, 55) mm, lr 1e-2
    decayed to 1e-4 over the steps; returns the fitted sigma and the context."""
    import torch
    from paper_1502_07478_gb300 import LogLik, Recon
    r = Recon.from_workload(w)
    r.upload_events(*ev)
    rho = torch.tensor(rho_np, dtype=torch.float32, device="cuda")
    logsig = torch.tensor(np.log([14.0, 55.0]), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([logsig], lr=1e-2)
    sched = torch.optim.lr_scheduler.ExponentialLR(opt, gamma=0.01 ** (1 / steps))
    for _ in range(steps):
        opt.zero_grad()
        loss = -LogLik.apply(r, rho, torch.exp(logsig)) / w.n_events
        loss.backward()
        opt.step()
        sched.step()
    return torch.exp(logsig).detach().numpy(), r, rho


def test_adam_sigma_full_adjoint_workload():
    """The same fit on all 1e6 events of the adjoint workload, against the
    oracle's maximiser on those events (tests/golden/sigma_mle.py 1000000).
    There the model's own bias is resolved: the oracle's maximum lies at
    -2.3% (sigma_z) and +1.9% (sigma_dl) from the simulated (10, 42) mm with a
    statistical spread of 0.6% and 0.2%, so the fit is held to the oracle
    (0.5%) and to the truth only within 2.5%."""
    m = _mle_module()
    w, ev, rho_np = m.fit_data(1_000_000)
    gold = m.read_golden(1_000_000)
    sig, r, _ = _adam_fit(w, ev, rho_np)
    r.close()
    print("fitted sigma", sig, "oracle maximiser", gold["sigma_z"], gold["sigma_dl"])
    assert abs(sig[0] / gold["sigma_z"] - 1) < 0.005, sig
    assert abs(sig[1] / gold["sigma_dl"] - 1) < 0.005, sig
    assert abs(sig[0] / w.sigma_z - 1) < 0.025, sig
    assert abs(sig[1] / w.sigma_dl - 1) < 0.025, sig


def test_adam_recovers_sigma():
    """Fit (log sigma_z, log sigma_dl) by Adam on -L with rho held at the true
    phantom (rasterised at pixel centres, scaled so that sum s rho = N), on the
    sigma-fit data of tests/golden/sigma_mle.py (the first 1e5 events of the
    adjoint workload, windows of 5 sigma rebuilt at every sigma, from
    (14, 55) mm).

    The bar is the FP64 oracle's own maximiser of the same likelihood on the
    same data (stored by tests/golden/sigma_mle.py, re-derived by
    tests/test_oracle_sigma_mle.py): the GPU fit lies within 0.5% of it, which
    separates the kernels' error from the model's.  On these 1e5 events that
    maximiser is -1.6% / +1.0% from the simulated (10, 42) mm (the model's bias
    plus a statistical spread of 1.9% / 0.6%), so the fit also recovers the
    truth within 2% here; the full workload resolves the bias (next test).

    5-sigma windows: with 3-sigma windows the truncated kernel loses about 1%
    of its mass and the gradient at fixed windows is biased towards smaller
    sigma (the fit then runs away)."""
    m = _mle_module()
    w, ev, rho_np = m.fit_data()
    gold = m.read_golden()
    sig, r, rho = _adam_fit(w, ev, rho_np)
    print("fitted sigma", sig, "oracle maximiser", gold["sigma_z"], gold["sigma_dl"])
    assert abs(sig[0] / gold["sigma_z"] - 1) < 0.005, sig
    assert abs(sig[1] / gold["sigma_dl"] - 1) < 0.005, sig
    assert abs(sig[0] / w.sigma_z - 1) < 0.02, sig
    assert abs(sig[1] / w.sigma_dl - 1) < 0.02, sig
    # converged: the gradient at the fitted point is small
    r.set_sigma(float(sig[0]), float(sig[1]))
    r.set_image(rho)
    _, _, gs = r.loglik_grad(want_rho=False)
    assert np.all(np.abs(gs * sig) / w.n_events < 1e-3), gs
    r.close()
