"""Pins of the oracle's MLEM update (Eq. iter, Eq. iter-p; Listing 1)."""
import numpy as np
import pytest

import oracle
from oracle import Setup
from synth import make_workload


@pytest.fixture(scope="module")
def small():
    w = make_workload("small_5mm")
    ev = [e[:4000].astype(np.float64) for e in w.events()]
    st = Setup.from_workload(w)
    return st, ev, oracle.sensitivity(st)


def test_count_conservation_each_iteration(small):
    """sum_l s_l rho_l^(t+1) = sum_j sum_l s_l P_jl rho_l / D_j = N_used."""
    st, ev, s = small
    rho = None
    for _ in range(4):
        rho, stats = oracle.mlem(st, ev, 1, rho0=rho, s=s)
        assert stats.n_used + stats.n_empty == len(ev[0])
        assert float((s * rho).sum()) == pytest.approx(stats.n_used, rel=1e-12)
        assert stats.sum_s_rho == pytest.approx(stats.n_used, rel=1e-12)
        assert np.all(rho >= 0.0)


def test_loglik_non_decreasing(small):
    """EM never decreases the likelihood."""
    st, ev, s = small
    _, _, ll = oracle.mlem(st, ev, 8, s=s, return_loglik=True)
    assert np.all(np.diff(ll) >= -1e-9 * np.abs(ll[1:]))
    assert ll[-1] > ll[0]


def test_constant_factor_cancels(small):
    st, ev, s = small
    rho1, _ = oracle.mlem(st, ev, 3, s=s)
    st2 = Setup(**{**st.__dict__, "pscale": 37.5})
    rho2, _ = oracle.mlem(st2, ev, 3, s=s)
    np.testing.assert_allclose(rho2, rho1, rtol=1e-12, atol=0)


def test_iter_p_form_is_s_times_rho(small):
    """Eq. iter-p on rho' = s rho reproduces Eq. iter."""
    st, ev, s = small
    rho, _ = oracle.mlem(st, ev, 3, s=s)
    stp = Setup(**{**st.__dict__, "form_p": True})
    rhop, _ = oracle.mlem(stp, ev, 3, rho0=s, s=s)
    np.testing.assert_allclose(rhop, s * rho, rtol=1e-11, atol=1e-300)


def test_single_event_closed_form(small):
    """One event from rho^0 = 1: rho^1_l = P_l / sum_i P_i s_i on its window."""
    st, ev, s = small
    one = [e[5:6] for e in ev]
    rho, stats = oracle.mlem(st, one, 1, s=s)
    ey, ez, t = oracle.direct(st, one[0][0], one[1][0], one[2][0])
    yc, zc = st.pixel_centres()
    Y, Z = np.meshgrid(yc, zc, indexing="ij")
    P, bq = oracle.kernel_batch(st, ey, ez, t, Y, Z)
    P = np.where(bq <= 9.0, P, 0.0)
    np.testing.assert_allclose(rho, P / (P * s).sum(), rtol=1e-12, atol=1e-300)
    assert stats.n_used == 1


def test_events_outside_the_image_are_skipped(small):
    """An event reconstructed beyond the grid has an empty window (D = 0)."""
    st, ev, s = small
    far = [np.concatenate([e[:100], np.array([x])]) for e, x in zip(ev, (0.0, 0.0, -2000.0))]
    rho, stats = oracle.mlem(st, far, 1, s=s)
    assert stats.n_empty == 1 and stats.n_used == 100
    assert float((s * rho).sum()) == pytest.approx(100.0, rel=1e-12)


def test_update_at_pixels_matches_full_update(small):
    st, ev, s = small
    rho0, _ = oracle.mlem(st, ev, 2, s=s)
    rho1, _ = oracle.mlem(st, ev, 1, rho0=rho0, s=s)
    # scattered pixels, a repeated one, and a compact 4 x 4 patch
    patch = [(60 + a) * 100 + 40 + b for a in range(4) for b in range(4)]
    pix = np.array([0, 777, 7050, 7051, 13999, 5000, 777] + patch)
    got = oracle.update_at_pixels(st, ev, rho0, pix, s=s)
    np.testing.assert_allclose(got, rho1.ravel()[pix], rtol=1e-12, atol=1e-300)


def test_denominators_give_the_loglik(small):
    st, ev, s = small
    rho, _ = oracle.mlem(st, ev, 2, s=s)
    D, cnt = oracle.denominators(st, ev, rho, s=s)
    L, _, _ = oracle.loglik_grad(st, ev, rho, s=s, want_rho=False, want_sigma=False)
    assert L == pytest.approx(np.log(D[D > 0]).sum() - (s * rho).sum(), rel=1e-12)
    _, _, ll = oracle.mlem(st, ev, 1, rho0=rho, s=s, return_loglik=True)
    assert ll[0] == pytest.approx(L, rel=1e-12)
    assert np.all(cnt > 0)
