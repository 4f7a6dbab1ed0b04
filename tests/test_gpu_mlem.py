"""GPU parity of the MLEM path (through the C ABI) against the FP64 oracle.

Bar: max relative error <= 1e-4 on pixels above 1% of the
image maximum, same seeded FP32 events on both sides.
"""
import numpy as np
import pytest

import oracle
from oracle import Setup
from synth import make_workload

pytestmark = pytest.mark.gpu

TOL = 1e-4


def rel_err(gpu, ref, frac=0.01):
    gpu = np.asarray(gpu, dtype=np.float64).reshape(ref.shape)
    mask = ref > frac * ref.max()
    return float(np.max(np.abs(gpu[mask] - ref[mask]) / ref[mask]))


def _recon(w, **kw):
    from paper_1502_07478_gb300 import Recon
    return Recon.from_workload(w, **kw)


def _run_gpu(w, ev, n_iter, rho0=None):
    r = _recon(w)
    r.upload_events(*ev)
    if rho0 is not None:
        r.set_image(rho0)
    r.iterate(n_iter)
    img = r.read_image(out=np.empty((w.ny, w.nz), np.float32))
    st = r.stats()
    r.close()
    assert st["n_clipped"] == 0 and st["n_qbad"] == 0
    return img, st


@pytest.fixture(scope="module")
def small():
    w = make_workload("small_5mm")
    return w, w.events()


def test_sensitivity_matches_oracle(small):
    w, _ = small
    r = _recon(w)
    s = r.compute_sensitivity().cpu().numpy()
    ref = oracle.sensitivity(Setup.from_workload(w))
    np.testing.assert_allclose(s, ref, rtol=2e-7, atol=1e-9)


@pytest.mark.parametrize("n_iter", [1, 5, 10])
def test_small_5mm_parity(small, n_iter):
    """5 mm pixels, 2e4 events (the full small workload)."""
    w, ev = small
    img, st = _run_gpu(w, ev, n_iter)
    ref, rst = oracle.mlem(Setup.from_workload(w), ev, n_iter)
    assert rel_err(img, ref) <= TOL
    assert st["n_used"] == rst.n_used
    assert st["n_empty"] == rst.n_empty


def test_conservation_each_iteration(small):
    """sum_l s_l rho_l^(t+1) = N_used after every update."""
    w, ev = small
    r = _recon(w)
    r.upload_events(*ev)
    s = r.compute_sensitivity().double()
    for _ in range(4):
        r.iterate(1)
        st = r.stats()
        rho = r.read_image().double()
        assert float((s * rho).sum()) == pytest.approx(st["n_used"], rel=2e-6)
        assert st["sum_s_rho"] == pytest.approx(st["n_used"], rel=2e-6)
        assert float(rho.min()) >= 0.0


@pytest.mark.parametrize("name,n,iters", [("paper_1mm", 20000, 10), ("adjoint_2mm", 50000, 10)])
def test_finer_grids_parity(name, n, iters):
    """1 mm and 2 mm grids on a subset of events: several tiles, ragged tails."""
    w = make_workload(name, n_events=n)
    ev = w.events()
    img, st = _run_gpu(w, ev, iters)
    ref, rst = oracle.mlem(Setup.from_workload(w), ev, iters)
    assert rel_err(img, ref) <= TOL
    assert st["n_used"] == rst.n_used


def test_outlier_path_parity():
    """Steep events (|tan theta~| up to 2) overflow their tile halo and take the
    global-memory path; results must not change."""
    w = make_workload("small_5mm", n_events=3000)
    zu, zd, dl = w.events()
    rng = np.random.default_rng(8)
    k = 600
    y = rng.uniform(-150, 150, k)
    z = rng.uniform(-100, 100, k)
    t = rng.uniform(1.2, 2.0, k) * rng.choice([-1, 1], k)
    zu2 = (z + (350 - y) * t).astype(np.float32)
    zd2 = (z - (350 + y) * t).astype(np.float32)
    dl2 = (-2 * y * np.sqrt(1 + t * t)).astype(np.float32)
    ev = (np.concatenate([zu, zu2]), np.concatenate([zd, zd2]), np.concatenate([dl, dl2]))
    img, st = _run_gpu(w, ev, 3)
    assert st["n_outliers"] > 0
    ref, _ = oracle.mlem(Setup.from_workload(w), ev, 3)
    assert rel_err(img, ref) <= TOL


def test_empty_event_list(small):
    w, _ = small
    e = np.zeros(0, np.float32)
    img, st = _run_gpu(w, (e, e, e), 2)
    assert st["n_events"] == 0 and st["n_used"] == 0
    assert np.all(img == 0.0)


def test_events_outside_the_grid_are_empty(small):
    w, ev = small
    k = 50
    far = (np.zeros(k, np.float32), np.zeros(k, np.float32), np.full(k, -5000.0, np.float32))
    ev2 = tuple(np.concatenate([a[:200], b]) for a, b in zip(ev, far))
    img, st = _run_gpu(w, ev2, 2)
    ref, rst = oracle.mlem(Setup.from_workload(w), ev2, 2)
    assert st["n_empty"] == k == rst.n_empty
    assert rel_err(img, ref) <= TOL


def test_single_event(small):
    w, ev = small
    one = tuple(a[7:8] for a in ev)
    img, st = _run_gpu(w, one, 1)
    ref, _ = oracle.mlem(Setup.from_workload(w), one, 1)
    assert st["n_used"] == 1
    assert rel_err(img, ref) <= TOL


def test_nonfinite_events_rejected(small):
    from paper_1502_07478_gb300 import TspError
    w, ev = small
    bad = [a[:100].copy() for a in ev]
    bad[2][17] = np.nan
    r = _recon(w)
    with pytest.raises(TspError) as ei:
        r.upload_events(*bad)
    assert ei.value.code == -1
    with pytest.raises(TspError) as ei:
        r.iterate(1)
    assert ei.value.code == -5


def test_device_and_host_inputs_agree(small):
    import torch
    w, ev = small
    a, _ = _run_gpu(w, ev, 3)
    r = _recon(w)
    r.upload_events(*(torch.from_numpy(x).cuda() for x in ev))
    r.iterate(3)
    b = r.read_image().cpu().numpy()
    np.testing.assert_allclose(b, a, rtol=1e-5, atol=1e-7 * a.max())


def test_split_iterations_and_resume(small):
    """Checkpoint/resume: 10 straight iterations equal 5, read image, set it in a
    fresh context, 5 more (atomic summation order aside)."""
    w, ev = small
    a, _ = _run_gpu(w, ev, 10)
    r = _recon(w)
    r.upload_events(*ev)
    r.iterate(2)
    r.iterate(3)
    mid = r.read_image().cpu().numpy()
    r.close()
    b, _ = _run_gpu(w, ev, 5, rho0=mid)
    assert rel_err(b, a.astype(np.float64)) <= 1e-5


def test_read_image_rho_prime(small):
    w, ev = small
    r = _recon(w)
    r.upload_events(*ev)
    r.iterate(2)
    rho = r.read_image().cpu().numpy()
    rp = r.read_image(which=1).cpu().numpy()
    s = r.compute_sensitivity().cpu().numpy()
    np.testing.assert_allclose(rp, s * rho, rtol=1e-6, atol=0)


def test_loglik_matches_oracle(small):
    w, ev = small
    r = _recon(w)
    r.upload_events(*ev)
    r.iterate(3)
    rho = r.read_image().cpu().numpy().astype(np.float64)
    L = r.loglik()
    Lref, _, _ = oracle.loglik_grad(Setup.from_workload(w), ev, rho, want_rho=False,
                                    want_sigma=False)
    assert L == pytest.approx(Lref, rel=1e-6)


def test_direct_image_matches_oracle_exactly(small):
    """Eq. 2 histogram: integer counts, bit-exact against the oracle, from host
    and into device memory, with events outside the grid left out."""
    w, ev = small
    far = (np.zeros(40, np.float32), np.zeros(40, np.float32), np.full(40, -5000.0, np.float32))
    ev2 = tuple(np.concatenate([a, b]) for a, b in zip(ev, far))
    r = _recon(w)
    r.upload_events(*ev2)
    ref = oracle.direct_image(Setup.from_workload(w), ev2)
    host = r.direct_image(out=np.empty((w.ny, w.nz), np.float32))
    dev = r.direct_image().cpu().numpy()
    np.testing.assert_array_equal(host, ref)
    np.testing.assert_array_equal(dev, ref)
    assert ref.sum() <= len(ev2[0]) - 40
    # the iteration is unaffected by the readout (A is cleared again)
    r.iterate(2)
    img = r.read_image(out=np.empty((w.ny, w.nz), np.float32))
    ref2, _ = oracle.mlem(Setup.from_workload(w), ev2, 2)
    assert rel_err(img, ref2) <= TOL
    r.close()


def test_direct_image_paper_scale_exact():
    """The 1e7-event, 1 mm workload: every pixel count equal to the oracle's."""
    w = make_workload("paper_1mm")
    ev = w.events()
    r = _recon(w)
    r.upload_events(*ev)
    img = r.direct_image().cpu().numpy()
    r.close()
    np.testing.assert_array_equal(img, oracle.direct_image(Setup.from_workload(w), ev))


def test_thread_granularity_variant_matches_oracle(small):
    """The one-thread-per-event ablation gives the oracle's image."""
    w, ev = small
    r = _recon(w)
    r.set_variant("thread")
    r.upload_events(*ev)
    r.iterate(5)
    img = r.read_image(out=np.empty((w.ny, w.nz), np.float32))
    st = r.stats()
    r.close()
    ref, rst = oracle.mlem(Setup.from_workload(w), ev, 5)
    assert rel_err(img, ref) <= TOL
    assert st["n_used"] == rst.n_used


def test_thread_granularity_variant_matches_tiles_1mm():
    w = make_workload("paper_1mm", n_events=20_000)
    ev = w.events()
    out = []
    for v in ("tiles", "thread"):
        r = _recon(w)
        r.set_variant(v)
        r.upload_events(*ev)
        r.iterate(3)
        out.append(r.read_image(out=np.empty((w.ny, w.nz), np.float32)))
        r.close()
    assert rel_err(out[1], out[0].astype(np.float64)) <= 1e-5


def test_gamma_cross_term_parity(small):
    """C^-1 with the cross term gamma (Sec. 3): the GPU image follows the
    oracle with the same gamma, and differs from the diagonal result."""
    w, ev = small
    gm = 5e-4
    r = _recon(w, gamma=gm)
    r.upload_events(*ev)
    r.iterate(5)
    img = r.read_image(out=np.empty((w.ny, w.nz), np.float32))
    L = r.loglik()
    r.close()
    st = Setup.from_workload(w, gamma=gm)
    ref, _ = oracle.mlem(st, ev, 5)
    assert rel_err(img, ref) <= TOL
    ref0, _ = oracle.mlem(Setup.from_workload(w), ev, 5)
    assert rel_err(ref, ref0) > 100 * TOL
    Lref = oracle.loglik_grad(st, ev, img, want_rho=False, want_sigma=False)[0]
    assert L == pytest.approx(Lref, rel=1e-6)


@pytest.mark.parametrize("variant", ["tiles", "thread"])
def test_z_dependent_sigma_parity(small, variant):
    """sigma_z growing towards the strip ends (Sec. 3; kappa_z = 1, i.e. twice
    the centre's sigma_z at the ends): the GPU image follows the oracle with
    the same profile and differs from the constant-sigma result."""
    w, ev = small
    kz = 1.0
    r = _recon(w, kappa_z=kz)
    r.set_variant(variant)
    r.upload_events(*ev)
    r.iterate(5)
    img = r.read_image(out=np.empty((w.ny, w.nz), np.float32))
    L = r.loglik()
    st_gpu = r.stats()
    r.close()
    st = Setup.from_workload(w, kappa_z=kz)
    ref, rst = oracle.mlem(st, ev, 5)
    assert rel_err(img, ref) <= TOL
    assert st_gpu["n_used"] == rst.n_used
    assert st_gpu["n_window"] == rst.n_window
    ref0, _ = oracle.mlem(Setup.from_workload(w), ev, 5)
    assert rel_err(ref, ref0) > 100 * TOL
    Lref = oracle.loglik_grad(st, ev, img, want_rho=False, want_sigma=False)[0]
    assert L == pytest.approx(Lref, rel=1e-6)


def test_state_and_argument_errors(small):
    """Entry points called out of order or with bad arguments return the
    documented codes and leave the context usable."""
    from paper_1502_07478_gb300 import TspError
    from paper_1502_07478_gb300._lib import TSP_EINVAL, TSP_ESTATE
    w, ev = small
    r = _recon(w)
    for call in (lambda: r.direct_image(), lambda: r.iterate(1), lambda: r.loglik(),
                 lambda: r.autotune()):
        with pytest.raises(TspError) as ei:
            call()
        assert ei.value.code == TSP_ESTATE
    with pytest.raises(TspError) as ei:
        r._chk(r._lib.tsp_set_variant(r._h, 7))
    assert ei.value.code == TSP_EINVAL
    with pytest.raises(TspError) as ei:                 # 2 gamma^2 >= iz il after the change
        r2 = _recon(w, gamma=1.5e-3)
        r2.set_sigma(20.0, 42.0)
    assert ei.value.code == TSP_EINVAL
    with pytest.raises(TspError):
        r.set_schedule(items_per_sm=0)
    r.upload_events(*ev)
    r.begin_events(10)
    r.append_events(*[x[:0] for x in ev])               # empty chunks are accepted
    r.append_events(*[x[:10] for x in ev])
    r.end_events()
    r.iterate(1)
    assert r.stats()["n_events"] == 10
    r.close()


def test_single_reconstruction_batch_matches_plain(small):
    from paper_1502_07478_gb300 import Batch
    w, ev = small
    b = Batch.from_workloads([w])
    b.upload_events(0, *ev)
    b.iterate(4)
    img = b.read_image(0, out=np.empty((w.ny, w.nz), np.float32))
    b.close()
    ref, _ = oracle.mlem(Setup.from_workload(w), ev, 4)
    assert rel_err(img, ref) <= TOL
