"""Parity at the workloads' full sizes, in the launch configuration the
benchmark times.  The FP64 oracle cannot run these reconstructions whole, but
one MLEM update is local: rho^(t+1) at pixel l needs only rho^t and the events
whose window holds l.  So each test takes the GPU image rho^t, applies one GPU
update, and compares the result at sampled pixels (above 1% of the maximum,
seeded) with the oracle's update of the same rho^t at those pixels
(max relative error <= 1e-4), plus the properties that hold at any size:
count conservation sum_l s_l rho_l = N_used and rho >= 0.  The adjoint workload
(1e6 events, 2 mm) is small enough for the whole oracle gradient.
"""
import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle
from oracle import Setup
from synth import batched_instances, make_workload

pytestmark = pytest.mark.gpu

TOL = 1e-4


def _pool():
    return cf.ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 4),
                                  mp_context=mp.get_context("spawn"))


def _chunk(args):
    name, n_events, k, chunk = args
    return make_workload(name, n_events=n_events).event_chunk(k, chunk)


def _batch_events(args):
    k, i = args
    return batched_instances(k, seed=3)[i].events()


def _sample_pixels(rho, n, seed):
    rng = np.random.default_rng(seed)
    flat = rho.ravel()
    cand = np.nonzero(flat > 0.01 * flat.max())[0]
    pick = rng.choice(cand, size=min(n, cand.size), replace=False)
    return np.unique(np.concatenate([pick, [int(np.argmax(flat))]]))


def _check_update(st, events, rho_t, rho_t1, pixels, s=None):
    ref = oracle.update_at_pixels(st, events, rho_t.astype(np.float64), pixels, s=s)
    got = rho_t1.ravel()[pixels].astype(np.float64)
    err = np.max(np.abs(got - ref) / ref)
    assert err <= TOL, (err, pixels[np.argmax(np.abs(got - ref) / ref)])
    return err


def _conservation(r):
    s = r.compute_sensitivity().double()
    rho = r.read_image().double()
    st = r.stats()
    assert float(rho.min()) >= 0.0
    assert float((s * rho).sum()) == pytest.approx(st["n_used"], rel=1e-5)


@pytest.mark.timeout(1200)
def test_paper_scale_1mm_sampled_update():
    """1e7 events, 700 x 500 at 1 mm: iterations 2 -> 3 of the benchmark's
    reconstruction (plain form, default schedule, graph replay)."""
    from paper_1502_07478_gb300 import Recon
    w = make_workload("paper_1mm")
    ev = w.events()
    r = Recon.from_workload(w)
    r.upload_events(*ev)
    r.iterate(2)
    rho2 = r.read_image().cpu().numpy()
    r.iterate(1)
    rho3 = r.read_image().cpu().numpy()
    _conservation(r)
    r.close()
    pix = _sample_pixels(rho3, 1, seed=11)
    _check_update(Setup.from_workload(w), ev, rho2, rho3, pix)


@pytest.mark.timeout(1200)
def test_batched_64_sampled_update():
    """The 64 reconstructions of the batched workload (2.4e7 events) in one
    batch with the autotuned schedule: the first update at the hottest pixel of
    every fourth reconstruction, conservation in all of them."""
    from paper_1502_07478_gb300 import Batch
    ws = batched_instances(64, seed=3)
    with _pool() as ex:
        evs = list(ex.map(_batch_events, [(64, i) for i in range(64)]))
    b = Batch.from_workloads(ws)
    for i, ev in enumerate(evs):
        b.upload_events(i, *ev)
    b.autotune()
    b.iterate(1)
    for i, (w, ev) in enumerate(zip(ws, evs)):
        rho1 = b.read_image(i).cpu().numpy()
        if i % 4 == 0:
            pix = _sample_pixels(rho1, 0, seed=100 + i)
            _check_update(Setup.from_workload(w), ev, np.ones_like(rho1), rho1, pix)
        st = b.stats(i)
        assert st["sum_s_rho"] == pytest.approx(st["n_used"], rel=1e-5)
    b.close()


@pytest.mark.timeout(1200)
def test_adjoint_full_gradient():
    """1e6 events, 350 x 250 at 2 mm: the whole gradient at sigma = (14, 55)
    against the FP64 oracle."""
    from paper_1502_07478_gb300 import Recon
    w = make_workload("adjoint_2mm")
    ev = w.events()
    r = Recon.from_workload(w)
    r.upload_events(*ev)
    r.iterate(5)
    rho = r.read_image().cpu().numpy().astype(np.float64)
    r.set_sigma(14.0, 55.0)
    L, g, gs = r.loglik_grad()
    r.close()
    Lref, gref, gsref = oracle.loglik_grad(Setup.from_workload(w, sigma_z=14.0, sigma_dl=55.0),
                                           ev, rho)
    g = g.cpu().numpy().astype(np.float64).ravel()
    gref = np.asarray(gref).ravel()
    assert L == pytest.approx(Lref, rel=1e-6)
    assert np.linalg.norm(g - gref) / np.linalg.norm(gref) <= 1e-4
    np.testing.assert_allclose(gs, gsref, rtol=1e-3)


@pytest.mark.timeout(1200)
def test_stress_05mm_streamed_full_size():
    """1e8 events streamed in ten 1e7-event pinned chunks, 1400 x 1000 at
    0.5 mm (accumulator-only tiles), two iterations: the properties that hold
    at any size (the oracle's per-pixel update over 1e8 events is too slow to
    sample here; the next test samples it on one chunk)."""
    import torch
    from paper_1502_07478_gb300 import Recon
    w = make_workload("stress_05mm")
    chunk = 10_000_000
    sizes = w.chunk_sizes(chunk)
    with _pool() as ex:
        chunks = list(ex.map(_chunk, [(w.name, w.n_events, k, chunk) for k in range(len(sizes))]))
    r = Recon.from_workload(w)
    r.begin_events(w.n_events)
    for c in chunks:
        r.append_events(*[torch.from_numpy(x).pin_memory() for x in c])
    r.end_events()
    st = r.stats()
    assert st["n_events"] == w.n_events and st["n_outliers"] < 0.01 * w.n_events
    for _ in range(2):
        r.iterate(1)
        _conservation(r)
    assert r.stats()["n_clipped"] == 0 and r.stats()["n_qbad"] == 0
    r.close()


@pytest.mark.timeout(1200)
def test_stress_05mm_one_chunk_sampled_update():
    """2e6 events of the stress workload (the start of its first streamed chunk)
    on the full 0.5 mm grid, streamed in two pieces: iterations 1 -> 2 at one
    sampled pixel and the hottest one."""
    from paper_1502_07478_gb300 import Recon
    w = make_workload("stress_05mm")
    ev = tuple(x[:2_000_000] for x in w.event_chunk(0, 10_000_000))
    r = Recon.from_workload(w)
    n = len(ev[0])
    r.begin_events(n)
    r.append_events(*[x[: n // 3] for x in ev])
    r.append_events(*[x[n // 3:] for x in ev])
    r.end_events()
    r.iterate(1)
    rho1 = r.read_image().cpu().numpy()
    r.iterate(1)
    rho2 = r.read_image().cpu().numpy()
    _conservation(r)
    r.close()
    pix = _sample_pixels(rho2, 1, seed=5)
    _check_update(Setup.from_workload(w), ev, rho1, rho2, pix)
