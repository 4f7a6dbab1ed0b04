"""Streamed (chunked) event upload and the fine-grid path.

A streamed upload (tsp_begin_events / tsp_append_events / tsp_end_events) must
give the reconstruction of a single upload of the concatenated chunks, from
host arrays, pinned host tensors or device tensors.  On the 0.5 mm grid of the
stress workload the window halo is too large to stage both rho' and the
accumulator; the tiles stage only the accumulator, read rho' from global
memory and split each row over two lanes, and must still match the FP64 oracle.
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


@pytest.fixture(scope="module")
def prob():
    w = make_workload("adjoint_2mm", n_events=60_000)
    return w, w.events()


def _single(w, ev, n_iter):
    from paper_1502_07478_gb300 import Recon
    r = Recon.from_workload(w)
    r.upload_events(*ev)
    r.iterate(n_iter)
    img = r.read_image().cpu().numpy()
    st = r.stats()
    r.close()
    return img, st


@pytest.mark.parametrize("kind", ["numpy", "pinned", "cuda"])
def test_streamed_equals_single_upload(prob, kind):
    import torch
    from paper_1502_07478_gb300 import Recon
    w, ev = prob
    ref, st_ref = _single(w, ev, 3)
    r = Recon.from_workload(w)
    n = len(ev[0])
    cuts = [0, 7_000, 31_000, n]
    r.begin_events(n)
    for a, b in zip(cuts[:-1], cuts[1:]):
        chunk = [x[a:b] for x in ev]
        if kind == "pinned":
            chunk = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory() for x in chunk]
        elif kind == "cuda":
            chunk = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in chunk]
        r.append_events(*chunk)
    r.end_events()
    r.iterate(3)
    img = r.read_image().cpu().numpy()
    st = r.stats()
    r.close()
    assert st["n_events"] == n
    assert st["n_window"] == st_ref["n_window"]
    assert st["n_used"] == st_ref["n_used"]
    assert rel_err(img, ref.astype(np.float64)) <= 1e-5


def test_streamed_upload_state_errors(prob):
    from paper_1502_07478_gb300 import Recon, TspError
    from paper_1502_07478_gb300._lib import TSP_EINVAL, TSP_ESTATE
    w, ev = prob
    r = Recon.from_workload(w)
    with pytest.raises(TspError) as ei:
        r.append_events(*[x[:10] for x in ev])
    assert ei.value.code == TSP_ESTATE
    r.begin_events(100)
    r.append_events(*[x[:60] for x in ev])
    with pytest.raises(TspError) as ei:
        r.append_events(*[x[:60] for x in ev])
    assert ei.value.code == TSP_EINVAL
    with pytest.raises(TspError) as ei:
        r.iterate(1)
    assert ei.value.code == TSP_ESTATE
    with pytest.raises(TspError) as ei:
        r.set_sigma(12.0, 40.0)
    assert ei.value.code == TSP_ESTATE
    r.append_events(*[x[60:100] for x in ev])
    r.end_events()
    r.iterate(1)
    assert r.stats()["n_events"] == 100
    with pytest.raises(TspError) as ei:
        r.end_events()
    assert ei.value.code == TSP_ESTATE
    r.close()


def test_fine_grid_accumulator_tiles_match_oracle():
    """0.5 mm pixels (1400 x 1000): accumulator-only tiles."""
    w = make_workload("stress_05mm", n_events=3000)
    ev = w.events()
    from paper_1502_07478_gb300 import Recon
    r = Recon.from_workload(w)
    r.upload_events(*ev)
    r.iterate(3)
    img = r.read_image().cpu().numpy()
    st = r.stats()
    r.close()
    assert st["n_outliers"] < 0.05 * st["n_events"]
    assert st["n_clipped"] == 0 and st["n_qbad"] == 0
    ref, rst = oracle.mlem(Setup.from_workload(w), ev, 3)
    assert st["n_used"] == rst.n_used
    assert rel_err(img, ref) <= TOL
