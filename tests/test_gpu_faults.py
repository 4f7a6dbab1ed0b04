"""Error paths of the C ABI under host-side fault injection (TSP_SIM_FAULT).

No device fault is made: the library simulates an exhausted allocator
(``oom``), a failed kernel launch before anything is enqueued (``launch``),
corrupt input (``nan_event``, a NaN written into the uploaded z_u) or a
bounded wait that gives up (``timeout``).  Each test
checks the return code and message, that the failed context can still be
destroyed without leaking device memory, and that a fresh context works
afterwards.
"""
import os

import numpy as np
import pytest

from synth import make_workload

pytestmark = pytest.mark.gpu

# device memory is handed out in pages; a leak of any image-sized buffer of
# these workloads is far larger than this slack
SLACK = 4 << 20


@pytest.fixture()
def fault():
    """Set TSP_SIM_FAULT for the duration of a block; always unset after."""
    def set_(kind):
        if kind is None:
            os.environ.pop("TSP_SIM_FAULT", None)
        else:
            os.environ["TSP_SIM_FAULT"] = kind
    yield set_
    os.environ.pop("TSP_SIM_FAULT", None)


def _free():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def _works(w, ev):
    """A fresh context reconstructs and conserves counts."""
    from paper_1502_07478_gb300 import Recon
    r = Recon.from_workload(w)
    r.upload_events(*ev)
    r.iterate(2)
    st = r.stats()
    r.close()
    assert st["n_used"] > 0
    assert st["sum_s_rho"] == pytest.approx(st["n_used"], rel=2e-6)


@pytest.fixture(scope="module")
def small():
    w = make_workload("small_5mm", n_events=5000)
    ev = w.events()
    _works(w, ev)                       # load the library and warm the allocator
    return w, ev


def test_oom_at_create(small, fault):
    from paper_1502_07478_gb300 import Recon, TspError
    from paper_1502_07478_gb300._lib import TSP_ENOMEM
    w, ev = small
    base = _free()
    fault("oom")
    with pytest.raises(TspError) as ei:
        Recon.from_workload(w)
    assert ei.value.code == TSP_ENOMEM
    assert "memory" in str(ei.value)
    fault(None)
    assert _free() >= base - SLACK
    _works(w, ev)


def test_oom_at_upload_then_destroy(small, fault):
    from paper_1502_07478_gb300 import Recon, TspError
    from paper_1502_07478_gb300._lib import TSP_ENOMEM
    w, ev = small
    base = _free()
    r = Recon.from_workload(w)
    fault("oom")
    with pytest.raises(TspError) as ei:
        r.upload_events(*ev)
    assert ei.value.code == TSP_ENOMEM
    fault(None)
    # the same context recovers: its event buffers are allocated again
    r.upload_events(*ev)
    r.iterate(1)
    st = r.stats()
    assert st["sum_s_rho"] == pytest.approx(st["n_used"], rel=2e-6)
    r.close()
    assert _free() >= base - SLACK
    _works(w, ev)


def test_launch_failure_at_iterate(small, fault):
    from paper_1502_07478_gb300 import Recon, TspError
    from paper_1502_07478_gb300._lib import TSP_ECUDA
    w, ev = small
    base = _free()
    r = Recon.from_workload(w)
    r.upload_events(*ev)
    fault("launch")
    with pytest.raises(TspError) as ei:
        r.iterate(3)
    assert ei.value.code == TSP_ECUDA
    assert "graph capture" in str(ei.value)
    with pytest.raises(TspError) as ei:
        r.loglik()
    assert ei.value.code == TSP_ECUDA
    fault(None)
    r.close()
    assert _free() >= base - SLACK
    _works(w, ev)


def test_launch_failure_at_upload(small, fault):
    from paper_1502_07478_gb300 import Recon, TspError
    from paper_1502_07478_gb300._lib import TSP_ECUDA
    w, ev = small
    r = Recon.from_workload(w)
    fault("launch")
    with pytest.raises(TspError) as ei:
        r.upload_events(*ev)
    assert ei.value.code == TSP_ECUDA
    fault(None)
    r.close()
    _works(w, ev)


def test_nan_event_rejected(small, fault):
    from paper_1502_07478_gb300 import Recon, TspError
    from paper_1502_07478_gb300._lib import TSP_EINVAL, TSP_ESTATE
    w, ev = small
    r = Recon.from_workload(w)
    fault("nan_event")
    with pytest.raises(TspError) as ei:
        r.upload_events(*ev)
    assert ei.value.code == TSP_EINVAL
    assert "not finite" in str(ei.value)
    # nothing usable was uploaded
    with pytest.raises(TspError) as ei:
        r.iterate(1)
    assert ei.value.code == TSP_ESTATE
    fault(None)
    # an input error leaves the context usable
    r.upload_events(*ev)
    r.iterate(2)
    st = r.stats()
    assert st["n_events"] == len(ev[0])
    assert st["sum_s_rho"] == pytest.approx(st["n_used"], rel=2e-6)
    r.close()


def test_batch_oom_at_create(small, fault):
    from paper_1502_07478_gb300 import Batch, TspError
    from paper_1502_07478_gb300._lib import TSP_ENOMEM
    w, ev = small
    base = _free()
    fault("oom")
    with pytest.raises(TspError) as ei:
        Batch.from_workloads([w, w])
    assert ei.value.code == TSP_ENOMEM
    fault(None)
    assert _free() >= base - SLACK
    b = Batch.from_workloads([w, w])
    for i in range(2):
        b.upload_events(i, *ev)
    b.iterate(1)
    assert b.stats(1)["sum_s_rho"] == pytest.approx(b.stats(1)["n_used"], rel=2e-6)
    b.close()


def test_simulated_timeout(small, fault):
    """TSP_SIM_FAULT=timeout: tsp_wait returns TSP_ETIMEOUT at once with its
    message; the queued work still completes and the context stays usable."""
    from paper_1502_07478_gb300 import Recon
    from paper_1502_07478_gb300._lib import TSP_ETIMEOUT, lib
    w, ev = small
    r = Recon.from_workload(w)
    r.upload_events(*ev)
    r.iterate(1)
    fault("timeout")
    assert r.wait(60_000) is False
    assert lib().tsp_wait(r._h, None, 60_000) == TSP_ETIMEOUT
    assert b"simulated" in lib().tsp_last_error(r._h)
    fault(None)
    assert r.wait(60_000) is True
    r.iterate(2)
    st = r.stats()
    assert st["sum_s_rho"] == pytest.approx(st["n_used"], rel=2e-6)
    r.close()
