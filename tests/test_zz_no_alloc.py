"""The allocation-free MLEM update, tsp_mlem_update_noalloc.

It serves callers that cannot allocate device memory (a fixed budget handed out
by a host framework, real-time loops, plug-ins).  It must give what the
context-based entry point gives: one update of Eq. iter, here compared with
tsp_iterate(1) on two calls in a row, within the tolerance of the other GPU
tests.  The file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-4


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _rel_err(a, b, frac=0.01):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    mask = b > frac * b.max()
    return float(np.max(np.abs(a[mask] - b[mask]) / b[mask]))


def test_noalloc_update_matches_iterate():
    import torch
    from paper_1502_07478_gb300 import Recon
    from paper_1502_07478_gb300 import _lib as L
    from synth import make_workload

    # 150k events: two full chunks of 65536 and a ragged tail
    w = make_workload("paper_1mm", n_events=150_000)
    ev = w.events()
    r = Recon.from_workload(w)
    r.upload_events(*ev)
    s = r.compute_sensitivity()
    dev_ev = [torch.from_numpy(e).cuda() for e in ev]
    rho = torch.ones(w.ny, w.nz, dtype=torch.float32, device="cuda")
    out = torch.empty_like(rho)
    lib = L.lib()
    err = C.create_string_buffer(256)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        rc = lib.tsp_mlem_update_noalloc(C.byref(r.params), *(_ptr(e) for e in dev_ev),
                                         len(ev[0]), _ptr(s), _ptr(rho), _ptr(out), stream, err,
                                         len(err))
        assert rc == 0, err.value
        r.iterate(1)
        ref = r.read_image()
        torch.cuda.synchronize()
        assert float(out.sum()) > 0.0
        assert _rel_err(out, ref) <= TOL
        rho, out = out, rho          # the next call starts from this call's output


def test_noalloc_update_with_kappa_matches_iterate():
    """The same with sigma_z growing towards the strip ends (kappa_z = 0.3)."""
    import torch
    from paper_1502_07478_gb300 import Recon
    from paper_1502_07478_gb300 import _lib as L
    from synth import make_workload

    w = make_workload("small_5mm")
    ev = w.events()
    r = Recon.from_workload(w, kappa_z=0.3)
    r.upload_events(*ev)
    s = r.compute_sensitivity()
    dev_ev = [torch.from_numpy(e).cuda() for e in ev]
    rho = torch.ones(w.ny, w.nz, dtype=torch.float32, device="cuda")
    out = torch.empty_like(rho)
    err = C.create_string_buffer(256)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.lib().tsp_mlem_update_noalloc(C.byref(r.params), *(_ptr(e) for e in dev_ev),
                                         len(ev[0]), _ptr(s), _ptr(rho), _ptr(out), stream,
                                         err, len(err))
    assert rc == 0, err.value
    r.iterate(1)
    ref = r.read_image()
    torch.cuda.synchronize()
    assert _rel_err(out, ref) <= TOL
    r.close()


def test_noalloc_rejects_images_beyond_the_scratch():
    import torch
    from paper_1502_07478_gb300 import _lib as L

    lib = L.lib()
    p = L.Params(350.0, 500.0, 2048, 1024, 0.0, 0.0, 10.0, 42.0, 3.0, 0, 0)
    buf = torch.ones(4, device="cuda")
    err = C.create_string_buffer(256)
    rc = lib.tsp_mlem_update_noalloc(C.byref(p), _ptr(buf), _ptr(buf), _ptr(buf), 0, _ptr(buf),
                                     _ptr(buf), _ptr(buf[2:]), None, err, len(err))
    assert rc == L.TSP_EINVAL
    assert b"exceeds" in err.value
