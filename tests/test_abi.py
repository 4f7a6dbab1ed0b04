"""The C ABI library: it loads without a GPU, exports every entry point that
include/tsp.h declares, and rejects bad arguments before touching the device."""
import ctypes as C
import os
import re

import pytest

from paper_1502_07478_gb300 import _lib as L
from paper_1502_07478_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build()
    return L.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "tsp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tsp_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["tsp_create", "tsp_destroy", "tsp_upload_events", "tsp_compute_sensitivity",
              "tsp_set_image", "tsp_iterate", "tsp_read_image", "tsp_loglik", "tsp_loglik_grad",
              "tsp_set_sigma", "tsp_stats", "tsp_last_error", "tsp_version"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for n in _declared():
        assert hasattr(lib, n), n
    declared = set(_declared())
    bound = {name for name, _, _ in L.SIGNATURES}
    assert declared == bound


def test_struct_layouts_match_header():
    assert C.sizeof(L.Params) == 8 * 2 + 4 * 2 + 8 * 5 + 4 * 2 + 8 + 8
    assert C.sizeof(L.Stats) == 8 * 11
    assert C.sizeof(L.Schedule) == 4 * 4


def test_version(lib):
    assert lib.tsp_version().decode().startswith("tsp ")


def _params(**kw):
    base = dict(R=350.0, L=500.0, ny=140, nz=100, dy=0.0, dz=0.0, sigma_z=10.0,
                sigma_dl=42.0, cut=3.0, flags=0, reserved=0, gamma=0.0, kappa_z=0.0)
    base.update(kw)
    return L.Params(**base)


@pytest.mark.parametrize("bad", [dict(R=0.0), dict(L=-1.0), dict(ny=0), dict(nz=-3),
                                 dict(sigma_z=0.0), dict(sigma_dl=float("nan")),
                                 dict(cut=-1.0), dict(flags=1), dict(dy=-1.0),
                                 dict(gamma=float("nan")), dict(gamma=2e-3),
                                 dict(kappa_z=-0.1), dict(kappa_z=1.5),
                                 dict(kappa_z=float("inf")),
                                 dict(gamma=1.4e-3, kappa_z=0.5)])
def test_create_rejects_bad_params(lib, bad):
    h = C.c_void_p(123)
    p = _params(**bad)
    rc = lib.tsp_create(C.byref(p), C.byref(h))
    assert rc == L.TSP_EINVAL
    assert h.value is None
    assert lib.tsp_last_error(None)


def test_null_arguments(lib):
    h = C.c_void_p()
    assert lib.tsp_create(None, C.byref(h)) == L.TSP_EINVAL
    assert lib.tsp_create(C.byref(_params()), None) == L.TSP_EINVAL
    lib.tsp_destroy(None)
    assert lib.tsp_iterate(None, 1, None) == L.TSP_EINVAL
    assert lib.tsp_upload_events(None, None, None, None, 0, 0, None) == L.TSP_EINVAL


def test_batch_rejects_bad_params(lib):
    h = C.c_void_p(123)
    ps = (L.Params * 3)(_params(), _params(ny=0), _params())
    assert lib.tsp_batch_create(ps, 3, C.byref(h)) == L.TSP_EINVAL
    assert h.value is None
    assert b"reconstruction 1" in lib.tsp_batch_last_error(None)
    assert lib.tsp_batch_create(ps, 0, C.byref(h)) == L.TSP_EINVAL
    assert lib.tsp_batch_create(None, 2, C.byref(h)) == L.TSP_EINVAL
    assert lib.tsp_batch_create(ps, 1, None) == L.TSP_EINVAL


def test_batch_null_arguments(lib):
    lib.tsp_batch_destroy(None)
    assert lib.tsp_batch_size(None) == 0
    assert lib.tsp_batch_iterate(None, 1, None) == L.TSP_EINVAL
    assert lib.tsp_batch_upload_events(None, 0, None, None, None, 0, 0, None) == L.TSP_EINVAL
    assert lib.tsp_batch_loglik_grad(None, None, None, None) == L.TSP_EINVAL
    assert lib.tsp_batch_autotune(None, None, None, None) == L.TSP_EINVAL
    s = L.Schedule(128, 8, 0, 0)
    assert lib.tsp_batch_set_schedule(None, C.byref(s), None) == L.TSP_EINVAL
    assert lib.tsp_set_schedule(None, C.byref(s), None) == L.TSP_EINVAL
    assert lib.tsp_autotune(None, None, None, None) == L.TSP_EINVAL
