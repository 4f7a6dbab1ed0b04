"""FP64 CPU oracle (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``oracle.c`` (plain C, double
precision, OpenMP over events) through ctypes and shares nothing with the CUDA
library.  ``bruteforce.py`` is a second, independent NumPy statement of the same
update for tiny inputs.

Parity status: every function here is pinned by a ``-m "not gpu"`` test against
something other than itself (closed forms, exact quadrature of the kernel's
defining integral, invariants of the MLEM update, brute force, finite
differences); see tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so with gcc (FP64, no
    fast-math, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and \
            os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(C.Structure):
    _fields_ = [
        ("R", C.c_double), ("L", C.c_double),
        ("ny", C.c_int32), ("nz", C.c_int32),
        ("dy", C.c_double), ("dz", C.c_double),
        ("sigma_z", C.c_double), ("sigma_dl", C.c_double), ("gamma", C.c_double),
        ("cut", C.c_double),
        ("wsigma_z", C.c_double), ("wsigma_dl", C.c_double),
        ("pscale", C.c_double),
        ("a3_printed", C.c_int32), ("form_p", C.c_int32), ("n_threads", C.c_int32),
        ("pad_", C.c_int32), ("kappa_z", C.c_double),
    ]


class Stats(C.Structure):
    _fields_ = [("n_used", C.c_int64), ("n_empty", C.c_int64), ("n_window", C.c_int64),
                ("n_qbad", C.c_int64), ("sum_s_rho", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d = C.c_double
        P = C.POINTER
        dp = P(C.c_double)
        _lib.orc_direct.argtypes = [P(Params), d, d, d, dp, dp, dp]
        _lib.orc_delta_l.argtypes = [P(Params), d, d, d, d]
        _lib.orc_delta_l.restype = d
        _lib.orc_sensitivity_at.argtypes = [P(Params), d, d]
        _lib.orc_sensitivity_at.restype = d
        _lib.orc_sensitivity.argtypes = [P(Params), dp]
        _lib.orc_kernel.argtypes = [P(Params), d, d, d, d, d, dp]
        _lib.orc_kernel.restype = d
        _lib.orc_kernel_batch.argtypes = [P(Params), C.c_int64, dp, dp, dp, dp, dp, dp, dp]
        _lib.orc_kernel_dlog.argtypes = [P(Params), d, d, d, d, d, dp]
        _lib.orc_bbox.argtypes = [P(Params), d, d, dp, dp]
        _lib.orc_mlem.argtypes = [P(Params), dp, dp, dp, C.c_int64, dp, dp, C.c_int,
                                  dp, P(Stats)]
        _lib.orc_mlem.restype = C.c_int
        _lib.orc_denominators.argtypes = [P(Params), dp, dp, dp, C.c_int64, dp, dp, dp,
                                          P(C.c_int64)]
        _lib.orc_update_at_pixels.argtypes = [P(Params), dp, dp, dp, C.c_int64, dp, dp,
                                              P(C.c_int64), C.c_int32, dp]
        _lib.orc_update_at_pixels.restype = C.c_int
        _lib.orc_loglik_grad.argtypes = [P(Params), dp, dp, dp, C.c_int64, dp, dp, dp, dp, dp]
        _lib.orc_loglik_grad.restype = C.c_int
        _lib.orc_direct_image.argtypes = [P(Params), dp, dp, dp, C.c_int64, dp]
    return _lib


@dataclass
class Setup:
    """Geometry, grid and resolution of one reconstruction (mirrors Params)."""
    R: float
    L: float
    ny: int
    nz: int
    sigma_z: float
    sigma_dl: float
    cut: float = 3.0
    gamma: float = 0.0
    wsigma_z: float = 0.0
    wsigma_dl: float = 0.0
    pscale: float = 1.0
    a3_printed: bool = False
    form_p: bool = False
    n_threads: int = 0
    kappa_z: float = 0.0

    @property
    def dy(self):
        return 2.0 * self.R / self.ny

    @property
    def dz(self):
        return self.L / self.nz

    @classmethod
    def from_workload(cls, w, **kw):
        base = dict(R=w.R, L=w.L, ny=w.ny, nz=w.nz, sigma_z=w.sigma_z, sigma_dl=w.sigma_dl,
                    cut=w.cut)
        base.update(kw)
        return cls(**base)

    def params(self) -> Params:
        return Params(self.R, self.L, self.ny, self.nz, self.dy, self.dz, self.sigma_z,
                      self.sigma_dl, self.gamma, self.cut, self.wsigma_z, self.wsigma_dl,
                      self.pscale, int(self.a3_printed), int(self.form_p), int(self.n_threads), 0,
                      self.kappa_z)

    def pixel_centres(self):
        yc = -self.R + (np.arange(self.ny) + 0.5) * self.dy
        zc = -0.5 * self.L + (np.arange(self.nz) + 0.5) * self.dz
        return yc, zc


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def direct(st: Setup, zu, zd, dl):
    """Eq. 2 for one event: (y, z, tan theta)."""
    y, z, t = C.c_double(), C.c_double(), C.c_double()
    p = st.params()
    lib().orc_direct(C.byref(p), float(zu), float(zd), float(dl), C.byref(y), C.byref(z),
                     C.byref(t))
    return y.value, z.value, t.value


def delta_l(st: Setup, y, z, zu, zd) -> float:
    p = st.params()
    return lib().orc_delta_l(C.byref(p), float(y), float(z), float(zu), float(zd))


def sensitivity_at(st: Setup, y, z) -> float:
    p = st.params()
    return lib().orc_sensitivity_at(C.byref(p), float(y), float(z))


def sensitivity(st: Setup) -> np.ndarray:
    s = np.zeros(st.ny * st.nz, dtype=np.float64)
    p = st.params()
    lib().orc_sensitivity(C.byref(p), _dp(s))
    return s.reshape(st.ny, st.nz)


def kernel(st: Setup, ey, ez, t, py, pz):
    """Eq. kernel for an event reconstructed at (ey, ez, tan theta = t) and a
    pixel centre (py, pz).  Returns (P, bC^-1b)."""
    bq = C.c_double()
    p = st.params()
    v = lib().orc_kernel(C.byref(p), float(ey), float(ez), float(t), float(py), float(pz),
                         C.byref(bq))
    return v, bq.value


def kernel_batch(st: Setup, ey, ez, t, py, pz):
    """Vectorised ``kernel``: arrays (P, bC^-1b) over broadcast inputs."""
    arrs = np.broadcast_arrays(*(np.asarray(a, dtype=np.float64) for a in (ey, ez, t, py, pz)))
    shape = arrs[0].shape
    arrs = [np.ascontiguousarray(a.ravel()) for a in arrs]
    n = arrs[0].size
    P = np.zeros(n)
    bq = np.zeros(n)
    p = st.params()
    lib().orc_kernel_batch(C.byref(p), n, *(_dp(a) for a in arrs), _dp(P), _dp(bq))
    return P.reshape(shape), bq.reshape(shape)


def kernel_dlog(st: Setup, ey, ez, t, py, pz):
    out = np.zeros(2)
    p = st.params()
    lib().orc_kernel_dlog(C.byref(p), float(ey), float(ez), float(t), float(py), float(pz),
                          _dp(out))
    return out


def bbox(st: Setup, t, ez: float = 0.0):
    """App. B half-extents (hy, hz) of the window of an event at z~ = ez."""
    hy, hz = C.c_double(), C.c_double()
    p = st.params()
    lib().orc_bbox(C.byref(p), float(ez), float(t), C.byref(hy), C.byref(hz))
    return hy.value, hz.value


def mlem(st: Setup, events: Sequence[np.ndarray], n_iter: int, rho0=None, s=None,
         return_loglik: bool = False):
    """Run n_iter updates of Eq. iter (or Eq. iter-p when st.form_p) from rho0
    (default all ones).  Returns (rho, stats[, loglik per iteration])."""
    zu, zd, dl = (_f64(e) for e in events)
    n = zu.size
    if s is None:
        s = sensitivity(st)
    s = _f64(s).ravel()
    rho = np.ones(st.ny * st.nz) if rho0 is None else _f64(rho0).ravel().copy()
    ll = np.zeros(max(n_iter, 1))
    stats = Stats()
    p = st.params()
    rc = lib().orc_mlem(C.byref(p), _dp(zu), _dp(zd), _dp(dl), n, _dp(s), _dp(rho), n_iter,
                        _dp(ll), C.byref(stats))
    if rc != 0:
        raise MemoryError("oracle mlem failed")
    out = (rho.reshape(st.ny, st.nz), stats)
    if return_loglik:
        out = out + (ll[:n_iter],)
    return out


def denominators(st: Setup, events, rho, s=None):
    zu, zd, dl = (_f64(e) for e in events)
    n = zu.size
    if s is None:
        s = sensitivity(st)
    s = _f64(s).ravel()
    rho = _f64(rho).ravel()
    D = np.zeros(n)
    cnt = np.zeros(n, dtype=np.int64)
    p = st.params()
    lib().orc_denominators(C.byref(p), _dp(zu), _dp(zd), _dp(dl), n, _dp(s), _dp(rho), _dp(D),
                           cnt.ctypes.data_as(C.POINTER(C.c_int64)))
    return D, cnt


def direct_image(st: Setup, events) -> np.ndarray:
    """Counts of the events' direct reconstructions (Eq. 2) per pixel, (ny, nz)."""
    zu, zd, dl = (_f64(e) for e in events)
    out = np.zeros(st.ny * st.nz)
    p = st.params()
    lib().orc_direct_image(C.byref(p), _dp(zu), _dp(zd), _dp(dl), zu.size, _dp(out))
    return out.reshape(st.ny, st.nz)


def update_at_pixels(st: Setup, events, rho, pixels, s=None):
    """rho^(t+1) of Eq. iter at the listed flat pixel indices only."""
    zu, zd, dl = (_f64(e) for e in events)
    n = zu.size
    if s is None:
        s = sensitivity(st)
    s = _f64(s).ravel()
    rho = _f64(rho).ravel()
    pix = np.ascontiguousarray(np.asarray(pixels, dtype=np.int64))
    out = np.zeros(pix.size)
    p = st.params()
    rc = lib().orc_update_at_pixels(C.byref(p), _dp(zu), _dp(zd), _dp(dl), n, _dp(s), _dp(rho),
                                    pix.ctypes.data_as(C.POINTER(C.c_int64)), pix.size,
                                    _dp(out))
    if rc != 0:
        raise MemoryError("oracle update_at_pixels failed")
    return out


def loglik_grad(st: Setup, events, rho, s=None, want_rho=True, want_sigma=True):
    """(L, g_rho or None, g_sigma or None) with the windows frozen at the window
    sigmas (st.wsigma_*, defaulting to the kernel's)."""
    zu, zd, dl = (_f64(e) for e in events)
    n = zu.size
    if s is None:
        s = sensitivity(st)
    s = _f64(s).ravel()
    rho = _f64(rho).ravel()
    L = C.c_double()
    g_rho = np.zeros(st.ny * st.nz) if want_rho else None
    g_sig = np.zeros(2) if want_sigma else None
    p = st.params()
    null = C.POINTER(C.c_double)()
    rc = lib().orc_loglik_grad(C.byref(p), _dp(zu), _dp(zd), _dp(dl), n, _dp(s), _dp(rho),
                               C.byref(L), _dp(g_rho) if want_rho else null,
                               _dp(g_sig) if want_sigma else null)
    if rc != 0:
        raise MemoryError("oracle loglik_grad failed")
    return L.value, (g_rho.reshape(st.ny, st.nz) if want_rho else None), g_sig
