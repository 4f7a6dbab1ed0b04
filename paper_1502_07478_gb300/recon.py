"""Python binding of libtsp: the same operations as include/tsp.h, with torch
tensors (device memory, streams) or NumPy arrays (host memory) as arguments.

Nothing here computes any part of the reconstruction; every call forwards to
the CUDA library.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Tuple

import numpy as np

from . import _lib as L

try:
    import torch
except ImportError:  # pragma: no cover
    torch = None


def _stream_handle(stream=None):
    if torch is None or not torch.cuda.is_available():
        return None
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _arg(x, dtype=np.float32):
    """(pointer, on_device, keepalive) for a torch tensor or array-like."""
    if torch is not None and isinstance(x, torch.Tensor):
        if x.is_cuda:
            if x.dtype != torch.float32 or not x.is_contiguous():
                x = x.to(torch.float32).contiguous()
            return C.c_void_p(x.data_ptr()), 1, x
        x = x.detach().numpy()
    a = np.ascontiguousarray(np.asarray(x, dtype=dtype))
    return C.c_void_p(a.ctypes.data), 0, a


class Recon:
    """One reconstruction: geometry, grid, resolution, events and image.

    Mirrors tsp_create / tsp_upload_events / tsp_compute_sensitivity /
    tsp_set_image / tsp_iterate / tsp_read_image / tsp_loglik /
    tsp_loglik_grad / tsp_set_sigma / tsp_stats."""

    def __init__(self, R: float, L_: float, ny: int, nz: int, sigma_z: float, sigma_dl: float,
                 cut: float = 3.0, dy: float = 0.0, dz: float = 0.0, device: Optional[int] = None,
                 gamma: float = 0.0, kappa_z: float = 0.0):
        self._lib = L.lib()
        if torch is not None and torch.cuda.is_available():
            if device is not None:
                torch.cuda.set_device(device)
            torch.cuda.init()
        self.ny, self.nz = int(ny), int(nz)
        self.params = L.Params(float(R), float(L_), self.ny, self.nz, float(dy), float(dz),
                               float(sigma_z), float(sigma_dl), float(cut), 0, 0, float(gamma),
                               float(kappa_z))
        h = C.c_void_p()
        rc = self._lib.tsp_create(C.byref(self.params), C.byref(h))
        L.check(None, rc)
        self._h = h
        self.device = torch.cuda.current_device() if torch is not None and \
            torch.cuda.is_available() else None

    @classmethod
    def from_workload(cls, w, **kw):
        return cls(w.R, w.L, w.ny, w.nz, w.sigma_z, w.sigma_dl, w.cut, **kw)

    # -- lifetime --------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.tsp_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _chk(self, rc):
        L.check(self._h, rc)

    # -- operations --------------------------------------------------------------
    def upload_events(self, zu, zd, dl, stream=None):
        pu, du, ku = _arg(zu)
        pd, dd, kd = _arg(zd)
        pl, dl_, kl = _arg(dl)
        if not (du == dd == dl_):
            raise ValueError("zu, zd, dl must all be host arrays or all be CUDA tensors")
        n = int(ku.numel() if du else ku.size)
        if (kd.numel() if dd else kd.size) != n or (kl.numel() if dl_ else kl.size) != n:
            raise ValueError("zu, zd, dl must have the same length")
        self._chk(self._lib.tsp_upload_events(self._h, pu, pd, pl, n, du, _stream_handle(stream)))

    def begin_events(self, n_total: int, stream=None):
        """Start a streamed upload of n_total events (tsp_begin_events)."""
        self._chk(self._lib.tsp_begin_events(self._h, int(n_total), _stream_handle(stream)))
        self._pending = []

    def append_events(self, zu, zd, dl, stream=None):
        """Append one chunk (host arrays, pinned CPU tensors or CUDA tensors).
        The chunk is kept alive until end_events, since the copy may still be
        in flight when this returns."""
        pu, du, ku = _arg(zu)
        pd, dd, kd = _arg(zd)
        pl, dl_, kl = _arg(dl)
        if not (du == dd == dl_):
            raise ValueError("zu, zd, dl must all be host arrays or all be CUDA tensors")
        n = int(ku.numel() if du else ku.size)
        if (kd.numel() if dd else kd.size) != n or (kl.numel() if dl_ else kl.size) != n:
            raise ValueError("zu, zd, dl must have the same length")
        self._chk(self._lib.tsp_append_events(self._h, pu, pd, pl, n, du, _stream_handle(stream)))
        getattr(self, "_pending", []).append((ku, kd, kl, zu, zd, dl))

    def end_events(self, stream=None):
        """Bin the appended events (tsp_end_events; synchronises)."""
        self._chk(self._lib.tsp_end_events(self._h, _stream_handle(stream)))
        self._pending = []

    def compute_sensitivity(self, out=None, stream=None):
        """Sensitivity map (Eq. s-yz) as a CUDA tensor (or into ``out``)."""
        if out is None:
            out = torch.empty(self.ny, self.nz, dtype=torch.float32, device="cuda")
        p, dev, keep = _arg(out)
        self._chk(self._lib.tsp_compute_sensitivity(self._h, p, dev, _stream_handle(stream)))
        return out

    def set_image(self, rho=None, stream=None):
        if rho is None:
            self._chk(self._lib.tsp_set_image(self._h, None, 0, _stream_handle(stream)))
            return
        p, dev, keep = _arg(rho)
        size = keep.numel() if dev else keep.size
        if size != self.ny * self.nz:
            raise ValueError("image must have ny*nz elements")
        self._chk(self._lib.tsp_set_image(self._h, p, dev, _stream_handle(stream)))

    def iterate(self, n_iter: int, stream=None):
        self._chk(self._lib.tsp_iterate(self._h, int(n_iter), _stream_handle(stream)))

    def read_image(self, which: int = 0, out=None, stream=None):
        """rho (which=0) or rho' = s rho (which=1) as a CUDA tensor, or into
        ``out`` (a CUDA tensor or a NumPy array)."""
        if out is None:
            out = torch.empty(self.ny, self.nz, dtype=torch.float32, device="cuda")
        if isinstance(out, np.ndarray):
            if out.dtype != np.float32 or not out.flags.c_contiguous or out.size != self.ny * self.nz:
                raise ValueError("out must be a contiguous float32 array of ny*nz elements")
            self._chk(self._lib.tsp_read_image(self._h, C.c_void_p(out.ctypes.data), int(which), 0,
                                               _stream_handle(stream)))
            return out
        p, dev, keep = _arg(out)
        if keep is not out:
            raise ValueError("out must be a contiguous float32 CUDA tensor")
        self._chk(self._lib.tsp_read_image(self._h, p, int(which), dev, _stream_handle(stream)))
        return out

    def backproject(self, out=None, stream=None):
        """Back-projection of this reconstruction's events at the current image
        (tsp_backproject): A[l] = sum_j P(e_j|l) / D_j, as a CUDA tensor or into
        ``out`` (a CUDA tensor or a NumPy array).  The image is unchanged."""
        if out is None:
            out = torch.empty(self.ny, self.nz, dtype=torch.float32, device="cuda")
        if isinstance(out, np.ndarray):
            if out.dtype != np.float32 or not out.flags.c_contiguous or out.size != self.ny * self.nz:
                raise ValueError("out must be a contiguous float32 array of ny*nz elements")
            self._chk(self._lib.tsp_backproject(self._h, C.c_void_p(out.ctypes.data), 0,
                                                _stream_handle(stream)))
            return out
        p, dev, keep = _arg(out)
        if keep is not out:
            raise ValueError("out must be a contiguous float32 CUDA tensor")
        self._chk(self._lib.tsp_backproject(self._h, p, dev, _stream_handle(stream)))
        return out

    def apply_update(self, A, stream=None):
        """rho <- rho * A (tsp_apply_update), A a CUDA tensor or host array of
        ny*nz floats, e.g. the sum of every shard's back-projection."""
        p, dev, keep = _arg(A)
        size = keep.numel() if dev else keep.size
        if size != self.ny * self.nz:
            raise ValueError("A must have ny*nz elements")
        self._chk(self._lib.tsp_apply_update(self._h, p, dev, _stream_handle(stream)))

    def wait(self, timeout_ms: int, stream=None) -> bool:
        """Wait up to timeout_ms for the work enqueued on the stream
        (tsp_wait): True when it finished, False when the limit ran out."""
        rc = self._lib.tsp_wait(self._h, _stream_handle(stream), int(timeout_ms))
        if rc == L.TSP_ETIMEOUT:
            return False
        self._chk(rc)
        return True

    def direct_image(self, out=None, stream=None):
        """Counts of the events' direct reconstructions (Eq. 2) per pixel, as a
        CUDA tensor or into ``out`` (CUDA tensor or NumPy array)."""
        if out is None:
            out = torch.empty(self.ny, self.nz, dtype=torch.float32, device="cuda")
        if isinstance(out, np.ndarray):
            if out.dtype != np.float32 or not out.flags.c_contiguous or out.size != self.ny * self.nz:
                raise ValueError("out must be a contiguous float32 array of ny*nz elements")
            self._chk(self._lib.tsp_direct_image(self._h, C.c_void_p(out.ctypes.data), 0,
                                                 _stream_handle(stream)))
            return out
        p, dev, keep = _arg(out)
        if keep is not out:
            raise ValueError("out must be a contiguous float32 CUDA tensor")
        self._chk(self._lib.tsp_direct_image(self._h, p, dev, _stream_handle(stream)))
        return out

    def loglik(self, stream=None) -> float:
        v = C.c_double()
        self._chk(self._lib.tsp_loglik(self._h, C.byref(v), _stream_handle(stream)))
        return v.value

    def loglik_grad(self, want_rho: bool = True, want_sigma: bool = True, stream=None):
        """(L, g_rho as a CUDA tensor or None, g_sigma as a length-2 array or None)."""
        v = C.c_double()
        g = torch.empty(self.ny, self.nz, dtype=torch.float32, device="cuda") if want_rho else None
        gs = (C.c_double * 2)() if want_sigma else None
        self._chk(self._lib.tsp_loglik_grad(
            self._h, C.byref(v), C.c_void_p(g.data_ptr()) if g is not None else None, 1,
            gs, _stream_handle(stream)))
        return v.value, g, (np.array([gs[0], gs[1]]) if gs is not None else None)

    def set_sigma(self, sigma_z: float, sigma_dl: float, stream=None):
        self._chk(self._lib.tsp_set_sigma(self._h, float(sigma_z), float(sigma_dl),
                                          _stream_handle(stream)))
        self.params.sigma_z = float(sigma_z)
        self.params.sigma_dl = float(sigma_dl)

    def stats(self, stream=None) -> dict:
        s = L.Stats()
        self._chk(self._lib.tsp_stats(self._h, C.byref(s), _stream_handle(stream)))
        return {k: getattr(s, k) for k, _ in L.Stats._fields_}

    def set_profiling(self, on: bool = True):
        self._chk(self._lib.tsp_set_profiling(self._h, int(bool(on))))

    def set_variant(self, variant: str = "tiles"):
        """MLEM pass of iterate(): "tiles" (default) or "thread" (one thread per
        event, the thread-granularity ablation)."""
        code = {"tiles": 0, "thread": 1}[variant]
        self._chk(self._lib.tsp_set_variant(self._h, code))

    @property
    def schedule(self) -> dict:
        s = L.Schedule()
        self._chk(self._lib.tsp_get_schedule(self._h, C.byref(s)))
        return _sched_dict(s)

    def set_schedule(self, ty_cap: int = 128, items_per_sm: int = 8, order: int = 0, stream=None):
        s = L.Schedule(int(ty_cap), int(items_per_sm), int(order), 0)
        self._chk(self._lib.tsp_set_schedule(self._h, C.byref(s), _stream_handle(stream)))

    def autotune(self, stream=None) -> Tuple[dict, float]:
        """Pick the fastest tile schedule by timing MLEM passes; returns
        (schedule, pass ms)."""
        s = L.Schedule()
        ms = C.c_float()
        self._chk(self._lib.tsp_autotune(self._h, C.byref(s), C.byref(ms), _stream_handle(stream)))
        return _sched_dict(s), ms.value

    def pass_times(self, max_count: int = 4096, stream=None):
        """Device durations (ms) of the MLEM kernel launches of the last iterate."""
        buf = (C.c_float * max_count)()
        cnt = C.c_int()
        self._chk(self._lib.tsp_pass_times(self._h, buf, max_count, C.byref(cnt),
                                           _stream_handle(stream)))
        return [buf[i] for i in range(cnt.value)]


def _sched_dict(s) -> dict:
    return {"ty_cap": s.ty_cap, "items_per_sm": s.items_per_sm, "order": s.order}


def _params(R, L_, ny, nz, sigma_z, sigma_dl, cut=3.0, dy=0.0, dz=0.0, gamma=0.0, kappa_z=0.0):
    return L.Params(float(R), float(L_), int(ny), int(nz), float(dy), float(dz), float(sigma_z),
                    float(sigma_dl), float(cut), 0, 0, float(gamma), float(kappa_z))


class Batch:
    """k independent reconstructions advanced together (tsp_batch_*): one
    persistent tile launch per iteration over the work of all of them.

    ``params`` is a sequence of dicts with the keys of ``Recon`` (R, L, ny, nz,
    sigma_z, sigma_dl, optionally cut, dy, dz) or of workload objects."""

    def __init__(self, params, device: Optional[int] = None):
        self._lib = L.lib()
        if torch is not None and torch.cuda.is_available():
            if device is not None:
                torch.cuda.set_device(device)
            torch.cuda.init()
        plist = []
        for p in params:
            if not isinstance(p, dict):
                p = dict(R=p.R, L=p.L, ny=p.ny, nz=p.nz, sigma_z=p.sigma_z,
                         sigma_dl=p.sigma_dl, cut=p.cut)
            plist.append(_params(p["R"], p["L"], p["ny"], p["nz"], p["sigma_z"], p["sigma_dl"],
                                 p.get("cut", 3.0), p.get("dy", 0.0), p.get("dz", 0.0),
                                 p.get("gamma", 0.0), p.get("kappa_z", 0.0)))
        if not plist:
            raise ValueError("a batch needs at least one reconstruction")
        self.params = (L.Params * len(plist))(*plist)
        self.shapes = [(p.ny, p.nz) for p in plist]
        h = C.c_void_p()
        rc = self._lib.tsp_batch_create(self.params, len(plist), C.byref(h))
        L.check_batch(None, rc)
        self._h = h

    @classmethod
    def from_workloads(cls, ws, **kw):
        return cls(list(ws), **kw)

    def __len__(self):
        return len(self.shapes)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.tsp_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _chk(self, rc):
        L.check_batch(self._h, rc)

    def upload_events(self, i: int, zu, zd, dl, stream=None):
        pu, du, ku = _arg(zu)
        pd, dd, kd = _arg(zd)
        pl, dl_, kl = _arg(dl)
        if not (du == dd == dl_):
            raise ValueError("zu, zd, dl must all be host arrays or all be CUDA tensors")
        n = int(ku.numel() if du else ku.size)
        if (kd.numel() if dd else kd.size) != n or (kl.numel() if dl_ else kl.size) != n:
            raise ValueError("zu, zd, dl must have the same length")
        self._chk(self._lib.tsp_batch_upload_events(self._h, int(i), pu, pd, pl, n, du,
                                                    _stream_handle(stream)))

    def set_image(self, i: int, rho=None, stream=None):
        if rho is None:
            self._chk(self._lib.tsp_batch_set_image(self._h, int(i), None, 0,
                                                    _stream_handle(stream)))
            return
        p, dev, keep = _arg(rho)
        ny, nz = self.shapes[i]
        if (keep.numel() if dev else keep.size) != ny * nz:
            raise ValueError("image must have ny*nz elements")
        self._chk(self._lib.tsp_batch_set_image(self._h, int(i), p, dev, _stream_handle(stream)))

    def set_sigma(self, i: int, sigma_z: float, sigma_dl: float, stream=None):
        self._chk(self._lib.tsp_batch_set_sigma(self._h, int(i), float(sigma_z), float(sigma_dl),
                                                _stream_handle(stream)))
        self.params[i].sigma_z = float(sigma_z)
        self.params[i].sigma_dl = float(sigma_dl)

    def iterate(self, n_iter: int, stream=None):
        self._chk(self._lib.tsp_batch_iterate(self._h, int(n_iter), _stream_handle(stream)))

    def read_image(self, i: int, which: int = 0, out=None, stream=None):
        """rho (0), rho' (1) or the last g_rho (2) of reconstruction i, as a
        CUDA tensor or into ``out`` (CUDA tensor or NumPy array)."""
        ny, nz = self.shapes[i]
        if out is None:
            out = torch.empty(ny, nz, dtype=torch.float32, device="cuda")
        if isinstance(out, np.ndarray):
            if out.dtype != np.float32 or not out.flags.c_contiguous or out.size != ny * nz:
                raise ValueError("out must be a contiguous float32 array of ny*nz elements")
            self._chk(self._lib.tsp_batch_read_image(self._h, int(i), C.c_void_p(out.ctypes.data),
                                                     int(which), 0, _stream_handle(stream)))
            return out
        p, dev, keep = _arg(out)
        if keep is not out:
            raise ValueError("out must be a contiguous float32 CUDA tensor")
        self._chk(self._lib.tsp_batch_read_image(self._h, int(i), p, int(which), dev,
                                                 _stream_handle(stream)))
        return out

    def loglik_grad(self, stream=None):
        """(L, g_sigma): arrays of shape (k,) and (k, 2); g_rho of
        reconstruction i is ``read_image(i, which=2)``."""
        k = len(self)
        Lv = (C.c_double * k)()
        gs = (C.c_double * (2 * k))()
        self._chk(self._lib.tsp_batch_loglik_grad(self._h, Lv, gs, _stream_handle(stream)))
        return np.array(Lv[:]), np.array(gs[:]).reshape(k, 2)

    def stats(self, i: int, stream=None) -> dict:
        s = L.Stats()
        self._chk(self._lib.tsp_batch_stats(self._h, int(i), C.byref(s), _stream_handle(stream)))
        return {k: getattr(s, k) for k, _ in L.Stats._fields_}

    @property
    def schedule(self) -> dict:
        s = L.Schedule()
        self._chk(self._lib.tsp_batch_get_schedule(self._h, C.byref(s)))
        return _sched_dict(s)

    def set_schedule(self, ty_cap: int = 128, items_per_sm: int = 8, order: int = 0, stream=None):
        s = L.Schedule(int(ty_cap), int(items_per_sm), int(order), 0)
        self._chk(self._lib.tsp_batch_set_schedule(self._h, C.byref(s), _stream_handle(stream)))

    def autotune(self, stream=None) -> Tuple[dict, float]:
        s = L.Schedule()
        ms = C.c_float()
        self._chk(self._lib.tsp_batch_autotune(self._h, C.byref(s), C.byref(ms),
                                               _stream_handle(stream)))
        return _sched_dict(s), ms.value

    def set_profiling(self, on: bool = True):
        self._chk(self._lib.tsp_batch_set_profiling(self._h, int(bool(on))))

    def pass_times(self, max_count: int = 4096, stream=None):
        buf = (C.c_float * max_count)()
        cnt = C.c_int()
        self._chk(self._lib.tsp_batch_pass_times(self._h, buf, max_count, C.byref(cnt),
                                                 _stream_handle(stream)))
        return [buf[i] for i in range(cnt.value)]


if torch is not None:

    class LogLik(torch.autograd.Function):
        """L(rho, sigma) = sum_j log D_j - sum_i s_i rho_i of a Recon's events,
        with its gradient from the library's adjoint pass (denominators
        recomputed, windows fixed at the evaluated sigma).

        Usage: ``LogLik.apply(recon, rho, sigma)`` with rho a (ny, nz) CUDA
        tensor and sigma a length-2 tensor (sigma_z, sigma_dl)."""

        @staticmethod
        def forward(ctx, recon: Recon, rho, sigma):
            s = sigma.detach().double().cpu().numpy()
            if (s[0], s[1]) != (recon.params.sigma_z, recon.params.sigma_dl):
                recon.set_sigma(float(s[0]), float(s[1]))
            recon.set_image(rho.detach().to(torch.float32).contiguous())
            want_rho, want_sigma = ctx.needs_input_grad[1], ctx.needs_input_grad[2]
            if want_rho or want_sigma:
                val, g, gs = recon.loglik_grad(want_rho=want_rho, want_sigma=want_sigma)
            else:
                val, g, gs = recon.loglik(), None, None
            ctx.g_rho = g
            ctx.g_sigma = None if gs is None else torch.tensor(gs, dtype=sigma.dtype,
                                                                device=sigma.device)
            return torch.tensor(val, dtype=torch.float64, device=rho.device)

        @staticmethod
        def backward(ctx, grad_out):
            go = float(grad_out)
            g_rho = None if ctx.g_rho is None else ctx.g_rho * go
            g_sig = None if ctx.g_sigma is None else ctx.g_sigma * go
            return None, g_rho, g_sig
