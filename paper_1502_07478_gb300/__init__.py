"""GB300 (sm_103a) list-mode MLEM reconstruction for the two-strip detector of
Bialas et al., arXiv:1502.07478.

The computation lives in libtsp (csrc/, C ABI in include/tsp.h); this package
holds its build script and a thin binding (``Recon``, ``Batch``, ``LogLik``).
"""
from .build import build  # noqa: F401

__all__ = ["build", "Recon", "Batch", "LogLik", "TspError"]


def __getattr__(name):
    if name in ("Recon", "Batch", "LogLik"):
        from . import recon
        return getattr(recon, name)
    if name == "TspError":
        from ._lib import TspError
        return TspError
    raise AttributeError(name)
