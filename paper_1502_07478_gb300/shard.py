"""Event-sharded MLEM iterations of one reconstruction over several ranks.

Eq. iter is a sum over events, and given the image rho^t the events are
independent.  So a reconstruction whose events are split over ranks (one GPU
each, every rank holding the same image) advances by one iteration as:
  1. each rank back-projects its own events at rho^t
     (``Recon.backproject``, tsp_backproject),
  2. the ranks' back-projections are summed (an all-reduce, e.g. NCCL),
  3. every rank applies the summed back-projection (``Recon.apply_update``,
     tsp_apply_update), so the images stay identical.
This module only orders those calls; the kernels run in libtsp and the sum in
the collective library.
"""
from __future__ import annotations

from typing import Callable, Optional


def sharded_iterate(recon, n_iter: int, all_reduce: Callable, buf=None) -> Optional[object]:
    """Apply n_iter iterations of Eq. iter to ``recon`` whose events are this
    rank's share of the list.  ``all_reduce(buf)`` must sum ``buf`` in place
    over all ranks (``torch.distributed.all_reduce`` does).  ``buf`` is the
    back-projection buffer (ny*nz float32, on the device for NCCL), allocated
    by ``recon.backproject`` when None.  Returns the buffer."""
    for _ in range(int(n_iter)):
        buf = recon.backproject(out=buf)
        all_reduce(buf)
        recon.apply_update(buf)
    return buf
