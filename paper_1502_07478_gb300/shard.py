"""Event-sharded MLEM iterations of one reconstruction over several ranks.

Eq. iter is a sum over events, and given the image rho^t the events are
independent.  So a reconstruction whose events are split over ranks (one GPU
each, every rank holding the same image) advances by one iteration as:
  1. each rank back-projects its own events at rho^t
     (``Recon.backproject``, tsp_backproject),
  2. the ranks' back-projections are summed (an all-reduce, e.g. NCCL),
  3. every rank applies the summed back-projection (``Recon.apply_update``,
     tsp_apply_update), so the images stay identical.
The log-likelihood and its gradients shard the same way (``sharded_loglik_grad``):
one all-reduce of g_rho and one of (L, g_sigma), plus the image terms that
every rank would otherwise count once each.
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


def sharded_loglik_grad(recon, all_reduce: Callable, world_size: int):
    """The log-likelihood and its gradients over the whole event list, from
    ``recon`` holding this rank's share (every rank the same image and
    resolution).  With L = sum_j log D_j - sum_i s_i rho_i,
    g_rho = s (sum_j P_j/D_j - 1) and g_sigma = sum_j (...)/D_j
    (``Recon.loglik_grad``), the event sums add over ranks and the image
    terms are counted once:
        L       = sum_r L_r       + (K - 1) sum_i s_i rho_i,
        g_rho   = sum_r g_rho,r   + (K - 1) s,
        g_sigma = sum_r g_sigma,r,
    for K ranks: one all-reduce of g_rho and one of (L, g_sigma).
    ``all_reduce(t)`` must sum a tensor in place over the ranks.  Returns
    (L, g_rho, g_sigma) on every rank."""
    import numpy as np
    import torch
    L, g, gs = recon.loglik_grad()
    extra = int(world_size) - 1
    s = recon.compute_sensitivity()
    S = float(recon.read_image(which=1).double().sum())
    all_reduce(g)
    if extra:
        g += extra * s.to(g.dtype)
    v = torch.tensor([L, gs[0], gs[1]], dtype=torch.float64, device=g.device)
    all_reduce(v)
    v = v.cpu().numpy()
    return float(v[0]) + extra * S, g, np.array(v[1:])
