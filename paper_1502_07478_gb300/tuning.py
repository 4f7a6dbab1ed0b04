"""Host-side helpers around a reconstruction: a persistent cache of tuned tile
schedules, and per-iteration metrics.

Schedules: ``Recon.autotune`` (tsp_autotune) times MLEM passes to pick the
tile schedule (tile height cap, items per SM, item order).  The best choice
depends on the grid, the pixel pitch, the resolution, the GPU and the order of
magnitude of the event count, not on the events' values, so
``tuned_schedule`` keeps it in a JSON file keyed by those and applies a cached
entry instead of timing again.

Metrics: ``iterate_logged`` applies single MLEM updates (Eq. iter) and records
after each one the quantities that check a reconstruction as it runs: events
used, sum_l s_l rho_l (equal to the events used: count conservation), the
log-likelihood (optional: it costs one more pass), empty windows, and the mean
number of window pixels per event.
"""
from __future__ import annotations

import json
import math
import os
from typing import IO, List, Optional


def schedule_key(recon, device_name: Optional[str] = None) -> str:
    """The cache key of ``recon``'s schedule: geometry, grid, pitch,
    resolution, window cut, gamma, kappa_z, GPU name and the decade of its
    event count."""
    p = recon.params
    if device_name is None:
        import torch
        device_name = torch.cuda.get_device_name(recon.device)
    n = max(1, int(recon.stats()["n_events"]))
    fields = (f"R={p.R:g}", f"L={p.L:g}", f"grid={p.ny}x{p.nz}", f"dy={p.dy:g}", f"dz={p.dz:g}",
              f"sz={p.sigma_z:g}", f"sdl={p.sigma_dl:g}", f"cut={p.cut:g}", f"gamma={p.gamma:g}",
              f"kappa_z={p.kappa_z:g}", f"events=1e{round(math.log10(n))}", f"gpu={device_name}")
    return "|".join(fields)


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def tuned_schedule(recon, path: str, device_name: Optional[str] = None) -> dict:
    """Apply the cached schedule for ``recon`` (events uploaded) from the JSON
    file ``path``, or autotune, apply and store it.  Returns {"schedule",
    "pass_ms", "cached"}.  The file is rewritten atomically (write, rename)."""
    key = schedule_key(recon, device_name)
    cache = _load(path)
    hit = cache.get(key)
    if isinstance(hit, dict) and isinstance(hit.get("schedule"), dict):
        recon.set_schedule(**hit["schedule"])
        return {"schedule": hit["schedule"], "pass_ms": hit.get("pass_ms"), "cached": True}
    sched, ms = recon.autotune()
    cache = _load(path)                      # merge with entries written meanwhile
    cache[key] = {"schedule": sched, "pass_ms": ms}
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
    return {"schedule": sched, "pass_ms": ms, "cached": False}


def iterate_logged(recon, n_iter: int, log: Optional[IO[str]] = None,
                   with_loglik: bool = True) -> List[dict]:
    """Apply ``n_iter`` single updates of Eq. iter to ``recon``; after each,
    record {"iteration", "n_used", "sum_s_rho", "conservation_rel", "loglik",
    "n_empty", "mean_window_pixels"} and write it to ``log`` as one JSON line.
    Returns the records."""
    out = []
    for _ in range(int(n_iter)):
        recon.iterate(1)
        st = recon.stats()
        used = int(st["n_used"])
        rec = {"iteration": int(st["iterations"]), "n_used": used,
               "sum_s_rho": float(st["sum_s_rho"]),
               "conservation_rel": float(st["sum_s_rho"]) / max(1, used) - 1.0,
               "loglik": float(recon.loglik()) if with_loglik else None,
               "n_empty": int(st["n_empty"]),
               "mean_window_pixels": float(st["n_window"]) / max(1, int(st["n_events"]))}
        out.append(rec)
        if log is not None:
            log.write(json.dumps(rec) + "\n")
            log.flush()
    return out
