"""Seeded list-mode event simulation for the two-strip detector.

Detector (Sec. 2 and Fig. 1 of the paper): two thin scintillator strips of length
L lie parallel to the z axis at y = +R (upper) and y = -R (lower).  An
annihilation at (y, z) emits two back-to-back photons along a line at angle
theta to the y axis.  Each detected event is the triple (z_u, z_d, delta_l): the
hit positions along the upper and lower strips and the difference of the path
lengths from the emission point to the upper and to the lower strip.

This module only produces data.  It traces the emission line to the two strip
planes with plain ray geometry and measures Euclidean path lengths; it contains
none of the reconstruction arithmetic.

Recipe (all draws from numpy ``Generator(PCG64(seed))``, in fixed-size batches
so that a seed always gives the same events):
  1. emission point (y, z) by rejection sampling from the phantom density;
  2. angle theta uniform on (-pi/2, pi/2) (drawn on the sub-range that can
     reach both strips, which gives the same accepted distribution);
  3. keep the event iff both true hit positions lie on the strips, |z| <= L/2;
  4. add independent Gaussian noise N(0, sigma_z) to z_u and z_d and
     N(0, sigma_dl) to delta_l (a diagonal correlation matrix);
  5. no cut on the measured values.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

_BATCH = 1 << 20


@dataclass(frozen=True)
class Geometry:
    R: float          # half of the strip separation (mm); strips at y = +-R
    L: float          # strip length (mm)
    sigma_z: float    # resolution of z_u, z_d (mm)
    sigma_dl: float   # resolution of delta_l (mm)


def _trace(y, z, theta, R):
    """Hit positions and path lengths of the emission line through (y, z).

    The line is parametrised as (y + s cos(theta), z + s sin(theta)).  It meets
    the plane y = +R at s_u = (R - y)/cos(theta) and y = -R at
    s_d = -(R + y)/cos(theta)."""
    ct = np.cos(theta)
    st = np.sin(theta)
    s_up = (R - y) / ct
    s_dn = -(R + y) / ct
    zu = z + s_up * st
    zd = z + s_dn * st
    # Euclidean distances from the emission point to each hit
    d_up = np.hypot(R - y, zu - z)
    d_dn = np.hypot(-R - y, zd - z)
    return zu, zd, d_up - d_dn


def simulate_events(phantom, geom: Geometry, n: int, seed, *, dtype=np.float64,
                    return_truth: bool = False):
    """Return ``n`` accepted, smeared events as arrays (zu, zd, dl) of ``dtype``.

    With ``return_truth`` also return the noise-free (zu, zd, dl) and the
    emission (y, z, theta) as float64 arrays."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ymin, ymax, zmin, zmax = phantom.bounding_box()
    rho_max = phantom.max_density()
    out = [np.empty(n, dtype=dtype) for _ in range(3)]
    truth = [np.empty(n, dtype=np.float64) for _ in range(6)] if return_truth else None
    filled = 0
    half_l = 0.5 * geom.L
    # Both hits lie on the strips only if |z_u - z_d| = 2R|tan(theta)| <= L, so
    # drawing theta uniformly on [-theta_c, theta_c] instead of (-pi/2, pi/2)
    # leaves the distribution of accepted events unchanged and wastes fewer draws.
    theta_c = np.arctan(half_l / geom.R)
    while filled < n:
        y = rng.uniform(ymin, ymax, _BATCH)
        z = rng.uniform(zmin, zmax, _BATCH)
        u = rng.uniform(0.0, rho_max, _BATCH)
        sel = u < phantom.density(y, z)
        y = y[sel]
        z = z[sel]
        theta = rng.uniform(-theta_c, theta_c, y.size)
        zu, zd, dl = _trace(y, z, theta, geom.R)
        keep = (np.abs(zu) <= half_l) & (np.abs(zd) <= half_l)
        idx = np.nonzero(keep)[0]
        take = min(idx.size, n - filled)
        idx = idx[:take]
        noise = rng.standard_normal((3, take))
        sl = slice(filled, filled + take)
        out[0][sl] = zu[idx] + geom.sigma_z * noise[0]
        out[1][sl] = zd[idx] + geom.sigma_z * noise[1]
        out[2][sl] = dl[idx] + geom.sigma_dl * noise[2]
        if return_truth:
            for k, arr in enumerate((zu, zd, dl, y, z, theta)):
                truth[k][sl] = arr[idx]
        filled += take
    if return_truth:
        return tuple(out), tuple(truth)
    return tuple(out)
