"""Brute-force NumPy statement of the list-mode MLEM update, for tiny inputs.

TEST INFRASTRUCTURE ONLY (see the package docstring).  It evaluates the paper's
kernel (Eq. kernel, with the vectors o, a, b and C^-1 of Sec. 3) for EVERY
(event, pixel) pair of the grid, with no bounding box, applies the window test
b C^-1 b <= cut^2 (Sec. 3), and forms Eq. iter with dense arrays.  It shares no
code with oracle.c; agreement of the two checks the C oracle's bounding-box
loop, caching and per-thread accumulation.
"""
from __future__ import annotations

import numpy as np


def _cinv(sz, sdl, gamma):
    iz, il = 1.0 / sz**2, 1.0 / sdl**2
    return np.array([[iz, 0.0, gamma], [0.0, iz, -gamma], [gamma, -gamma, il]])


def kernel_matrix(setup, events, window_sigma=None):
    """Dense P[j, i] (events x pixels), zero outside each event's window."""
    zu, zd, dl = (np.asarray(e, dtype=np.float64) for e in events)
    R = setup.R
    # Eq. 2, first forms
    t = (zu - zd) / (2.0 * R)
    ey = -0.5 * dl / np.sqrt(1.0 + t * t)
    ez = 0.5 * (zu + zd + 2.0 * ey * t)
    yc, zc = setup.pixel_centres()
    Y, Z = np.meshgrid(yc, zc, indexing="ij")
    Y = Y.ravel()[None, :]
    Z = Z.ravel()[None, :]
    ey, ez, t = ey[:, None], ez[:, None], t[:, None]
    sec = np.sqrt(1.0 + t * t)
    dY = Y - ey
    dZ = Z - ez
    a3f = -1.0 if setup.a3_printed else -2.0
    o = np.stack([-(dY + ey - R) * t * sec**2,
                  -(dY + ey + R) * t * sec**2,
                  -(dY + ey) * sec * (1.0 + 2.0 * t * t)], axis=-1)
    a = np.stack([-(dY + ey - R) * sec**2,
                  -(dY + ey + R) * sec**2,
                  a3f * (dY + ey) * sec * t], axis=-1)
    b = np.stack([dZ - dY * t, dZ - dY * t, -2.0 * dY * sec], axis=-1)
    Ck = _cinv(setup.sigma_z, setup.sigma_dl, setup.gamma)
    ws = window_sigma or (setup.wsigma_z or setup.sigma_z, setup.wsigma_dl or setup.sigma_dl)
    Cw = _cinv(ws[0], ws[1], setup.gamma)
    q = lambda u, M, v: np.einsum("...r,rc,...c->...", u, M, v)
    inside = q(b, Cw, b) <= setup.cut**2
    aCa, oCb, bCb, aCb = q(a, Ck, a), q(o, Ck, b), q(b, Ck, b), q(a, Ck, b)
    Q = aCa + 2.0 * oCb
    good = Q > 0
    Qs = np.where(good, Q, 1.0)
    pref = np.sqrt(np.linalg.det(Ck)) / (2.0 * np.pi**2 * np.sqrt(Qs))
    P = setup.pscale * pref * np.exp(-0.5 * (bCb - aCb**2 / Qs))
    return np.where(inside & good, P, 0.0)


def mlem(setup, events, n_iter, s, rho0=None):
    """Eq. iter with dense matrices: rho <- rho * P^T (1/D), D = P (s rho)."""
    P = kernel_matrix(setup, events)
    s = np.asarray(s, dtype=np.float64).ravel()
    rho = np.ones(P.shape[1]) if rho0 is None else np.asarray(rho0, np.float64).ravel().copy()
    for _ in range(n_iter):
        D = P @ (s * rho)
        used = D > 0
        invD = np.where(used, 1.0 / np.where(used, D, 1.0), 0.0)
        rho = rho * (P.T @ invD)
    return rho.reshape(setup.ny, setup.nz)
