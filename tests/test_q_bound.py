"""The lower bound of Q = aC^-1a + 2 oC^-1b over an event's window that the
upload step uses to flag events (reading R5's clip cannot apply to them),
checked against the minimum of Q over every window pixel, evaluated from the
vectors o, a, b of Sec. 3 (derived a3, reading R3) for seeded events of the
5 mm and 1 mm workloads: the bound never exceeds the minimum, and it clears
its 1e-3 margin for every event, so these workloads' events are all flagged."""
import numpy as np

from synth import make_workload


def _events(w, n):
    zu, zd, dl = (e.astype(np.float64) for e in w.events())
    zu, zd, dl = zu[:n], zd[:n], dl[:n]
    R = w.R
    t = (zu - zd) / (2.0 * R)                          # Eq. 2, first forms
    ey = -0.5 * dl / np.sqrt(1.0 + t * t)
    ez = 0.5 * (zu + zd + 2.0 * ey * t)
    return ey, ez, t


def _q_min_over_window(w, ey, ez, t):
    iz, il, R = 1.0 / w.sigma_z ** 2, 1.0 / w.sigma_dl ** 2, w.R
    yc = -R + (np.arange(w.ny) + 0.5) * w.dy
    zc = -w.L / 2 + (np.arange(w.nz) + 0.5) * w.dz
    # the window lies within |y - ey| <= cut sdl/2 and |z - ez| <= cut sz/sqrt2 + |t| cut sdl/2
    hy = w.cut * w.sigma_dl / 2.0 + w.dy
    hz = w.cut * w.sigma_z / np.sqrt(2.0) + abs(t) * hy + w.dz
    yc = yc[np.abs(yc - ey) <= hy]
    zc = zc[np.abs(zc - ez) <= hz]
    Y, Z = np.meshgrid(yc, zc, indexing="ij")
    sec = np.sqrt(1.0 + t * t)
    dY, dZ = Y - ey, Z - ez
    y = dY + ey
    b = (dZ - dY * t, dZ - dY * t, -2.0 * dY * sec)
    inside = iz * (b[0] ** 2 + b[1] ** 2) + il * b[2] ** 2 <= w.cut ** 2
    a = (-(y - R) * sec ** 2, -(y + R) * sec ** 2, -2.0 * y * sec * t)
    o = (-(y - R) * t * sec ** 2, -(y + R) * t * sec ** 2, -y * sec * (1.0 + 2.0 * t * t))
    aCa = iz * (a[0] ** 2 + a[1] ** 2) + il * a[2] ** 2
    oCb = iz * (o[0] * b[0] + o[1] * b[1]) + il * o[2] * b[2]
    Q = aCa + 2.0 * oCb
    return float(Q[inside].min()) if inside.any() else np.inf


def _bound(w, ey, t):
    """The upload step's bound (kEvQPos), restated in double precision."""
    iz, il, R = 1.0 / w.sigma_z ** 2, 1.0 / w.sigma_dl ** 2, w.R
    c2i = 1.0 + t * t
    hy = w.cut * w.sigma_dl / 2.0 / np.sqrt(c2i) * 1.001 + w.dy
    umax = w.cut / np.sqrt(2.0 * iz) + w.dz
    ymax = abs(ey) + hy
    lead = 2.0 * iz * R * R * c2i * c2i
    q = lead - 4.0 * il * ymax * (2.0 * t * t + 1.0) * hy * c2i - 4.0 * iz * ymax * abs(t) * c2i * umax
    return q, lead


def test_q_bound_below_window_minimum():
    for name, n in (("small_5mm", 400), ("paper_1mm", 60)):
        w = make_workload(name, n_events=n)
        ey, ez, t = _events(w, n)
        for j in range(n):
            qmin = _q_min_over_window(w, ey[j], ez[j], t[j])
            q, lead = _bound(w, ey[j], t[j])
            assert q <= qmin, (name, j, q, qmin)
            assert q > 1e-3 * lead, (name, j, q, lead)
