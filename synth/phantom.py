"""Ellipse phantoms.

A phantom is an ordered list of ellipses, each with a centre, two half-axes, a
counter-clockwise rotation angle and a relative tracer density.  Where ellipses
overlap, the density of the ellipse listed first wins (App. A, "Phantom").

Coordinates: the paper's table uses (x, y); this project maps x to z (along the
strips) and y to y (across the gap between the strips).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Sequence

import numpy as np


@dataclass(frozen=True)
class Ellipse:
    z: float      # centre along the strips (mm); the table's x
    y: float      # centre across the gap (mm)
    a: float      # half-axis along z before rotation (mm)
    b: float      # half-axis along y before rotation (mm)
    phi_deg: float  # counter-clockwise rotation (degrees)
    rho: float    # relative density


@dataclass(frozen=True)
class Phantom:
    ellipses: tuple

    def density(self, y: np.ndarray, z: np.ndarray) -> np.ndarray:
        """Density at points (y, z); the first-listed containing ellipse wins."""
        y = np.asarray(y, dtype=np.float64)
        z = np.asarray(z, dtype=np.float64)
        out = np.zeros(np.broadcast(y, z).shape, dtype=np.float64)
        assigned = np.zeros(out.shape, dtype=bool)
        for e in self.ellipses:
            inside = self._inside(e, y, z) & ~assigned
            out[inside] = e.rho
            assigned |= inside
        return out

    @staticmethod
    def _inside(e: Ellipse, y, z):
        phi = np.deg2rad(e.phi_deg)
        dz = z - e.z
        dy = y - e.y
        # rotate the offset by -phi into the ellipse's own axes
        zr = dz * np.cos(phi) + dy * np.sin(phi)
        yr = -dz * np.sin(phi) + dy * np.cos(phi)
        return (zr / e.a) ** 2 + (yr / e.b) ** 2 <= 1.0

    def bounding_box(self):
        """(ymin, ymax, zmin, zmax) enclosing every ellipse with density > 0."""
        ys, zs = [], []
        for e in self.ellipses:
            if e.rho <= 0:
                continue
            phi = np.deg2rad(e.phi_deg)
            hz = np.hypot(e.a * np.cos(phi), e.b * np.sin(phi))
            hy = np.hypot(e.a * np.sin(phi), e.b * np.cos(phi))
            ys += [e.y - hy, e.y + hy]
            zs += [e.z - hz, e.z + hz]
        return min(ys), max(ys), min(zs), max(zs)

    def max_density(self) -> float:
        return max(e.rho for e in self.ellipses)

    def rasterize(self, ny: int, nz: int, R: float, L: float) -> np.ndarray:
        """Density at pixel centres of an ny x nz grid over [-R,R] x [-L/2,L/2]."""
        dy = 2.0 * R / ny
        dz = L / nz
        yc = -R + (np.arange(ny) + 0.5) * dy
        zc = -0.5 * L + (np.arange(nz) + 0.5) * dz
        Y, Z = np.meshgrid(yc, zc, indexing="ij")
        return self.density(Y, Z)


def paper_phantom(cold_row: int | None = None) -> Phantom:
    """The six-ellipse phantom of App. A (table "Phantom description").

    The numbers are typed here; ``tests/golden/paper_phantom.txt`` holds the same
    table with its citation and a test checks that the two agree.  ``cold_row``
    (0-based) sets that row's density to 0, giving a cold insert.
    """
    rows = [
        # x(->z)  y     a     b    phi   rho
        (0.0, 0.0, 30.0, 60.0, 0.0, 0.3),
        (50.0, -62.0, 10.0, 33.0, -40.0, 0.3),
        (-50.0, -63.0, 20.0, 33.0, 45.0, 0.5),
        (60.0, 65.0, 13.0, 14.0, 0.0, 0.5),
        (35.0, 55.0, 12.0, 12.0, 0.0, 0.7),
        (0.0, 0.0, 120.0, 110.0, 0.0, 0.1),
    ]
    ells = []
    for i, (x, y, a, b, phi, rho) in enumerate(rows):
        if cold_row is not None and i == cold_row:
            rho = 0.0
        ells.append(Ellipse(z=x, y=y, a=a, b=b, phi_deg=phi, rho=rho))
    return Phantom(tuple(ells))


def random_phantom(rng: np.random.Generator, n_ellipses: int, R: float, L: float,
                   rho_range=(0.5, 2.0), axis_range=(20.0, 100.0)) -> Phantom:
    """Seeded random ellipses: centres uniform in |y|<=R/2, |z|<=L/4, half-axes
    uniform in ``axis_range``, angle uniform in [0, 180), density uniform in
    ``rho_range``.  Half-axes shrink (x0.9 steps) until the ellipse lies inside
    |y| < 0.9 R and |z| < 0.45 L."""
    ells: List[Ellipse] = []
    for _ in range(n_ellipses):
        cy = rng.uniform(-0.5 * R, 0.5 * R)
        cz = rng.uniform(-0.25 * L, 0.25 * L)
        a = rng.uniform(*axis_range)
        b = rng.uniform(*axis_range)
        phi = rng.uniform(0.0, 180.0)
        rho = rng.uniform(*rho_range)
        for _shrink in range(200):
            e = Ellipse(z=cz, y=cy, a=a, b=b, phi_deg=phi, rho=rho)
            ymin, ymax, zmin, zmax = Phantom((e,)).bounding_box()
            if ymin > -0.9 * R and ymax < 0.9 * R and zmin > -0.45 * L and zmax < 0.45 * L:
                break
            a *= 0.9
            b *= 0.9
        ells.append(e)
    return Phantom(tuple(ells))


def phantom_from_rows(rows: Sequence[Sequence[float]]) -> Phantom:
    return Phantom(tuple(Ellipse(z=r[0], y=r[1], a=r[2], b=r[3], phi_deg=r[4], rho=r[5])
                         for r in rows))
