"""Named synthetic workloads.

Geometry and resolution follow the paper's detector (Sec. 2, Sec. 3: sigma_z about
10 mm, sigma_dl about 40 mm, 3-sigma windows); the paper's own simulated event
sets are not published, so every workload is generated here from a seed.

Image grid: ny x nz pixels over y in [-R, R], z in [-L/2, L/2]; row-major with z
contiguous; pixel (iy, iz) has centre y = -R + (iy + 1/2) dy, z = -L/2 + (iz + 1/2) dz.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Callable, Dict, Optional

import numpy as np

from .events import Geometry, simulate_events
from .phantom import Ellipse, Phantom, paper_phantom, random_phantom


@dataclass(frozen=True)
class Workload:
    name: str
    R: float
    L: float
    ny: int
    nz: int
    sigma_z: float
    sigma_dl: float
    cut: float
    n_events: int
    n_iter: int
    seed: int
    phantom_fn: Callable[[], Phantom] = field(compare=False, repr=False)

    @property
    def dy(self) -> float:
        return 2.0 * self.R / self.ny

    @property
    def dz(self) -> float:
        return self.L / self.nz

    @property
    def geometry(self) -> Geometry:
        return Geometry(R=self.R, L=self.L, sigma_z=self.sigma_z, sigma_dl=self.sigma_dl)

    def phantom(self) -> Phantom:
        return self.phantom_fn()

    def events(self, dtype=np.float32):
        """(zu, zd, dl) arrays of length n_events, drawn from the seed."""
        return simulate_events(self.phantom(), self.geometry, self.n_events, self.seed,
                               dtype=dtype)

    def chunk_sizes(self, chunk: int):
        return [min(chunk, self.n_events - f) for f in range(0, self.n_events, chunk)]

    def event_chunk(self, k: int, chunk: int, dtype=np.float32):
        """Chunk k (of chunk_sizes(chunk)) of the streamed form of the event set:
        chunk k is drawn from the seed sequence (seed, k), so chunks can be made
        independently and in parallel.  (A different event set from events(),
        with the same distribution.)"""
        n = self.chunk_sizes(chunk)[k]
        return simulate_events(self.phantom(), self.geometry, n, (self.seed, k), dtype=dtype)

    def event_chunks(self, chunk: int = 10_000_000, dtype=np.float32):
        """Iterate over the chunks of the streamed event set."""
        for k in range(len(self.chunk_sizes(chunk))):
            yield self.event_chunk(k, chunk, dtype)


def _small_phantom():
    rng = np.random.Generator(np.random.PCG64(1001))
    return random_phantom(rng, 3, 350.0, 500.0)


def _stress_phantom():
    rng = np.random.Generator(np.random.PCG64(5005))
    ells = []
    # four hot spots (radius 2-5 mm, density 8) listed first so they win overlaps
    for _ in range(4):
        r = rng.uniform(2.0, 5.0)
        ells.append(Ellipse(z=rng.uniform(-150, 150), y=rng.uniform(-120, 120),
                            a=r, b=r, phi_deg=0.0, rho=8.0))
    for _ in range(3):
        ells.append(Ellipse(z=rng.uniform(-120, 120), y=rng.uniform(-100, 100),
                            a=rng.uniform(20, 60), b=rng.uniform(20, 60),
                            phi_deg=rng.uniform(0, 180), rho=rng.uniform(0.3, 2.0)))
    ells.append(Ellipse(z=0.0, y=0.0, a=200.0, b=250.0 * 0.8, phi_deg=0.0, rho=1.0))
    return Phantom(tuple(ells))


WORKLOADS: Dict[str, Workload] = {
    # 5 mm pixels, 2e4 events, 5 iterations: small enough for the full FP64 oracle
    "small_5mm": Workload("small_5mm", 350.0, 500.0, 140, 100, 10.0, 42.0, 3.0,
                          20_000, 5, 1, _small_phantom),
    # 1 mm pixels, 1e7 events, 20 iterations: the paper-scale headline workload
    "paper_1mm": Workload("paper_1mm", 350.0, 500.0, 700, 500, 10.0, 42.0, 3.0,
                          10_000_000, 20, 2, lambda: paper_phantom(cold_row=1)),
    # 2 mm pixels, 1e6 events: the adjoint (gradient) workload
    "adjoint_2mm": Workload("adjoint_2mm", 350.0, 500.0, 350, 250, 10.0, 42.0, 3.0,
                            1_000_000, 10, 4, lambda: paper_phantom(cold_row=1)),
    # 0.5 mm pixels, 1e8 events: the stress workload
    "stress_05mm": Workload("stress_05mm", 350.0, 500.0, 1400, 1000, 10.0, 42.0, 3.0,
                            100_000_000, 10, 5, _stress_phantom),
    # the paper's own figure geometry (R=130, L=300, 4 mm pixels), 1 iteration
    "paper_geom_4mm": Workload("paper_geom_4mm", 130.0, 300.0, 65, 75, 10.0, 40.0, 3.0,
                               10_000_000, 1, 6, lambda: paper_phantom()),
}


def make_workload(name: str, **overrides) -> Workload:
    """A named workload, optionally with fields replaced (e.g. a smaller n_events)."""
    w = WORKLOADS[name]
    return replace(w, **overrides) if overrides else w


def batched_instances(k: int = 64, seed: int = 3):
    """Independent reconstructions for the batched workload: each with its own
    2-6 ellipse phantom, pixel size drawn from {1, 2, 4} mm, event count
    log-uniform in [1e4, 2e6], sigma_z in [8, 12] mm, sigma_dl in [30, 50] mm,
    10 iterations."""
    ss = np.random.SeedSequence(seed)
    out = []
    for i, child in enumerate(ss.spawn(k)):
        rng = np.random.Generator(np.random.PCG64(child))
        n_ell = int(rng.integers(2, 7))
        pix = float(rng.choice([1.0, 2.0, 4.0]))
        n_ev = int(round(10 ** rng.uniform(4.0, np.log10(2e6))))
        sz = float(rng.uniform(8.0, 12.0))
        sdl = float(rng.uniform(30.0, 50.0))
        ph_seed = int(rng.integers(0, 2**31 - 1))
        ev_seed = int(rng.integers(0, 2**31 - 1))

        def _ph(ph_seed=ph_seed, n_ell=n_ell):
            return random_phantom(np.random.Generator(np.random.PCG64(ph_seed)), n_ell,
                                  350.0, 500.0)

        w = Workload(f"batch_{i:02d}", 350.0, 500.0, int(round(700 / pix)),
                     int(round(500 / pix)), sz, sdl, 3.0, n_ev, 10, ev_seed, _ph)
        out.append(w)
    return out
