"""The paper's printed tables, kept as fixtures under tests/golden/."""
import os

import numpy as np

from synth import paper_phantom

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(x) for x in line.split()])
    return np.array(rows)


def test_phantom_table_matches_generator():
    """App. A table: the generator's paper phantom has the same six rows, in order."""
    tab = _rows("paper_phantom.txt")
    ph = paper_phantom()
    got = np.array([[e.z, e.y, e.a, e.b, e.phi_deg, e.rho] for e in ph.ellipses])
    np.testing.assert_array_equal(got, tab)


def test_phantom_priority_topmost_row_wins():
    """Overlaps take the density of the topmost row: the centre is row 1 (0.3),
    not the body (0.1)."""
    ph = paper_phantom()
    assert ph.density(np.array([0.0]), np.array([0.0]))[0] == 0.3
    assert ph.density(np.array([100.0]), np.array([0.0]))[0] == 0.1
    assert ph.density(np.array([55.0]), np.array([35.0]))[0] == 0.7


def test_timing_table_is_linear_with_25x_speedup():
    """The paper's timing table: time grows linearly with events; CPU/warp ~ 25."""
    t = _rows("paper_timings.txt")
    ev, cpu, warp = t[:, 0], t[:, 1], t[:, 2]
    assert np.all(np.abs(cpu / warp - 25.0) < 0.5)
    slope = np.polyfit(ev, warp, 1)[0]
    assert abs(slope - 46.6) < 0.2  # ms per million events
