"""The streamed form of a workload's events: chunk k is drawn from the seed
sequence (seed, k), so chunks made one by one, in any order or in parallel,
are the same arrays."""
import numpy as np

from synth import make_workload


def test_chunks_are_reproducible_and_sized():
    w = make_workload("stress_05mm", n_events=30_000)
    a = [c[0] for c in w.event_chunks(12_000)]
    b = [w.event_chunk(k, 12_000)[0] for k in (2, 0, 1)]
    assert [len(x) for x in a] == [12_000, 12_000, 6_000]
    for x, y in zip(a, [b[1], b[2], b[0]]):
        np.testing.assert_array_equal(x, y)
    assert not np.array_equal(a[0][:100], a[1][:100])


def test_chunks_follow_the_detector_acceptance():
    """Every event of a chunk had both true hits on the strips: the measured
    |z_u|, |z_d| exceed L/2 only by the smearing (a few sigma_z)."""
    w = make_workload("stress_05mm", n_events=20_000)
    zu, zd, dl = w.event_chunk(0, 20_000)
    assert zu.dtype == np.float32 and len(zu) == 20_000
    lim = 0.5 * w.L + 6 * w.sigma_z
    assert np.all(np.abs(zu) < lim) and np.all(np.abs(zd) < lim)
