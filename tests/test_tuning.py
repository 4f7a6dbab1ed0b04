"""Host logic of paper_1502_07478_gb300.tuning on CPU: the schedule cache's key,
hit/miss behaviour and file handling, and the per-iteration metrics records,
against a stand-in reconstruction (no GPU)."""
import io
import json

import pytest

from paper_1502_07478_gb300._lib import Params
from paper_1502_07478_gb300.tuning import iterate_logged, schedule_key, tuned_schedule


class _Stub:
    """Records calls; autotune returns a fixed schedule; iterate keeps counts."""

    def __init__(self, ny=140, nz=100, n_events=20000, sigma_z=10.0):
        self.params = Params(350.0, 500.0, ny, nz, 0.0, 0.0, sigma_z, 42.0, 3.0, 0, 0, 0.0, 0.0)
        self.device = 0
        self.n_events = n_events
        self.calls = []
        self.it = 0

    def stats(self):
        return {"n_events": self.n_events, "n_used": self.n_events - 5, "n_empty": 5,
                "n_window": 160 * self.n_events, "iterations": self.it,
                "sum_s_rho": float(self.n_events - 5) * (1 + 1e-9)}

    def autotune(self):
        self.calls.append("autotune")
        return {"ty_cap": 64, "items_per_sm": 4, "order": 1}, 1.25

    def set_schedule(self, **kw):
        self.calls.append(("set_schedule", kw))

    def iterate(self, n):
        self.it += n

    def loglik(self):
        return -1000.0 - self.it


def test_cache_miss_then_hit(tmp_path):
    path = str(tmp_path / "sched.json")
    a = _Stub()
    r = tuned_schedule(a, path, device_name="GB300")
    assert r == {"schedule": {"ty_cap": 64, "items_per_sm": 4, "order": 1}, "pass_ms": 1.25,
                 "cached": False}
    assert a.calls == ["autotune"]
    b = _Stub()
    r = tuned_schedule(b, path, device_name="GB300")
    assert r["cached"] and r["schedule"]["ty_cap"] == 64
    assert b.calls == [("set_schedule", {"ty_cap": 64, "items_per_sm": 4, "order": 1})]
    assert len(json.load(open(path))) == 1


def test_key_separates_what_the_schedule_depends_on(tmp_path):
    base = schedule_key(_Stub(), "GB300")
    assert schedule_key(_Stub(), "GB300") == base
    assert schedule_key(_Stub(ny=700, nz=500), "GB300") != base            # grid
    assert schedule_key(_Stub(sigma_z=12.0), "GB300") != base             # resolution
    assert schedule_key(_Stub(), "B200") != base                          # GPU
    assert schedule_key(_Stub(n_events=2_000_000), "GB300") != base       # decade of events
    assert schedule_key(_Stub(n_events=25_000), "GB300") == base          # same decade
    path = str(tmp_path / "s.json")
    tuned_schedule(_Stub(), path, "GB300")
    tuned_schedule(_Stub(ny=700, nz=500), path, "GB300")
    assert len(json.load(open(path))) == 2


def test_unreadable_cache_is_rebuilt(tmp_path):
    path = tmp_path / "s.json"
    path.write_text("{ not json")
    a = _Stub()
    r = tuned_schedule(a, str(path), "GB300")
    assert not r["cached"] and a.calls == ["autotune"]
    assert len(json.loads(path.read_text())) == 1


def test_iterate_logged_records():
    a = _Stub()
    buf = io.StringIO()
    recs = iterate_logged(a, 3, buf)
    assert [r["iteration"] for r in recs] == [1, 2, 3]
    lines = [json.loads(x) for x in buf.getvalue().splitlines()]
    assert lines == recs
    r = recs[-1]
    assert r["conservation_rel"] == pytest.approx(1e-9, rel=1e-6)
    assert r["loglik"] == -1003.0
    assert r["mean_window_pixels"] == 160.0 and r["n_empty"] == 5
    assert iterate_logged(_Stub(), 1, with_loglik=False)[0]["loglik"] is None
