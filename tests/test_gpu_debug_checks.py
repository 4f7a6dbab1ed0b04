"""The bounds-checking build (TSP_DEBUG_CHECKS) on the tile passes' paths.

Every shared-memory access of the pixel loops (pass-1 rho' loads, pass-2
fixed-point and float adds, the scalar pass's loads and adds) is tested
against the block's dynamic shared-memory window; an access outside it would
be skipped and recorded (tsp_stats().dbg_violation).  The build is made here
(``build(debug=True)``) and run in a child process that loads it through
TSP_LIBRARY: on each path the record must stay 0 and the results must still
meet the parity bar against the FP64 oracle.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = r'''
import json, sys
import numpy as np
sys.path.insert(0, ROOT)
import oracle
from oracle import Setup
from synth import make_workload
from paper_1502_07478_gb300 import Recon, Batch

def rel(a, b, frac=0.01):
    a = np.asarray(a, np.float64).reshape(b.shape); m = b > frac * b.max()
    return float(np.max(np.abs(a[m] - b[m]) / b[m]))

out = {}
for name, n, it in (("small_5mm", None, 3), ("paper_1mm", 20000, 2), ("stress_05mm", 20000, 1)):
    w = make_workload(name, **({"n_events": n} if n else {}))
    ev = w.events()
    r = Recon.from_workload(w)
    r.upload_events(*ev)
    r.iterate(it)
    img = r.read_image().cpu().numpy()
    st = r.stats()
    r.close()
    ref, _ = oracle.mlem(Setup.from_workload(w), ev, it)
    out[name] = {"dbg": st["dbg_violation"], "rel": rel(img, ref), "clipped": st["n_clipped"]}

w = make_workload("small_5mm")
ev = w.events()
r = Recon.from_workload(w)
r.upload_events(*ev)
r.iterate(2)
rho = r.read_image().cpu().numpy().astype(np.float64)
L, g, gs = r.loglik_grad()
st = r.stats()
r.close()
Lr, gr, gsr = oracle.loglik_grad(Setup.from_workload(w), ev, rho)
gr = np.asarray(gr).reshape(g.shape)
out["adjoint"] = {"dbg": st["dbg_violation"],
                  "rel": float(np.linalg.norm(g.cpu().numpy() - gr) / np.linalg.norm(gr)),
                  "clipped": st["n_clipped"]}

ws = [make_workload("small_5mm", n_events=8000), make_workload("small_5mm", n_events=3000, seed=7)]
b = Batch.from_workloads(ws)
evs = [x.events() for x in ws]
for i, e in enumerate(evs):
    b.upload_events(i, *e)
b.iterate(2)
worst, dbg = 0.0, 0
for i, (x, e) in enumerate(zip(ws, evs)):
    ref, _ = oracle.mlem(Setup.from_workload(x), e, 2)
    worst = max(worst, rel(b.read_image(i).cpu().numpy(), ref))
    dbg |= b.stats(i)["dbg_violation"]
b.close()
out["batch"] = {"dbg": dbg, "rel": worst, "clipped": 0}
print("RESULT " + json.dumps(out))
'''


@pytest.fixture(scope="module")
def debug_lib():
    from paper_1502_07478_gb300.build import build
    return build(debug=True)


def test_bounds_checked_build_parity(debug_lib):
    env = dict(os.environ, TSP_LIBRARY=debug_lib)
    code = _CHILD.replace("ROOT", repr(ROOT))
    p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=1800, cwd=ROOT)
    assert p.returncode == 0, p.stderr[-3000:]
    line = [x for x in p.stdout.splitlines() if x.startswith("RESULT ")][-1]
    res = json.loads(line[len("RESULT "):])
    for case, r in res.items():
        assert r["dbg"] == 0, f"{case}: site {r['dbg'] >> 32}, byte offset {(r['dbg'] & 0xffffffff) - 1}"
        assert r["clipped"] == 0, case
        assert r["rel"] <= 1e-4, (case, r["rel"])
