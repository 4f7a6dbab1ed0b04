#!/usr/bin/env python3
"""Benchmark: list-mode MLEM event-iterations/s on the paper-scale workload.

Workload (default): two strips at +-350 mm, 500 mm long, 1 mm pixels
(700 x 500), sigma_z = 10 mm, sigma_dl = 42 mm, 3-sigma windows, the paper's
six-ellipse phantom with a cold insert, 1e7 seeded events, 20 iterations.  One
step is one full reconstruction: reset the image and apply the 20 MLEM
iterations (tsp_iterate, replayed from a CUDA graph) with the events resident
in HBM.  value = events x iterations x steps / time of the timed steps.

Also reported: batched vs plain on the batched workload (64 reconstructions
with their own grids, resolutions and event counts, 10 iterations each; one
tsp_batch with the autotuned schedule against 64 plain contexts run one after
another, images compared), the adjoint pass on the 2 mm workload, the same
metric end to end through the C ABI with host buffers
(e2e: pinned-host event upload, per-event preparation and binning, the
iterations and the image readout, every step), the dominant kernel's achieved
pixel-evaluation rate against its roofline (max of the SFU and FMA-pipe time
per evaluation), the FP64 CPU oracle timed on the host's cores on a bounded
sample of the same workload, and a stress record: the 1e8-event 0.5 mm
workload streamed in pinned 1e7-event chunks (one timed step of 10
iterations, with its own roofline) and the adjoint pass of 16 reconstructions
batched against 16 plain passes.  The stress inputs are generated by a spawned
process pool while the main leg runs.

``--impl reference`` times the FP64 CPU oracle instead (the reference arm).
Multi-GPU (torchrun, one rank per GPU): one reconstruction whose events are
sharded over the ranks -- rank r holds its own seeded share of the event count
(weak scaling: the list grows with the ranks) -- and every iteration is a
back-projection on each rank, an NCCL all-reduce (sum) of the back-projection
and the same image update on every rank; value is the events of all ranks x
iterations / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLEM event-iterations/s (1e7 events, 1 mm grid), batched vs plain, rel err <=1e-4"
UNIT = "event-iterations/s"
# Roofline of the MLEM pass (one unit = one in-window pixel evaluation of the
# kernel P; the count W per launch is exact, from the event preparation).  The
# algorithmic work per unit: 2 SFU operations (one rsqrt, one ex2) and 17
# FMA-pipe operations (the kernel's quadratic forms, the exponent, P, the
# denominator sum and the scatter's product, row constants amortised).
# Per-SM rates per clock: 128 FP32 FMA lanes; the SFU rates measured by
# microbenchmark on this GB300 (rsqrt.approx 15.9, ex2.approx 31.7).  The pass
# cannot beat max(SFU time, FMA time) per unit.
SFU_RSQRT_PER_SM_CLK = 15.9
SFU_EX2_PER_SM_CLK = 31.7
FMA_PER_SM_CLK = 128
FMA_OPS_PER_PIXEL = 17
# DRAM bytes per event of one MLEM tile pass (dram__bytes_read.sum +
# dram__bytes_write.sum of one ncu-captured launch over 1e6 events of the
# 1 mm workload); the traffic grows with the events.
TILE_PASS_DRAM_B_PER_EVENT = 47.6
# The same for the accumulator-only tile pass of the 0.5 mm stress workload
# (one launch over its first 1e6 events; rho' re-read through L1/L2).
GLD_PASS_DRAM_B_PER_EVENT = 66.0
# Warp instructions issued per in-window pixel evaluation (smsp__inst_executed.sum
# / W of the same captures): the pass is issue-bound, so this is its tracked cost.
TILE_PASS_WARP_INST_PER_EVAL = 1.06
GLD_PASS_WARP_INST_PER_EVAL = 1.16


def roofline_basis(device: int):
    """Peak pixel-evaluation rate of the MLEM pass on this device (per second)
    and the formula behind it."""
    import torch
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    f = float(_peaks().get("sm_max_mhz", 2070.0)) * 1e6
    t_sfu = 1.0 / SFU_RSQRT_PER_SM_CLK + 1.0 / SFU_EX2_PER_SM_CLK     # clocks per unit per SM
    t_fma = FMA_OPS_PER_PIXEL / FMA_PER_SM_CLK
    return {"peak": sms * f / max(t_sfu, t_fma), "sfu_only": sms * f / t_sfu,
            "basis": f"{sms} SMs x {f/1e6:.0f} MHz / max(1/{SFU_RSQRT_PER_SM_CLK} + "
                     f"1/{SFU_EX2_PER_SM_CLK} SFU clk, {FMA_OPS_PER_PIXEL}/{FMA_PER_SM_CLK} "
                     f"FMA clk) per pixel evaluation"}


def roofline_dict(W, t_pass, basis, kernel, traffic=None, inst_per_eval=None):
    """The bench line's roofline object for a pass of W pixel evaluations
    taking t_pass seconds (None when not timed)."""
    achieved = W / t_pass if t_pass else None
    return {"bound": "alu", "achieved": achieved / 1e9 if achieved else None,
            "peak": basis["peak"] / 1e9, "unit": "Gpixel-evals/s",
            "frac": achieved / basis["peak"] if achieved else None,
            "frac_of_sfu_bound": achieved / basis["sfu_only"] if achieved else None,
            "traffic": traffic,
            "traffic_basis": ("ncu DRAM bytes of one 1e6-event launch, scaled by events"
                              if traffic is not None else None),
            "warp_inst_per_eval": inst_per_eval,
            "kernel": kernel, "pixel_evals_per_launch": W,
            "launch_ms": t_pass * 1e3 if t_pass else None,
            "peak_basis": basis["basis"]}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_baseline(workload, target_s: float = 12.0):
    """Time the FP64 oracle (all host cores, as it stands) on a bounded sample:
    one MLEM iteration over the first n events of the workload, n sized for
    about target_s seconds.  Returns the baseline dict."""
    import oracle
    from oracle import Setup
    st = Setup.from_workload(workload)
    s = oracle.sensitivity(st)
    w_small = _replace(workload, n_events=2000)
    ev = w_small.events()
    t0 = time.perf_counter()
    oracle.mlem(st, ev, 1, s=s)
    dt = max(time.perf_counter() - t0, 1e-3)
    n = int(min(workload.n_events, max(2000, 2000 * target_s / dt)))
    ev = _replace(workload, n_events=n).events()
    t0 = time.perf_counter()
    oracle.mlem(st, ev, 1, s=s)
    dt = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    # the same oracle on one thread, over a sample 1/cores as long (about as many seconds)
    n1 = max(500, n // max(1, cores))
    st1 = _replace(st, n_threads=1)
    t0 = time.perf_counter()
    oracle.mlem(st1, ev_first(workload, n1), 1, s=s)
    dt1 = time.perf_counter() - t0
    return {"value": n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"1 iteration of Eq. iter over the first {n} events of the "
                      f"{workload.name} workload ({workload.ny}x{workload.nz} grid), FP64, "
                      f"{dt:.1f} s",
            "single_thread": {"value": n1 / dt1, "unit": UNIT, "cores": 1,
                              "sample": f"the first {n1} events, {dt1:.1f} s"}}


def ev_first(workload, n):
    """The first n events of the workload (the seed's first n draws)."""
    return _replace(workload, n_events=n).events()


def _replace(w, **kw):
    from dataclasses import replace
    return replace(w, **kw)


def run_reference(args, workload):
    """The reference arm: the FP64 CPU oracle, timed as it stands."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    from oracle import Setup
    st = Setup.from_workload(workload)
    s = oracle.sensitivity(st)
    # size one step (one iteration over a sample) so the whole run takes ~minutes
    probe = _replace(workload, n_events=2000).events()
    t0 = time.perf_counter()
    oracle.mlem(st, probe, 1, s=s)
    per_event = (time.perf_counter() - t0) / 2000
    budget = 150.0 / max(1, args.steps + args.warmup)
    n = int(min(workload.n_events, max(2000, budget / per_event)))
    ev = _replace(workload, n_events=n).events()
    rho = None
    for _ in range(args.warmup):
        rho, _ = oracle.mlem(st, ev, 1, rho0=rho, s=s)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        rho, _ = oracle.mlem(st, ev, 1, rho0=rho, s=s)
    dt = time.perf_counter() - t0
    value = n * args.steps / dt
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded phantom events)",
        "config": {"workload": workload.name, "events": workload.n_events, "grid": [workload.ny, workload.nz],
                   "pixel_mm": workload.dz, "sigma_z": workload.sigma_z, "sigma_dl": workload.sigma_dl,
                   "cut": workload.cut, "step": f"1 MLEM iteration over a {n}-event sample"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{n} events of {workload.name}, 1 iteration per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def rel_err_images(a, b, frac=0.01):
    """max |a - b| / b over the pixels of b above frac * max(b)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    m = b > frac * b.max()
    return float(np.max(np.abs(a[m] - b[m]) / b[m])) if m.any() else 0.0


def bench_batched(steps: int, warmup: int, k: int = 64, seed: int = 3):
    """Batched vs plain on the batched workload: k reconstructions (seeded 2-6
    ellipse phantoms, 1/2/4 mm pixels, 1e4-2e6 events, sigma_z 8-12 mm,
    sigma_dl 30-50 mm, 10 iterations each).  Plain: one context per
    reconstruction, iterated one after another on one stream.  Batched: one
    tsp_batch with the autotuned schedule.  One step = reset every image and
    apply the 10 iterations to all k.  Images of the two forms are compared."""
    import torch
    from paper_1502_07478_gb300 import Batch, Recon
    from synth import batched_instances
    ws = batched_instances(k, seed=seed)
    evs = [w.events() for w in ws]
    n_iter = ws[0].n_iter
    total = sum(w.n_events for w in ws)
    stream = torch.cuda.current_stream()

    def timed(step):
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    plain = []
    for w, ev in zip(ws, evs):
        r = Recon.from_workload(w)
        r.upload_events(*ev)
        plain.append(r)

    def plain_step():
        for r in plain:
            r.set_image(None)
            r.iterate(n_iter)

    l0 = sum(r.stats()["launches"] for r in plain)
    t_plain = timed(plain_step)
    l_plain = (sum(r.stats()["launches"] for r in plain) - l0) / (steps + warmup)
    img_plain = [r.read_image().cpu().numpy() for r in plain]
    for r in plain:
        r.close()

    b = Batch.from_workloads(ws)
    for i, ev in enumerate(evs):
        b.upload_events(i, *ev)
    t0 = time.perf_counter()
    sched, tuned_ms = b.autotune()
    t_tune = time.perf_counter() - t0

    def batch_step():
        for i in range(k):
            b.set_image(i, None)
        b.iterate(n_iter)

    b0 = b.stats(0)["launches"]
    t_batch = timed(batch_step)
    l_batch = (b.stats(0)["launches"] - b0) / (steps + warmup)
    err = max(rel_err_images(b.read_image(i).cpu().numpy(), img_plain[i]) for i in range(k))
    used = sum(b.stats(i)["n_used"] for i in range(k))
    b.close()
    return {"workload": f"batched_{k}", "instances": k, "events": total,
            "iterations_per_step": n_iter, "steps": steps,
            "pixel_mm": sorted({w.dz for w in ws}),
            "batched": total * n_iter * steps / t_batch, "plain": total * n_iter * steps / t_plain,
            "unit": UNIT, "speedup": t_plain / t_batch,
            "ms_per_step": {"batched": 1e3 * t_batch / steps, "plain": 1e3 * t_plain / steps},
            "kernel_launches_per_step": {"batched": l_batch, "plain": l_plain},
            "rel_err_batched_vs_plain": err, "n_used": used,
            "schedule": sched, "autotune": {"best_pass_ms": tuned_ms, "seconds": t_tune}}


def _make_chunk(args):
    name, n_events, k, chunk = args
    from synth import make_workload
    return make_workload(name, n_events=n_events).event_chunk(k, chunk)


def _make_events(args):
    name, seed = args
    from synth import make_workload
    return make_workload(name, seed=seed).events()


def bench_adjoint(reps: int = 5):
    """The adjoint workload (350 x 250 at 2 mm, 1e6 events): time of one
    log-likelihood + gradient pass (L, g_rho, g_sigma; denominators recomputed)
    at sigma = (14, 55) after 5 MLEM iterations, wall clock around the
    synchronising call, best of reps."""
    from paper_1502_07478_gb300 import Recon
    from synth import make_workload
    w = make_workload("adjoint_2mm")
    r = Recon.from_workload(w)
    r.upload_events(*w.events())
    r.iterate(5)
    r.set_sigma(14.0, 55.0)
    r.loglik_grad()
    best = float("inf")
    for _ in range(reps):
        t0 = time.perf_counter()
        r.loglik_grad()
        best = min(best, time.perf_counter() - t0)
    W = r.stats()["n_window"]
    r.close()
    return {"workload": w.name, "events": w.n_events, "grid": [w.ny, w.nz],
            "ms_per_gradient": 1e3 * best, "events_per_s": w.n_events / best,
            "pixel_evals_per_s": W / best,
            "includes": "rho' refresh, gradient pass, g = s(A - 1), readout of L and g_sigma"}


STRESS_CHUNK = 10_000_000
ADJ_INSTANCES = 16


def _adjoint_instances():
    from synth import make_workload
    return [make_workload("adjoint_2mm", seed=4 + 1000 * (i + 1)) for i in range(ADJ_INSTANCES)]


def start_stress_inputs(workload, chunk: int = STRESS_CHUNK):
    """Start generating the stress workload's streamed chunks and the 16 adjoint
    event sets in a spawned process pool (no GPU use); returns (pool, chunk
    futures, adjoint futures).  The default run starts this before its main
    leg so that generation overlaps the GPU timing."""
    import concurrent.futures as cf
    import multiprocessing as mp
    sizes = workload.chunk_sizes(chunk)
    ex = cf.ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 4),
                                mp_context=mp.get_context("spawn"))
    cf_chunks = [ex.submit(_make_chunk, (workload.name, workload.n_events, k, chunk))
                 for k in range(len(sizes))]
    cf_adj = [ex.submit(_make_events, ("adjoint_2mm", w.seed)) for w in _adjoint_instances()]
    return ex, cf_chunks, cf_adj


def stress_record(workload, inputs, steps: int, warmup_iters: int, with_e2e: bool,
                  chunk: int = STRESS_CHUNK):
    """The stress workload: 0.5 mm pixels (1400 x 1000), 1e8 events streamed to
    the device in 1e7-event pinned chunks (tsp_begin/append/end_events), 10
    iterations per step after ``warmup_iters`` single iterations; plus the
    adjoint pass of 16 independent 2 mm reconstructions (1e6 events each)
    batched in one launch against 16 plain passes.  Returns the record (dict)
    with its own roofline for the accumulator-only tile kernel."""
    import torch
    from paper_1502_07478_gb300 import Batch, Recon
    ex, cf_chunks, cf_adj = inputs
    chunks = [f.result() for f in cf_chunks]
    adj_ev = [f.result() for f in cf_adj]
    ex.shutdown()
    adj = _adjoint_instances()
    sizes = workload.chunk_sizes(chunk)
    torch.cuda.set_device(0)
    pinned = [[torch.from_numpy(x).pin_memory() for x in c] for c in chunks]
    del chunks
    stream = torch.cuda.current_stream()
    n = workload.n_events
    n_iter = workload.n_iter
    r = Recon.from_workload(workload)
    out = torch.empty((workload.ny, workload.nz), dtype=torch.float32).pin_memory()

    def upload():
        r.begin_events(n)
        for c in pinned:
            r.append_events(*c)
        r.end_events()

    upload()                                  # allocation and first-use costs
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    upload()
    torch.cuda.synchronize()
    t_upload = time.perf_counter() - t0
    e2e = None
    if with_e2e:
        t0 = time.perf_counter()
        upload()
        r.iterate(n_iter)
        r.read_image(out=out.numpy())
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        e2e = {"value": n * n_iter / t_e2e, "unit": UNIT,
               "h2d_bytes_per_step": 12 * n, "d2h_bytes_per_step": 4 * workload.ny * workload.nz,
               "steps": 1, "includes": "streamed upload + binning + iterations + readout"}
    r.set_profiling(True)
    for _ in range(warmup_iters):
        r.iterate(1)
    r.set_image(None)
    torch.cuda.synchronize()
    st0 = r.stats()
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        r.set_image(None)
        r.iterate(n_iter)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    pass_ms = r.pass_times()
    st1 = r.stats()
    s_map = r.compute_sensitivity().double()
    rho = r.read_image().double()
    cons = float((s_map * rho).sum()) / max(1, st1["n_used"]) - 1.0
    r.close()
    del pinned

    # batched adjoint: 16 reconstructions, gradients at sigma = (14, 55)
    b = Batch.from_workloads(adj)
    plain = []
    for i, (w, ev) in enumerate(zip(adj, adj_ev)):
        b.upload_events(i, *ev)
        b.set_sigma(i, 14.0, 55.0)
        p = Recon.from_workload(w)
        p.upload_events(*ev)
        p.set_sigma(14.0, 55.0)
        plain.append(p)
    b.loglik_grad()
    for p in plain:
        p.loglik_grad(want_rho=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Lb, gsb = b.loglik_grad()
    t_b = time.perf_counter() - t0
    t0 = time.perf_counter()
    res = [p.loglik_grad() for p in plain]
    t_p = time.perf_counter() - t0
    gerr = max(float((b.read_image(i, 2) - res[i][1]).norm() / res[i][1].norm())
               for i in range(len(adj)))
    Lerr = max(abs(Lb[i] / res[i][0] - 1) for i in range(len(adj)))
    n_adj = sum(w.n_events for w in adj)
    b.close()
    for p in plain:
        p.close()

    W = st1["n_window"]
    t_pass = float(np.mean(pass_ms[-n_iter:])) / 1e3 if pass_ms else float("nan")
    roof = roofline_basis(0)
    return {
        "metric": METRIC, "value": n * n_iter * steps / (ms / 1e3), "unit": UNIT,
        "n_gpus": 1, "steps": steps, "warmup": warmup_iters, "ms_per_step": ms / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded phantom events, streamed form: chunk k from seed (5, k))",
        "config": {"workload": workload.name, "events": n, "iterations_per_step": n_iter,
                   "grid": [workload.ny, workload.nz], "pixel_mm": workload.dz,
                   "sigma_z": workload.sigma_z, "sigma_dl": workload.sigma_dl,
                   "cut": workload.cut, "form": "plain, streamed upload",
                   "upload": f"{len(sizes)} pinned chunks of <= {chunk} events",
                   "warmup": f"{warmup_iters} single iterations",
                   "l2": "inputs larger than L2", "parallelism": "1 GPU"},
        "roofline": roofline_dict(W, t_pass if pass_ms else None, roof,
                                  "k_tiles (accumulator-only tiles, rho' from global), per launch",
                                  traffic=(GLD_PASS_DRAM_B_PER_EVENT * n
                                           if workload.name == "stress_05mm" else None),
                                  inst_per_eval=(GLD_PASS_WARP_INST_PER_EVAL
                                                 if workload.name == "stress_05mm" else None)),
        "upload_s": t_upload,
        "e2e": e2e,
        "adjoint_batched_16": {"instances": ADJ_INSTANCES, "events": n_adj, "grid": [350, 250],
                               "batched_s": t_b, "plain_s": t_p, "speedup": t_p / t_b,
                               "events_per_s_batched": n_adj / t_b,
                               "max_rel_err_g_rho_vs_plain": gerr, "max_rel_err_L_vs_plain": Lerr},
        "gpu_launches": st1["launches"] - st0["launches"], "clocks": clk,
        "checks": {"conservation_rel": cons, "n_used": st1["n_used"],
                   "n_outliers": st1["n_outliers"], "n_empty": st1["n_empty"]},
    }


def main_batched(args, ws):
    """--workload batched_64: the batched-vs-plain comparison alone, as the
    line (value = the batched form's event-iterations/s)."""
    if ws > 1:
        print(json.dumps({"error": "the batched workload runs on one GPU"}))
        return 1
    import torch
    if not torch.cuda.is_available():
        print(json.dumps({"error": "no CUDA device"}))
        return 1
    torch.cuda.set_device(0)
    clocks = ClockSampler(0)
    clocks.start()
    b = bench_batched(steps=args.steps, warmup=max(1, args.warmup))
    clk = clocks.stop()
    line = {"metric": METRIC, "value": b["batched"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": max(1, args.warmup),
            "ms_per_step": b["ms_per_step"]["batched"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded phantom events, 64 reconstructions)",
            "config": {"workload": "batched_64", "instances": b["instances"], "events": b["events"],
                       "iterations_per_step": b["iterations_per_step"],
                       "pixel_mm": b["pixel_mm"], "form": "batched (one Batch) vs 64 plain contexts",
                       "parallelism": "1 GPU"},
            "batched": b, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def bench_stress(args, workload):
    """--workload stress_05mm: the stress record as the bench line, with its
    end-to-end leg and the CPU baseline.  Warm-up is 3 single iterations."""
    rec = stress_record(workload, start_stress_inputs(workload), steps=args.steps,
                        warmup_iters=3, with_e2e=True)
    rec["cpu_baseline"] = None if args.no_cpu_baseline else cpu_baseline(workload, target_s=10.0)
    print(json.dumps(rec), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tsp", choices=["tsp", "reference"])
    ap.add_argument("--workload", default="paper_1mm",
                    help="paper_1mm (default), stress_05mm, batched_64, or another synth workload")
    ap.add_argument("--n-events", type=int, default=None, help="override the event count")
    ap.add_argument("--iters", type=int, default=None, help="override iterations per step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched-vs-plain comparison")
    ap.add_argument("--no-stress", action="store_true",
                    help="skip the stress record (1e8 events at 0.5 mm, batched adjoint)")
    ap.add_argument("--variant", default="tiles", choices=["tiles", "thread"],
                    help="MLEM pass: the tile kernel, or one thread per event (ablation)")
    args = ap.parse_args()

    from synth import make_workload
    ws, rank, local = _dist()
    if args.workload == "batched_64":
        if args.impl == "reference":
            if rank == 0:
                print(json.dumps({"impl": "reference", "unavailable":
                                  "the batched comparison has no CPU reference arm; the oracle "
                                  "is timed on the paper_1mm workload"}))
            return 0
        return main_batched(args, ws)
    over = {}
    if args.n_events:
        over["n_events"] = args.n_events
    if args.iters:
        over["n_iter"] = args.iters
    workload = make_workload(args.workload, **over)
    if args.impl == "reference":
        return run_reference(args, workload)

    if workload.name == "stress_05mm":
        if ws > 1:
            print(json.dumps({"error": "the stress workload runs on one GPU"}))
            return 1
        return bench_stress(args, workload)
    # the stress record's inputs are generated by a spawned pool while the
    # main leg runs (no GPU use in the pool)
    stress_inputs = None
    if ws == 1 and not args.no_stress and args.workload == "paper_1mm" and not args.n_events:
        stress_inputs = start_stress_inputs(make_workload("stress_05mm"))
    import torch
    if not torch.cuda.is_available():
        print(json.dumps({"error": "no CUDA device"}))
        return 1
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
        # one reconstruction of ws x n events: rank r holds its seeded share
        workload = _replace(workload, seed=workload.seed + 1000 * rank)

    from paper_1502_07478_gb300 import Recon
    from paper_1502_07478_gb300.shard import sharded_iterate
    ev = workload.events()
    n_iter = workload.n_iter
    n = workload.n_events
    # pinned host copies for the end-to-end leg
    pinned = [torch.from_numpy(e).pin_memory() for e in ev]
    r = Recon.from_workload(workload)
    r.set_variant(args.variant)
    r.upload_events(*ev)
    r.set_profiling(True)
    stream = torch.cuda.current_stream()
    buf = torch.empty((workload.ny, workload.nz), dtype=torch.float32, device="cuda")

    def iterations():
        if pg is None:
            r.iterate(n_iter)           # graph replay of n_iter updates
        else:                           # back-projection, NCCL all-reduce, update
            sharded_iterate(r, n_iter, pg.all_reduce, buf)

    def step():
        r.set_image(None)
        iterations()

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    st0 = r.stats()
    if pg:
        pg.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    pass_ms = r.pass_times()
    st1 = r.stats()
    launches = st1["launches"] - st0["launches"]
    used = st1["n_used"]
    if pg:
        t = torch.tensor([ms], device="cuda")
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms = float(t.item())
        u = torch.tensor([used], dtype=torch.int64, device="cuda")
        pg.all_reduce(u)
        used = int(u.item())
        # the back-projection alone, for the roofline (no graph, one launch)
        torch.cuda.synchronize()
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        r.backproject(out=buf)
        b1.record(stream)
        torch.cuda.synchronize()
        pass_ms = [b0.elapsed_time(b1)]
    sec = ms / 1e3
    value = ws * n * n_iter * args.steps / sec

    # parity check at the benchmark's own size and launch configuration:
    # count conservation sum_l s_l rho_l = N_used (all ranks) after the last
    # iteration
    s_map = r.compute_sensitivity().double()
    rho = r.read_image().double()
    cons = float((s_map * rho).sum()) / max(1, used) - 1.0

    # dominant kernel: the MLEM tile kernel; algorithmic work = in-window pixel
    # evaluations per launch (exact count from the event preparation)
    W = st1["n_window"]
    t_pass = float(np.mean(pass_ms)) / 1e3 if pass_ms else None
    roofline = roofline_dict(
        W, t_pass, roofline_basis(local),
        ("k_tiles" if args.variant == "tiles" else "k_thread_events") + " (MLEM pass, per launch)",
        traffic=(TILE_PASS_DRAM_B_PER_EVENT * n
                 if workload.name == "paper_1mm" and args.variant == "tiles" else None),
        inst_per_eval=(TILE_PASS_WARP_INST_PER_EVAL
                       if workload.name == "paper_1mm" and args.variant == "tiles" else None))

    e2e = None
    if not args.no_e2e:
        pinned_out = torch.empty((workload.ny, workload.nz), dtype=torch.float32).pin_memory()
        r.set_profiling(False)

        def e2e_step():
            r.upload_events(*pinned)
            iterations()
            r.read_image(out=pinned_out.numpy())

        e2e_step()
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        t0 = time.perf_counter()
        k_e2e = max(1, min(args.steps, 3))
        for _ in range(k_e2e):
            e2e_step()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if pg:
            t = torch.tensor([dt], device="cuda")
            pg.all_reduce(t, op=pg.ReduceOp.MAX)
            dt = float(t.item())
        e2e = {"value": ws * n * n_iter * k_e2e / dt, "unit": UNIT,
               "h2d_bytes_per_step": int(sum(p.numel() * 4 for p in pinned)),
               "d2h_bytes_per_step": int(pinned_out.numel() * 4), "steps": k_e2e}
    r.close()

    batched = adjoint = stress = None
    if not args.no_batched and ws == 1:
        batched = bench_batched(steps=max(1, min(args.steps, 2)), warmup=1)
        adjoint = bench_adjoint()
    if stress_inputs is not None:
        stress = stress_record(make_workload("stress_05mm"), stress_inputs, steps=1,
                               warmup_iters=1, with_e2e=False)

    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return 0
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        cpu = cpu_baseline(workload)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded phantom events; the paper's event sets are not published)",
        "config": {"workload": workload.name, "events": n * ws, "events_per_gpu": n,
                   "iterations_per_step": n_iter,
                   "grid": [workload.ny, workload.nz], "pixel_mm": workload.dz,
                   "sigma_z": workload.sigma_z, "sigma_dl": workload.sigma_dl,
                   "cut": workload.cut, "form": "plain",
                   "kernel_variant": args.variant,
                   "l2": "inputs larger than L2 (prepared events 24 B x 1e7 = 240 MB)",
                   "parallelism": (f"one reconstruction, events sharded over {ws} GPUs, NCCL "
                                   f"all-reduce of the back-projection each iteration"
                                   if ws > 1 else "1 GPU")},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "batched": batched,
        "adjoint": adjoint, "stress": stress,
        "gpu_launches": launches,
        "clocks": clk,
        "checks": {"conservation_rel": cons, "n_used": used,
                   "n_outliers": st1["n_outliers"], "n_empty": st1["n_empty"]},
    }
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
