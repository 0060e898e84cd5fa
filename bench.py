#!/usr/bin/env python
"""Benchmark of the split shallow-water step (Cliffs, arXiv 1410.0753) on GB300.

Headline workload: the 8192 x 8192 Cartesian shelf-and-islands grid (67 M cells, 50 m, ten
conical islands with their shorelines, an N-wave line source; workloads.shelf_islands), the
largest single-GPU configuration, as a pure step (no outputs due). One bench step = one model
time step: one launch of the fused x-sweep + y-sweep kernel. Its 1.9 GB working set is far
larger than the 129 MB L2, so consecutive steps cannot be served from L2 and no flush is
needed between them.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cuda|reference]

Timing: W untimed steps, then K steps, every step kernel timed with CUDA events on the grid's
stream; the K steps are bracketed by a barrier and a device synchronisation; the maximum over
ranks is reported. With N > 1 each rank advances its own replica of the grid (the path does
not shard: replicas only).

With one GPU the line also carries ``forms``: the 2048 x 2048 geographic grid with max-wave,
64 gauges and 4 enclosed-grid boundary series every step (L2 flushed before each step), the
stress grid with max-wave every step, the batched ensemble (256 scenarios of uneven duration
on a shared 512 x 512 bathymetry in one persistent, graph-captured launch) and the adjoint
(gradient of a 32-gauge misfit over 2000 steps of a 1024 x 1024 grid), the batched and
adjoint forms next to the plain single-scenario forward on the same GPU; ``oracle_error``
(FP32 against the FP64 oracle for each of the five workloads) and ``cpu_baselines`` (the
oracle on one host thread and on all host cores, for each workload).

``--impl reference`` times the FP64 CPU oracle on the same workload on the host cores.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gcell-updates/s and % HBM roofline (FP32 fwd, batched, adjoint) vs FP64 oracle error"
UNIT = "Gcell-updates/s"
BYTES_PER_CELL = 28      # read eta, u, v, d; write eta, u, v (FP32)
HEADLINE = "shelf_islands_8192x8192"
HORIZON = 2000           # the workload's stated number of steps


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernel_source_sha():
    h = hashlib.sha256()
    for f in ("sweep.cuh", "step_kernels.cuh", "cliffs_step.cu", "internal.h"):
        h.update(open(os.path.join(ROOT, "paper_1410_0753_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled(name, rows_per_warp=None):
    """The committed ncu summary of a kernel (DRAM bytes and warp-instructions per launch),
    if it was taken on this source and at this run's tile shape; else (None, why)."""
    p = os.path.join(ROOT, "profiles", name + ".json")
    try:
        d = json.load(open(p))
    except Exception:
        return None, None
    if d.get("source_sha") != kernel_source_sha():
        return None, "stale"
    if d.get("rows_per_warp") and rows_per_warp and d["rows_per_warp"] != rows_per_warp:
        t = d.get("tiles", {}).get(str(rows_per_warp))
        if not t:
            return None, "profiled at %d rows per warp, this run took %d" % (d["rows_per_warp"], rows_per_warp)
        d = dict(d, rows_per_warp=rows_per_warp, **t)
    return d, d.get("note")


def issue_roof(prof, cells, value, sm_mhz, sms):
    """The instruction-issue ceiling of the step kernel: each of an SM's 4 schedulers issues
    at most one warp-instruction per cycle, so a kernel issuing I warp-instructions per cell
    cannot exceed 4 * SMs * clock / I cell-updates/s, whatever its bytes."""
    if not prof or not prof.get("warp_inst_per_launch") or not sm_mhz:
        return None
    ipc = prof["warp_inst_per_launch"] / cells
    peak = 4.0 * sms * sm_mhz * 1e6 / ipc / 1e9
    return {"warp_inst_per_cell": ipc, "peak": peak, "unit": "Gcell-updates/s", "frac": value / peak,
            "sms": sms, "sm_mhz": sm_mhz}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                                       "-i", str(device_id), "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [l.split(",") for l in open(self.f.name).read().strip().splitlines() if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for k, n in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def bench_config(w, world):
    """The workload description both arms print (identical keys and values)."""
    return {"workload": w.name, "cells": int(w.cells), "grid": "%d x %d Cartesian, dx = 50 m" % (w.nx, w.ny),
            "outputs": "none due (pure step)", "steps_horizon": HORIZON,
            "l2": "working set %.2f GB, larger than the 129 MB L2: no flush between steps"
                  % (7 * 4 * w.cells / 1e9),
            "parallelism": "replicas" if world > 1 else "single"}


def run_reference(args, world, rank):
    """The FP64 oracle as it stands, on the host cores, for the same workload and metric. The
    W warm-up steps and the K timed steps each run as one oracle call. Each step covers the
    full grid when K + W steps fit in about 150 s at the oracle's speed on the box (~0.12
    Gcell/s on 16 cores); otherwise a band of rows across the whole width (the line source
    and its wave run along x), so that the run stays within a few minutes."""
    if rank != 0:
        return
    import oracle
    import workloads
    w = workloads.shelf_islands(args.nx, args.ny, steps=HORIZON)
    config = bench_config(w, world)
    threads = oracle.threads(os.cpu_count() or 1)
    d = oracle.depth_filter(w.depth, w.filter_alpha, w.filter_min_depth)[0]
    budget_cells = 0.12e9 * 150.0 / max(1, args.steps + args.warmup)
    rows = int(min(w.ny, max(64, budget_cells // w.nx)))
    if rows < w.ny:
        j0 = max(0, min(w.ny - rows, w.ny // 2 - rows // 2))
        sl = slice(j0, j0 + rows)
        w = workloads.Workload(w.name + "_band%d" % rows, w.nx, rows, w.coords, w.x, w.y[sl], w.depth[sl],
                               w.eta0[sl], w.dt, w.steps, h_min=w.h_min, manning_n2=w.manning_n2,
                               maxout=w.maxout, gout=w.gout, bndout=w.bndout)
        d = d[sl]
        sample = "a band of %d of %d rows across the full width" % (rows, args.ny)
    else:
        sample = "the full grid"
    p = oracle.params_from(w)
    kw = dict(maxout=w.maxout, gout=w.gout)
    r = oracle.run(p, w.x, w.y, d, w.eta0, nsteps=args.warmup, **kw)
    t = time.perf_counter()
    oracle.run(p, w.x, w.y, d, r["eta"], r["u"], r["v"], nsteps=args.steps, step0=args.warmup, **kw)
    el = time.perf_counter() - t
    cells = w.nx * w.ny
    val = cells * args.steps / el / 1e9
    line = {"metric": METRIC, "value": val, "unit": UNIT, "impl": "reference",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": "%d consecutive steps of %s (%d cells per step; FP64 C++ oracle, "
                                       "OpenMP over lines)" % (args.steps, sample, cells)},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _event_ms(torch, stream, fn):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


def measure_forms(torch, stream, only=None, adjoint_steps=None, ensemble=None, rows_per_warp=0):
    """The batched ensemble (256 scenarios of uneven duration on one 512 x 512 bathymetry, one
    persistent graph-captured launch) and the adjoint (1024 x 1024, 2000 steps, checkpoint
    every 100), each reported against the plain single-scenario forward on this GPU."""
    import workloads
    from paper_1410_0753_gb300 import CliffsGrid
    out = {}
    s = stream.cuda_stream
    if only in (None, "spherical"):
        out["spherical"] = _form_spherical(torch, stream, workloads, CliffsGrid, rows_per_warp=rows_per_warp)
    if only in (None, "batched"):
        out["batched"] = _form_batched(torch, stream, workloads, CliffsGrid, ensemble)
    if only in (None, "stress"):
        out["stress"] = _form_stress(torch, stream, workloads, CliffsGrid)
    if only in (None, "adjoint"):
        out["adjoint"] = _form_adjoint(torch, stream, workloads, CliffsGrid, adjoint_steps)
    return out


def _form_batched(torch, stream, workloads, CliffsGrid, ensemble=None):
    # ensemble = (scenarios, shortest, longest duration) shrinks the 256-scenario ensemble to
    # a case small enough for a profiler capture
    s = stream.cuda_stream
    w = workloads.ensemble_512() if ensemble is None else \
        workloads.ensemble_512(batch=ensemble[0], dmin=ensemble[1], dmax=ensemble[2])
    g = CliffsGrid.from_workload(w, stream=s)
    g.set_bathy(w.x, w.y, w.depth, True, w.filter_alpha, w.filter_min_depth)
    eta0 = w.eta0.astype(np.float32)
    g.set_initial(eta0)
    g.set_durations(w.durations)
    tune = g.autotune(2)
    g.step(10, persistent=True)                     # capture the graph, warm up
    g.set_initial(eta0)
    T = int(w.durations.max())
    ms_b = _event_ms(torch, stream, lambda: g.step(T, persistent=True))
    useful = float(w.durations.sum()) * w.cells
    g.close()
    g1 = CliffsGrid.from_workload(w, batch=1, stream=s)
    g1.set_bathy(w.x, w.y, w.depth, True, w.filter_alpha, w.filter_min_depth)
    g1.set_initial(eta0[0])
    g1.step(20)
    n1 = 1000
    ms_1 = _event_ms(torch, stream, lambda: g1.step(n1))
    g1.close()
    v_b = useful / (ms_b / 1e3) / 1e9
    v_1 = w.cells * n1 / (ms_1 / 1e3) / 1e9
    # per useful cell-update: eta, u and v read and written (FP32); the one depth plane is
    # shared by every live scenario, so it adds 4 B / batch
    bpc = 24.0 + 4.0 / w.batch
    peaks, _ = measured_peaks()
    return {
        "workload": w.name, "scenarios": int(w.batch), "durations": [int(w.durations.min()), int(w.durations.max())],
        "value": v_b, "unit": UNIT, "ms": ms_b, "launches": 1,
        "bytes_per_cell": bpc, "achieved_gbs": v_b * bpc, "frac": v_b * bpc / peaks["hbm_gbs"],
        "rows_per_warp": min(tune, key=tune.get) if tune else None,
        "single_scenario_forward": {"value": v_1, "unit": UNIT, "steps": n1,
                                    "note": "one scenario, one launch per step, same grid"},
        "vs_single_scenario_forward": v_b / v_1,
        "note": "useful cell-updates (each scenario up to its own duration) / time of one "
                "persistent, cooperative, graph-captured launch"}


def _form_stress(torch, stream, workloads, CliffsGrid):
    # the stress grid (8192 x 8192, shorelines around 10 islands) with max-wave every step
    s = stream.cuda_stream
    w = workloads.shelf_islands()
    peaks, _ = measured_peaks()
    out = {"workload": w.name, "cells": w.cells}
    for tag, maxout, bpc in (("maxwave_every_step", 1, 36),):
        g = CliffsGrid.from_workload(w, stream=s, maxout=maxout, gauges=[], nests=[])
        g.set_bathy(w.x, w.y, w.depth, True, w.filter_alpha, w.filter_min_depth)
        g.set_initial(w.eta0.astype(np.float32))
        tune = g.autotune(2)
        g.step(5)
        n = 60
        ms = _event_ms(torch, stream, lambda: g.step(n))
        v = w.cells * n / (ms / 1e3) / 1e9
        out[tag] = {"value": v, "unit": UNIT, "steps": n, "ms_per_step": ms / n,
                    "bytes_per_cell": bpc, "achieved_gbs": v * bpc,
                    "frac": v * bpc / peaks["hbm_gbs"],
                    "rows_per_warp": min(tune, key=tune.get) if tune else None}
        g.close()
    return out


def _form_spherical(torch, stream, workloads, CliffsGrid, steps=20, rows_per_warp=0):
    """The 2048 x 2048 geographic grid (1 arc-minute) with every output due every step:
    max-wave, 64 gauges and the boundary series of 4 enclosed grids; L2 (~150 MB working set)
    flushed by a 256 MiB device write before every timed step."""
    s = stream.cuda_stream
    w = workloads.spherical_coast(2048, 2048, steps=3600)
    g = CliffsGrid.from_workload(w, stream=s)
    g.set_bathy(w.x, w.y, w.depth, True, w.filter_alpha, w.filter_min_depth)
    g.set_initial(w.eta0.astype(np.float32))
    if rows_per_warp:                     # a fixed tile (to profile the configuration a run chose)
        g.set_rows_per_warp(rows_per_warp)
        rows = rows_per_warp
    else:
        tune = g.autotune(3)
        rows = min(tune, key=tune.get) if tune else None
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for i in range(5):
        flush.fill_(i & 0xFF)
        g.step(1)
    torch.cuda.synchronize()
    g.kernel_time(-1)
    g.kernel_time(1)
    for i in range(steps):
        flush.fill_((i + 1) & 0xFF)
        g.step(1)
    torch.cuda.synchronize()
    ms, launches = g.kernel_time(0)
    g.close()
    del flush
    v = w.cells * steps / (ms / 1e3) / 1e9
    peaks, _ = measured_peaks()
    prof, _ = profiled("k_step_fused_spherical_2048", rows)
    return {"workload": w.name, "cells": w.cells, "value": v, "unit": UNIT, "steps": steps,
            "ms_per_step": ms / steps, "launches": int(launches), "bytes_per_cell": 36,
            "achieved_gbs": v * 36, "frac": v * 36 / peaks["hbm_gbs"], "rows_per_warp": rows,
            "traffic": prof.get("dram_bytes_per_launch") if prof else None,
            "note": "max-wave, 64 gauges and 4 enclosed-grid boundary series every step; "
                    "L2 flushed before every timed step"}


def _form_adjoint(torch, stream, workloads, CliffsGrid, steps=None):
    s = stream.cuda_stream
    w = workloads.inversion_1024(steps=steps or 2000)
    g = CliffsGrid.from_workload(w, stream=s)
    g.set_bathy(w.x, w.y, w.depth, True, w.filter_alpha, w.filter_min_depth)
    e0 = w.eta0.astype(np.float32)
    g.set_initial(e0)
    g.autotune(2)
    n = w.steps
    seed = np.random.default_rng(1).standard_normal((n // w.gout + 1, len(w.gauges))).astype(np.float32)
    grad = torch.empty((w.ny, w.nx), dtype=torch.float32, device="cuda")
    g.adjoint(50, seed[:51], 100, grad)             # allocate work space, warm up
    g.set_initial(e0)
    g.step(10)
    g.set_initial(e0)
    ms_f = _event_ms(torch, stream, lambda: g.step(n))
    g.set_initial(e0)
    ms_a = _event_ms(torch, stream, lambda: g.adjoint(n, seed, 100, grad))
    # the same gradient after a forward that recorded its checkpoints (the autograd path)
    g.set_initial(e0)
    g.adjoint_record(100)
    ms_fr = _event_ms(torch, stream, lambda: g.step(n))
    ms_ar = _event_ms(torch, stream, lambda: g.adjoint_recorded(seed, grad))
    ref = grad.clone()
    # every state kept (a checkpoint each step: 12 B/node x n in HBM), so the gradient needs
    # no recomputation; the same bits as with checkpoints
    g.set_initial(e0)
    g.adjoint_record(1)
    g.step(n)                                      # grows the state store once
    g.set_initial(e0)                              # the record starts again, the store stays
    ms_f1 = _event_ms(torch, stream, lambda: g.step(n))
    ms_a1 = _event_ms(torch, stream, lambda: g.adjoint_recorded(seed, grad))
    same = bool(torch.equal(grad, ref))
    g.adjoint_record(0)
    g.close()
    return {
        "workload": w.name, "steps": n, "checkpoint_every": 100, "gauges": len(w.gauges),
        "gradient_ms": ms_a, "forward_ms": ms_f, "gradient_over_forward": ms_a / ms_f,
        "value": w.cells * n / (ms_a / 1e3) / 1e9, "unit": UNIT,
        "forward_value": w.cells * n / (ms_f / 1e3) / 1e9,
        "after_recorded_forward": {"forward_ms": ms_fr, "gradient_ms": ms_ar,
                                   "gradient_over_forward": ms_ar / ms_f,
                                   "note": "forward with a checkpoint kept every 100 steps "
                                           "(cliffs_adjoint_record), then cliffs_adjoint_recorded: "
                                           "segment recomputation + adjoint steps"},
        "after_forward_keeping_every_state": {
            "forward_ms": ms_f1, "gradient_ms": ms_a1, "gradient_over_forward": ms_a1 / ms_f,
            "state_bytes": 12 * w.cells * (n + 1), "same_gradient_bits": same,
            "note": "cliffs_adjoint_record(1): every state stays in HBM, the adjoint reads them "
                    "in place; no recomputation (timed on a second recorded run, the store "
                    "already grown, as in an inversion loop)"},
        "note": "gradient = checkpoint pass + segment recomputation + adjoint steps, one call "
                "of cliffs_adjoint_n; forward = cliffs_step_n over the same steps"}


# ---------------------------------------------------------------- FP64 oracle: error and CPU time

NEAR = 1e-5     # wet/dry decisions within 1e-5 max(1, |d|) of h_min count as near round-off


def _errors(eta32, eta64, d32, hmin, g32=None, g64=None, scale=None):
    """FP32 against FP64: per-gauge max_t|eta32 - eta64| / max_t|eta64| (absolute for traces
    below 1e-3 m), max |eta| difference over wet nodes, wet-mask mismatches away from
    round-off and the near-round-off count."""
    out = {}
    if g64 is not None and g64.shape[1]:
        rel, ab = [], []
        for k in range(g64.shape[1]):
            m = np.abs(g64[:, k, 0]).max()
            e = np.abs(np.asarray(g32[:, k, 0], np.float64) - g64[:, k, 0]).max()
            (rel if m >= 1e-3 else ab).append(e / m if m >= 1e-3 else e)
        out.update(gauges=int(g64.shape[1]), gauge_rel_max=float(max(rel)) if rel else None,
                   gauge_abs_max_small=float(max(ab)) if ab else None)
    wet32 = (eta32.astype(np.float32) + d32.astype(np.float32)) >= np.float32(hmin)
    h64 = eta64 + d32
    wet64 = h64 >= hmin
    near = np.abs(h64 - hmin) < NEAR * np.maximum(1.0, np.abs(d32))
    de = np.abs(eta32.astype(np.float64) - eta64)
    out.update(eta_abs_max=float(de[wet64].max(initial=0.0)),
               eta_scale=float(scale if scale is not None else np.abs(eta64[wet64]).max(initial=0.0)),
               mask_mismatch=int(((wet32 != wet64) & ~near).sum()), near_round_off=int(near.sum()))
    return out


def _timed_oracle(fn):
    t = time.perf_counter()
    r = fn()
    return r, time.perf_counter() - t


def oracle_reports(torch, stream):
    """For each of the five workloads: the FP32 GPU result against the FP64 oracle on the
    same seeded inputs (``oracle_error``), and the oracle's own speed on all host cores (that
    same comparison run) and on one host thread (a short sample) (``cpu_baselines``)."""
    import oracle
    import workloads
    from paper_1410_0753_gb300 import CliffsGrid
    s = stream.cuda_stream
    ncores = oracle.threads(os.cpu_count() or 1)
    errs, cpus = {}, {}

    def gpu(w, n, eta0=None, **kw):
        g = CliffsGrid.from_workload(w, stream=s, batch=1, **kw)
        g.set_bathy(w.x, w.y, w.depth, True, w.filter_alpha, w.filter_min_depth)
        g.set_initial((w.eta0 if eta0 is None else eta0).astype(np.float32))
        ms = _event_ms(torch, stream, lambda: g.step(n))
        e, _, _ = g.state()
        gg = g.gauges() if g.n_gauges else None
        g.close()
        return e, gg, w.cells * n / (ms / 1e3) / 1e9

    def depth32(w):
        # the oracle's own depth filter, rounded to FP32 as the device stores it
        d = oracle.depth_filter(w.depth, w.filter_alpha, w.filter_min_depth)[0]
        return d.astype(np.float32).astype(np.float64)

    def one_thread(w, d, n, eta0=None, **kw):
        oracle.threads(1)
        try:
            p = oracle.params_from(w)
            _, el = _timed_oracle(lambda: oracle.run(p, w.x, w.y, d, w.eta0 if eta0 is None else eta0,
                                                     nsteps=n, **kw))
        finally:
            oracle.threads(ncores)
        return {"value": w.cells * n / el / 1e9, "unit": UNIT, "cores": 1,
                "sample": "%d steps of the full %dx%d grid (%.1f s)" % (n, w.nx, w.ny, el)}

    def entry(name, w, cells, steps, el, sample, one):
        cpus[name] = {"all_cores": {"value": cells * steps / el / 1e9, "unit": UNIT, "cores": ncores,
                                    "sample": sample + " (%.1f s)" % el},
                      "one_thread": one}

    # 1: the 200^2 beach over its 1000 steps, every output
    w = workloads.beach_200()
    d32 = depth32(w)
    e32, g32, gv = gpu(w, w.steps)
    p = oracle.params_from(w)
    kw = dict(maxout=w.maxout, gout=w.gout, gauges=w.gauges)
    o, el = _timed_oracle(lambda: oracle.run(p, w.x, w.y, d32, w.eta0, nsteps=w.steps, **kw))
    errs[w.name] = dict(steps=w.steps, horizon=w.steps, gpu_value=gv, **_errors(e32, o["eta"], d32, w.h_min, g32, o["gauges"]))
    entry(w.name, w, w.cells, w.steps, el, "the full %d-step horizon" % w.steps, one_thread(w, d32, 200, **kw))
    # 2: the 2048^2 geographic grid, every output, over the steps that fit ~20 s of oracle time
    w = workloads.spherical_coast()
    d32 = depth32(w)
    p = oracle.params_from(w)
    kw = dict(maxout=w.maxout, gout=w.gout, gauges=w.gauges, bndout=w.bndout, nests=w.nests)
    _, t1 = _timed_oracle(lambda: oracle.run(p, w.x, w.y, d32, w.eta0, nsteps=2, **kw))
    n = int(max(10, min(400, 20.0 / max(t1 / 2, 1e-3))))
    e32, g32, gv = gpu(w, n)
    o, el = _timed_oracle(lambda: oracle.run(p, w.x, w.y, d32, w.eta0, nsteps=n, **kw))
    errs[w.name] = dict(steps=n, horizon=w.steps, gpu_value=gv, **_errors(e32, o["eta"], d32, w.h_min, g32, o["gauges"]))
    entry(w.name, w, w.cells, n, el, "the first %d steps, all outputs" % n, one_thread(w, d32, 2, **kw))
    # 3: the 8192^2 stress grid over 300 steps, on windows (the oracle re-runs the domain of
    # dependence, 3 nodes per sweep per step, around sampled blocks, whose results are exact)
    w = workloads.shelf_islands()
    k = 300
    d32 = depth32(w)
    e32, _, gv = gpu(w, k)
    half = 16
    R = 3 * k + 4 + half
    c = int(round(40.0e3 / 50.0))
    shift = int(np.sqrt(9.81 * 200.0) * w.dt * k / 50.0)
    centres = [(w.ny // 2, c + shift), (w.ny // 4, c - shift)]
    blocks = []
    for (cy, cx) in centres:
        j0, j1 = max(0, cy - R), min(w.ny, cy + R + 1)
        i0, i1 = max(0, cx - R), min(w.nx, cx + R + 1)
        pw = oracle.params(i1 - i0, j1 - j0, w.dt, w.coords, w.h_min, w.manning_n2, w.itopo, w.dwall,
                           w.transverse)
        dwin = d32[j0:j1, i0:i1]
        o = oracle.run(pw, w.x[i0:i1], w.y[j0:j1], dwin, w.eta0[j0:j1, i0:i1], nsteps=k)
        sl64 = (slice(cy - j0 - half, cy - j0 + half + 1), slice(cx - i0 - half, cx - i0 + half + 1))
        sl32 = (slice(cy - half, cy + half + 1), slice(cx - half, cx + half + 1))
        b = _errors(e32[sl32], o["eta"][sl64], dwin[sl64], w.h_min, scale=np.abs(w.eta0).max())
        b["moved"] = float(np.abs(o["eta"][sl64] - w.eta0[sl32]).max())
        blocks.append(b)
    errs[w.name] = dict(steps=k, horizon=w.steps, gpu_value=gv, blocks=blocks,
                        eta_rel_max=max(b["eta_abs_max"] / b["eta_scale"] for b in blocks),
                        mask_mismatch=sum(b["mask_mismatch"] for b in blocks),
                        note="%d blocks of %d^2 nodes around the wave fronts; each oracle window holds the "
                             "block's domain of dependence" % (len(blocks), 2 * half + 1))
    # the oracle's speed on the full grid: a few steps on all cores (about 0.5 s each)
    p = oracle.params_from(w)
    _, t1 = _timed_oracle(lambda: oracle.run(p, w.x, w.y, d32, w.eta0, nsteps=1))
    n = int(max(2, min(40, 10.0 / max(t1, 1e-3))))
    _, el = _timed_oracle(lambda: oracle.run(p, w.x, w.y, d32, w.eta0, nsteps=n))
    entry(w.name, w, w.cells, n, el, "%d steps of the full %dx%d grid" % (n, w.nx, w.ny), one_thread(w, d32, 1))
    # 4: one scenario of the ensemble (the shortest duration) over its duration
    w = workloads.ensemble_512()
    b = int(np.argmin(w.durations))
    n = int(w.durations[b])
    d32 = depth32(w)
    e32, g32, gv = gpu(w, n, eta0=w.eta0[b])
    p = oracle.params_from(w)
    kw = dict(maxout=w.maxout, gout=w.gout, gauges=w.gauges)
    o, el = _timed_oracle(lambda: oracle.run(p, w.x, w.y, d32, w.eta0[b], nsteps=n, **kw))
    errs[w.name] = dict(steps=n, horizon=n, scenario=b, gpu_value=gv,
                        **_errors(e32, o["eta"], d32, w.h_min, g32, o["gauges"]))
    entry(w.name, w, w.cells, n, el, "scenario %d over its %d steps" % (b, n),
          one_thread(w, d32, 40, eta0=w.eta0[b], **kw))
    # 5: the inversion grid over its 2000 steps, 32 gauges
    w = workloads.inversion_1024()
    d32 = depth32(w)
    e32, g32, gv = gpu(w, w.steps)
    p = oracle.params_from(w)
    kw = dict(maxout=w.maxout, gout=w.gout, gauges=w.gauges)
    o, el = _timed_oracle(lambda: oracle.run(p, w.x, w.y, d32, w.eta0, nsteps=w.steps, **kw))
    errs[w.name] = dict(steps=w.steps, horizon=w.steps, gpu_value=gv,
                        **_errors(e32, o["eta"], d32, w.h_min, g32, o["gauges"]))
    entry(w.name, w, w.cells, w.steps, el, "the full %d-step horizon" % w.steps, one_thread(w, d32, 20, **kw))
    host = {"cores": ncores, "cpu": platform_cpu()}
    return errs, cpus, host


def platform_cpu():
    import platform
    name = platform.processor() or platform.machine()
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                name = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return "%s (%s)" % (name, platform.machine())


def run_cuda(args, world, rank, local):
    import torch
    import workloads
    from paper_1410_0753_gb300 import CliffsGrid, _build
    from paper_1410_0753_gb300.ranks import max_over_ranks

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    _build.build()
    w = workloads.shelf_islands(args.nx, args.ny, steps=HORIZON)
    stream = torch.cuda.current_stream()
    g = CliffsGrid.from_workload(w, stream=stream.cuda_stream, gauges=[], nests=[])
    g.set_bathy(w.x, w.y, w.depth, True, w.filter_alpha, w.filter_min_depth)
    eta0 = w.eta0.astype(np.float32)
    g.set_initial(eta0)
    dev_id = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local if world > 1 else 0]
    # the SM clock sampler (every 200 ms) starts before the tile autotuning and the warm-up,
    # so that its samples cover the GPU under load around a timed region of a few ms
    clk = Clocks(dev_id)
    if args.rows_per_warp:                # a fixed tile (to profile the configuration a run chose)
        g.set_rows_per_warp(args.rows_per_warp)
        rows_per_warp = args.rows_per_warp
    else:
        tune = g.autotune(3)              # rows per warp of the fused step, by measurement
        rows_per_warp = min(tune, key=tune.get) if tune else None

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    g.step(args.warmup)
    torch.cuda.synchronize()
    g.kernel_time(-1)
    g.kernel_time(1)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.step(args.steps)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - t0
    clocks = clk.stop()
    ms, launches = g.kernel_time(0)
    g.kernel_time(-1)
    ms_max = max_over_ranks(ms)
    ms_step = ms_max / args.steps
    value = world * w.cells * args.steps / (ms_max / 1e3) / 1e9
    peaks, peak_kind = measured_peaks()
    achieved = BYTES_PER_CELL * w.cells / (ms / args.steps / 1e3) / 1e9
    prof, tnote = profiled("k_step_fused_shelf_8192", rows_per_warp)
    traffic = prof.get("dram_bytes_per_launch") if prof else None

    # end to end through the public API over the workload's horizon: eta0 from pinned host
    # memory in, HORIZON steps, the final surface read into pinned host memory
    e2e = None
    if not args.no_e2e:
        pin_eta = torch.from_numpy(eta0).pin_memory()
        pin_out = torch.empty((w.ny, w.nx), dtype=torch.float32).pin_memory()
        from paper_1410_0753_gb300 import cliffs_read_state
        n_e2e = HORIZON if not args.e2e_steps else args.e2e_steps
        barrier()
        torch.cuda.synchronize()
        t = time.perf_counter()
        g.set_initial(pin_eta.numpy())
        g.step(n_e2e)
        cliffs_read_state(g.h, 0, pin_out.numpy(), None, None)
        torch.cuda.synchronize()
        barrier()
        te = max_over_ranks(time.perf_counter() - t)
        e2e = {"value": world * w.cells * n_e2e / te / 1e9, "unit": UNIT, "steps": n_e2e,
               "h2d_bytes_per_step": pin_eta.numel() * 4 / n_e2e,
               "d2h_bytes_per_step": pin_out.numel() * 4 / n_e2e,
               "note": "set_initial from pinned host eta0, step_n over the %d-step horizon, the final "
                       "eta read into pinned host memory (C ABI, host buffers), wall clock" % n_e2e}
    g.close()

    # the FP64 oracle on host cores (rank 0, one GPU): its speed per workload, and the FP32
    # error against it per workload
    cpu = cpus = errs = host = None
    if rank == 0 and world == 1 and not args.no_cpu:
        errs, cpus, host = oracle_reports(torch, stream)
        c = cpus[HEADLINE]["all_cores"]
        cpu = {"value": c["value"], "unit": UNIT, "cores": c["cores"], "kind": "oracle",
               "sample": c["sample"] + "; FP64 C++ oracle, OpenMP over lines, on " + host["cpu"]}

    forms = None
    if rank == 0 and world == 1 and not args.no_forms:
        forms = measure_forms(torch, stream)

    if rank == 0:
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": bench_config(w, world),
            "rows_per_warp": rows_per_warp,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                         "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                         "kernel": "k_step_fused", "bytes_per_cell": BYTES_PER_CELL,
                         "peak_kind": peak_kind,
                         "issue": issue_roof(prof, w.cells, value / world,
                                             (clocks or {}).get("sm_mhz") or (clocks or {}).get("sm_max_mhz"), sms)},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "wall_ms": 1e3 * wall,
            "clocks": clocks,
            "oracle_error": errs,
            "cpu_baselines": cpus,
            "host": host,
            "forms": forms,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="cuda", choices=["cuda", "reference"])
    ap.add_argument("--nx", type=int, default=8192)
    ap.add_argument("--ny", type=int, default=8192)
    ap.add_argument("--e2e-steps", type=int, default=0, help="steps of the end-to-end run (default: the horizon)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--forms-only", choices=["spherical", "batched", "stress", "adjoint"],
                    help="measure one form only and print it (no headline line)")
    ap.add_argument("--adjoint-steps", type=int, default=None)
    ap.add_argument("--ensemble", default=None, metavar="B,DMIN,DMAX",
                    help="batched form on B scenarios of DMIN..DMAX steps instead of 256 of 500..4000")
    ap.add_argument("--rows-per-warp", type=int, default=0,
                    help="fix the fused step's tile instead of autotuning it (headline and geographic form)")
    args = ap.parse_args()
    world, rank, local = dist_init()
    if args.forms_only:
        import torch
        from paper_1410_0753_gb300 import _build
        _build.build()
        ens = tuple(int(t) for t in args.ensemble.split(",")) if args.ensemble else None
        print(json.dumps({"forms": measure_forms(torch, torch.cuda.current_stream(), args.forms_only,
                                                 args.adjoint_steps, ens, args.rows_per_warp)}), flush=True)
    elif args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_cuda(args, world, rank, local)


if __name__ == "__main__":
    main()
