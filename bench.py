#!/usr/bin/env python
"""Benchmark of the split shallow-water step (Cliffs, arXiv 1410.0753) on GB300.

Workload: the 2048 x 2048 geographic grid at 1 arc-minute (lat 20-54 N) with a 2 m elliptical
source, 64 gauges, max-wave every step and boundary series for 4 enclosed grids every step
(workloads.spherical_coast). One bench step = one model time step: the fused x-sweep +
y-sweep kernel with its max-wave / gauge / enclosed-grid epilogue.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cuda|reference]

Timing: W untimed steps, then K steps, each preceded by a 256 MiB device write that flushes
the 129 MB L2 (the step's inputs, ~100 MB, would otherwise stay resident); every step kernel
is timed with CUDA events on the grid's stream; the K steps are bracketed by a barrier and a
device synchronisation; the maximum over ranks is reported. With N > 1 each rank advances
its own replica of the grid (the path does not shard: replicas only).

With one GPU the line also carries ``forms``: the batched ensemble (256 scenarios of uneven
duration on a shared 512 x 512 bathymetry in one persistent, graph-captured launch), the
8192 x 8192 shelf-and-islands stress grid (pure step and max-wave every step) and the
adjoint (gradient of a 32-gauge misfit over 2000 steps of a 1024 x 1024 grid), the batched
and adjoint forms next to the plain single-scenario forward on the same GPU.

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
BYTES_PER_CELL = 36      # read eta, u, v, d, eta_max, speed_max; write eta, u, v (FP32)


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


def oracle_sample(w, seconds, depth=None):
    """Time the FP64 oracle on the first steps of the workload (all host cores)."""
    import oracle
    threads = oracle.threads(os.cpu_count() or 1)
    d = depth if depth is not None else oracle.depth_filter(w.depth, w.filter_alpha, w.filter_min_depth)[0]
    p = oracle.params_from(w)
    out = dict(eta=w.eta0, u=None, v=None)
    kw = dict(maxout=w.maxout, gout=w.gout, gauges=w.gauges, bndout=w.bndout, nests=w.nests)
    t = time.perf_counter()
    r = oracle.run(p, w.x, w.y, d, w.eta0, nsteps=1, **kw)
    t1 = time.perf_counter() - t
    m = int(max(1, min(400, round(seconds / max(t1, 1e-3)))))
    t = time.perf_counter()
    r = oracle.run(p, w.x, w.y, d, w.eta0, nsteps=m, **kw)
    el = time.perf_counter() - t
    return dict(value=w.cells * m / el / 1e9, steps=m, seconds=el, threads=threads, result=r,
                depth=d)


def run_reference(args, world, rank):
    """The FP64 oracle as it stands, on the host cores, for the same workload and metric. The
    W warm-up steps and the K timed steps each run as one oracle call (its outputs recorded
    every step as in the CUDA arm). Each step covers the full grid when K + W steps fit in
    about 150 s at the oracle's speed on the box (~0.12 Gcell/s on 16 cores); otherwise a band
    of rows around the source (gauges inside the band, no enclosed grids), so that the run
    stays within a few minutes."""
    if rank != 0:
        return
    import oracle
    import workloads
    w = workloads.spherical_coast(args.nx, args.ny, steps=3600)
    threads = oracle.threads(os.cpu_count() or 1)
    d = oracle.depth_filter(w.depth, w.filter_alpha, w.filter_min_depth)[0]
    budget_cells = 0.12e9 * 150.0 / max(1, args.steps + args.warmup)
    rows = int(min(w.ny, max(64, budget_cells // w.nx)))
    if rows < w.ny:
        j0 = max(0, min(w.ny - rows, w.ny // 2 - rows // 2))
        sl = slice(j0, j0 + rows)
        gauges = np.array([(ix, iy - j0) for ix, iy in w.gauges if j0 <= iy < j0 + rows], np.int32)
        w = workloads.Workload(w.name + "_band%d" % rows, w.nx, rows, w.coords, w.x, w.y[sl], w.depth[sl],
                               w.eta0[sl], w.dt, w.steps, h_min=w.h_min, manning_n2=w.manning_n2,
                               maxout=w.maxout, gout=w.gout, bndout=w.bndout, gauges=gauges)
        d = d[sl]
        sample = "a band of %d of %d rows around the source, gauges inside it, no enclosed grids" % (rows, args.ny)
    else:
        sample = "the full grid with all outputs"
    p = oracle.params_from(w)
    kw = dict(maxout=w.maxout, gout=w.gout, gauges=w.gauges if len(w.gauges) else None,
              bndout=w.bndout, nests=w.nests or None)
    r = oracle.run(p, w.x, w.y, d, w.eta0, nsteps=args.warmup, **kw)
    t = time.perf_counter()
    oracle.run(p, w.x, w.y, d, r["eta"], r["u"], r["v"], nsteps=args.steps, step0=args.warmup, **kw)
    el = time.perf_counter() - t
    cells = w.nx * w.ny
    val = cells * args.steps / el / 1e9
    line = {"metric": METRIC, "value": val, "unit": UNIT, "impl": "reference",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "spherical_coast_%dx%d" % (args.nx, args.ny), "cells_per_step": cells,
                       "steps_horizon": 3600, "sample": sample},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": "%d consecutive steps of %s (FP64 C++ oracle, OpenMP over lines)"
                                       % (args.steps, sample)},
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


def measure_forms(torch, stream, only=None, adjoint_steps=None, ensemble=None):
    """The batched ensemble (256 scenarios of uneven duration on one 512 x 512 bathymetry, one
    persistent graph-captured launch) and the adjoint (1024 x 1024, 2000 steps, checkpoint
    every 100), each reported against the plain single-scenario forward on this GPU."""
    import workloads
    from paper_1410_0753_gb300 import CliffsGrid
    out = {}
    s = stream.cuda_stream
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
    # the HBM stress grid (8192 x 8192, shorelines around 10 islands), as a pure step and with
    # max-wave every step; its 1.9 GB working set is far larger than L2
    s = stream.cuda_stream
    w = workloads.shelf_islands()
    peaks, _ = measured_peaks()
    out = {"workload": w.name, "cells": w.cells}
    for tag, maxout, bpc in (("pure_step", 10 ** 9, 28), ("maxwave_every_step", 1, 36)):
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
    w = workloads.spherical_coast(args.nx, args.ny, steps=3600)
    stream = torch.cuda.current_stream()
    g = CliffsGrid.from_workload(w, stream=stream.cuda_stream)
    g.set_bathy(w.x, w.y, w.depth, True, w.filter_alpha, w.filter_min_depth)
    eta0 = w.eta0.astype(np.float32)
    g.set_initial(eta0)
    if args.rows_per_warp:                # a fixed tile (to profile the configuration a run chose)
        g.set_rows_per_warp(args.rows_per_warp)
        rows_per_warp = args.rows_per_warp
    else:
        tune = g.autotune(3)              # rows per warp of the fused step, by measurement
        rows_per_warp = min(tune, key=tune.get) if tune else None
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for i in range(args.warmup):
        flush.fill_(i & 0xFF)
        g.step(1)
    torch.cuda.synchronize()
    g.kernel_time(-1)
    g.kernel_time(1)
    dev_id = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local if world > 1 else 0]
    barrier()
    torch.cuda.synchronize()
    clk = Clocks(dev_id)
    t0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_((i + 1) & 0xFF)
        g.step(1)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - t0
    clocks = clk.stop()
    ms, launches = g.kernel_time(0)
    ms_max = max_over_ranks(ms)
    ms_step = ms_max / args.steps
    value = world * w.cells * args.steps / (ms_max / 1e3) / 1e9
    peaks, peak_kind = measured_peaks()
    achieved = BYTES_PER_CELL * w.cells / (ms / args.steps / 1e3) / 1e9
    prof, tnote = profiled("k_step_fused_spherical_2048", rows_per_warp)
    traffic = prof.get("dram_bytes_per_launch") if prof else None

    # end to end through the public API: pinned host inputs in, host outputs out
    e2e = None
    if not args.no_e2e:
        pin_eta = torch.from_numpy(eta0).pin_memory()
        nrec = args.steps + 1
        pin_g = torch.empty((nrec, g.n_gauges, 3), dtype=torch.float32).pin_memory()
        pin_em = torch.empty((w.ny, w.nx), dtype=torch.float32).pin_memory()
        pin_sm = torch.empty((w.ny, w.nx), dtype=torch.float32).pin_memory()
        pin_b = [[torch.empty((nrec, 3, (n.ny if e < 2 else n.nx)), dtype=torch.float64).pin_memory()
                  for e in range(4)] for n in w.nests]
        from paper_1410_0753_gb300 import (cliffs_read_boundary, cliffs_read_gauges,
                                           cliffs_read_maxwave)
        barrier()
        torch.cuda.synchronize()
        t = time.perf_counter()
        g.set_initial(pin_eta.numpy())
        g.step(args.steps)
        cliffs_read_gauges(g.h, 0, pin_g.numpy())
        cliffs_read_maxwave(g.h, 0, pin_em.numpy(), pin_sm.numpy())
        for m in range(len(w.nests)):
            for e in range(4):
                cliffs_read_boundary(g.h, m, e, pin_b[m][e].numpy())
        torch.cuda.synchronize()
        barrier()
        te = max_over_ranks(time.perf_counter() - t)
        d2h = pin_g.numel() * 4 + 2 * pin_em.numel() * 4 + sum(b.numel() * 8 for bb in pin_b for b in bb)
        e2e = {"value": world * w.cells * args.steps / te / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": pin_eta.numel() * 4 / args.steps,
               "d2h_bytes_per_step": d2h / args.steps,
               "note": "set_initial from pinned host eta0, step_n(K), read gauges, max-wave and "
                       "16 boundary series into pinned host buffers; no L2 flush"}

    # the FP64 oracle on host cores (rank 0, one GPU), and the FP32 error on that horizon
    cpu = None
    oracle_error = None
    if rank == 0 and world == 1 and not args.no_cpu:
        s = oracle_sample(w, args.cpu_seconds)
        cpu = {"value": s["value"], "unit": UNIT, "cores": s["threads"], "kind": "oracle",
               "sample": "first %d steps of %s, all outputs recorded (%.1f s, FP64 C++ oracle, "
                         "OpenMP over lines)" % (s["steps"], w.name, s["seconds"])}
        gv = CliffsGrid.from_workload(w, stream=stream.cuda_stream)
        gv.set_bathy(w.x, w.y, w.depth, True, w.filter_alpha, w.filter_min_depth)
        gv.set_initial(eta0)
        gv.step(s["steps"])
        g32 = gv.gauges()[:, :, 0].astype(np.float64)
        g64 = s["result"]["gauges"][:, :, 0]
        rel = [np.abs(g32[:, k] - g64[:, k]).max() / np.abs(g64[:, k]).max()
               for k in range(g64.shape[1]) if np.abs(g64[:, k]).max() >= 1e-3]
        e32, _, _ = gv.state()
        e64 = s["result"]["eta"]
        oracle_error = {"steps": s["steps"], "gauge_rel_max": float(max(rel)) if rel else None,
                        "gauges_compared": len(rel),
                        "eta_max_abs": float(np.abs(e32 - e64).max()),
                        "eta_scale": float(np.abs(e64).max())}
        gv.close()

    forms = None
    if rank == 0 and world == 1 and not args.no_forms:
        forms = measure_forms(torch, stream)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": w.name, "cells": w.cells, "coords": "geographic 1 arc-min",
                       "gauges": int(g.n_gauges), "nests": len(w.nests), "maxout": w.maxout,
                       "gout": w.gout, "bndout": w.bndout, "steps_horizon": 3600,
                       "l2": "flushed before every timed step (256 MiB device write)",
                       "rows_per_warp": rows_per_warp,
                       "parallelism": "replicas" if world > 1 else "single"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                         "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                         "kernel": "k_step_fused", "bytes_per_cell": BYTES_PER_CELL,
                         "peak_kind": peak_kind,
                         "issue": issue_roof(prof, w.cells, value / world,
                                             (clocks or {}).get("sm_mhz") or (clocks or {}).get("sm_max_mhz"),
                                             torch.cuda.get_device_properties(local).multi_processor_count)},
            "cpu_baseline": cpu,
            "oracle_error": oracle_error,
            "forms": forms,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "wall_ms": 1e3 * wall,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    g.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3600)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="cuda", choices=["cuda", "reference"])
    ap.add_argument("--nx", type=int, default=2048)
    ap.add_argument("--ny", type=int, default=2048)
    ap.add_argument("--cpu-seconds", type=float, default=25.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--forms-only", choices=["batched", "stress", "adjoint"],
                    help="measure one form only and print it (no headline line)")
    ap.add_argument("--adjoint-steps", type=int, default=None)
    ap.add_argument("--ensemble", default=None, metavar="B,DMIN,DMAX",
                    help="batched form on B scenarios of DMIN..DMAX steps instead of 256 of 500..4000")
    ap.add_argument("--rows-per-warp", type=int, default=0,
                    help="fix the fused step's tile instead of autotuning it")
    args = ap.parse_args()
    world, rank, local = dist_init()
    if args.forms_only:
        import torch
        from paper_1410_0753_gb300 import _build
        _build.build()
        ens = tuple(int(t) for t in args.ensemble.split(",")) if args.ensemble else None
        print(json.dumps({"forms": measure_forms(torch, torch.cuda.current_stream(), args.forms_only,
                                                 args.adjoint_steps, ens)}), flush=True)
    elif args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_cuda(args, world, rank, local)


if __name__ == "__main__":
    main()
