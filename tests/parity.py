"""Helpers for the GPU-vs-oracle parity tests: run the same seeded workload through the CUDA
library (C ABI) and through the FP64 oracle, and compare outputs the way the error report is
defined: per gauge max_t|eta32 - eta64| / max_t|eta64| (absolute when the oracle's trace stays
below 1e-3 m), and wet/dry masks with near-round-off cells counted separately."""
import json
import os

import numpy as np

import oracle
from paper_1410_0753_gb300 import CliffsGrid

GAUGE_RTOL = 1e-4          # relative, on gauge traces over the run
GAUGE_ATOL_SMALL = 1e-7    # absolute, for gauges whose trace stays below 1e-3 m
NEAR = 1e-5                # near-round-off band for wet/dry decisions, times max(1, |d|)


def report(name, **vals):
    """Append measured parity numbers to $PARITY_REPORT (JSON lines) when set."""
    path = os.environ.get("PARITY_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(dict(test=name, **{k: (float(v) if np.ndim(v) == 0 else v)
                                                  for k, v in vals.items()})) + "\n")


def oracle_depth(w):
    d, passes = oracle.depth_filter(w.depth, w.filter_alpha, w.filter_min_depth)
    assert passes > 0
    return d


def f32(a):
    return np.asarray(a, np.float64).astype(np.float32).astype(np.float64)


def gpu_run(w, nsteps, scenario=None, grid=None, **kw):
    g = grid or CliffsGrid.from_workload(w, **kw)
    g.set_bathy(w.x, w.y, w.depth, True, w.filter_alpha, w.filter_min_depth)
    eta0 = w.eta0.astype(np.float32)
    g.set_initial(eta0, None if w.u0 is None else w.u0.astype(np.float32),
                  None if w.v0 is None else w.v0.astype(np.float32))
    if w.durations is not None:
        g.set_durations(w.durations)
    g.step(nsteps)
    out = dict(grid=g)
    out["eta"], out["u"], out["v"] = g.state(0 if scenario is None else scenario)
    out["gauges"] = g.gauges(0 if scenario is None else scenario) if g.n_gauges else None
    out["eta_max"], out["speed_max"] = g.maxwave(0 if scenario is None else scenario)
    out["depth"] = g.depth()
    if w.nests:
        out["boundary"] = [[g.boundary(m, e) for e in range(4)] for m in range(len(w.nests))]
    return out


def oracle_run(w, nsteps, depth, scenario=0, form=0):
    eta0 = w.eta0 if w.eta0.ndim == 2 else w.eta0[scenario]
    p = oracle.params_from(w, form=form)
    return oracle.run(p, w.x, w.y, depth, eta0, w.u0, w.v0, nsteps=nsteps, maxout=w.maxout,
                      gout=w.gout, gauges=w.gauges if len(w.gauges) else None, bndout=w.bndout,
                      nests=w.nests or None)


def gauge_errors(g32, g64):
    """Per-gauge error of eta: relative to the oracle's max |eta|, or absolute for tiny traces."""
    g32 = np.asarray(g32, np.float64)
    rel, absol = [], []
    for k in range(g64.shape[1]):
        m = np.abs(g64[:, k]).max()
        e = np.abs(g32[:, k] - g64[:, k]).max()
        (rel if m >= 1e-3 else absol).append(e / m if m >= 1e-3 else e)
    return np.array(rel), np.array(absol)


def wet_masks(eta32, eta64, d32, d64, hmin):
    wet32 = (eta32.astype(np.float32) + d32.astype(np.float32)) >= np.float32(hmin)
    h64 = eta64 + d64
    wet64 = h64 >= hmin
    near = np.abs(h64 - hmin) < NEAR * np.maximum(1.0, np.abs(d64))
    return wet32, wet64, near
