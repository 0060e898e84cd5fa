"""FP32 against the FP64 oracle over each workload's stated horizon (the precision report).

Configurations and horizons: the 1024^2 inversion grid over its 2000 steps (32 gauges,
friction, a shore), scenarios of the 256 x 512^2 ensemble over their full durations (up to
about 4000 steps), and the 2048^2 geographic grid over its 3600 steps. The 200^2 beach over
its 1000 steps is in test_gpu_parity.py and the 8192^2 grid is checked on windows there.

Tolerances as in test_gpu_parity.py: gauge traces within 1e-4 of the oracle's max |eta| per
gauge (1e-7 m absolute for traces below 1e-3 m), wet masks equal.

The GPU and the oracle are advanced together, in chunks, and their wet/dry masks compared
after every chunk. While the masks agree, both take the same branch of every threshold of
the method (steps (a) and (b) of the inundation algorithm), and the gauge tolerance holds.
Over long run-up a decision can land within an FP32-sized distance of its threshold (a
flooding margin eta_j + d_i - h_min or a wet margin h - h_min of ~1e-6): FP32 and FP64 then
take it differently, and the two runs continue from states that differ by a wetted or a
dried node. Such a run is checked in three parts:
  1. up to the step before the first mask difference, the gauge tolerance holds;
  2. at that step the FP64 oracle, started from the GPU's own state one step earlier, takes
     the GPU's decisions (the two sides apply the same method to states an FP32-sized
     deviation apart), except at nodes it leaves within the near-round-off band of the wet
     threshold, |h - h_min| < 1e-5 max(1, |d|), where the step's own FP32 arithmetic decides
     (the band in which the masks of the parity tests may differ);
  3. over the rest of the horizon the GPU's gauge deviation is what the FP64 scheme itself
     produces from the GPU's state before the flip (the oracle continued from that state
     against the oracle's own run): within three times that deviation plus the tolerance.
"""
import dataclasses

import numpy as np
import pytest

import oracle
import workloads
from paper_1410_0753_gb300 import CliffsGrid, cliffs_read_state
from tests import parity as P

pytestmark = pytest.mark.gpu

CHUNK = 10


def _eta(g):
    e = np.empty((g.ny, g.nx), np.float32)
    cliffs_read_state(g.h, 0, e, None, None)
    return e


def _wet(eta, d32, hmin, fp32):
    if fp32:
        return (eta.astype(np.float32) + d32.astype(np.float32)) >= np.float32(hmin)
    return (eta + d32) >= hmin


def _gauge_rel(g32, g64):
    rel, absol = P.gauge_errors(g32, g64)
    return float(rel.max(initial=0.0)), float(absol.max(initial=0.0))


def horizon(name, w, eta0, n, make_grid):
    """Co-step a GPU grid (make_grid(): configured, bathymetry set) and the oracle over n
    steps from eta0; returns the report dict after the assertions of the module docstring."""
    assert w.gout == 1                     # record r is the state after r steps
    d32 = P.f32(P.oracle_depth(w))
    p = oracle.params_from(w)
    kw = dict(gout=w.gout, gauges=w.gauges)
    g = make_grid()
    e0 = eta0.astype(np.float32)
    g.set_initial(e0)
    o = dict(eta=e0.astype(np.float64), u=np.zeros_like(d32), v=np.zeros_like(d32))
    recs, k, first = [], 0, None
    start = None                           # (k, oracle state) at the start of the first mismatching chunk
    while k < n:
        m = min(CHUNK, n - k)
        prev = (k, o)
        g.step(m)
        r = oracle.run(p, w.x, w.y, d32, o["eta"], o["u"], o["v"], nsteps=m, step0=k, record_initial=k == 0, **kw)
        recs.append(r["gauges"][:, :, 0])
        o = dict(eta=r["eta"], u=r["u"], v=r["v"])
        k += m
        if first is None and np.any(_wet(_eta(g), d32, w.h_min, True) != _wet(o["eta"], d32, w.h_min, False)):
            first, start = k, prev
    g64 = np.concatenate(recs)
    g32 = g.gauges()[:, :, 0].astype(np.float64)
    assert g32.shape == g64.shape
    e32 = _eta(g)
    rel, absol = _gauge_rel(g32, g64)
    out = dict(steps=n, gauge_rel_max=rel, gauge_abs_max=absol,
               eta_abs_max=float(np.abs(e32 - o["eta"])[_wet(o["eta"], d32, w.h_min, False)].max(initial=0.0)))
    if first is None:
        out.update(flip_step=-1)
        P.report(name, **out)
        assert rel <= P.GAUGE_RTOL and absol <= P.GAUGE_ATOL_SMALL, out
        g.close()
        return out
    # replay the first mismatching chunk step by step on both sides (the GPU run repeats
    # bit for bit from the initial state)
    k0, ost = start
    g.set_initial(e0)
    g.step(k0)
    s = k0
    while True:
        gprev = g.state()
        oprev = dict(ost)
        g.step(1)
        r = oracle.run(p, w.x, w.y, d32, ost["eta"], ost["u"], ost["v"], nsteps=1, step0=s, record_initial=False)
        ost = dict(eta=r["eta"], u=r["u"], v=r["v"])
        s += 1
        m32 = _wet(_eta(g), d32, w.h_min, True)
        if np.any(m32 != _wet(ost["eta"], d32, w.h_min, False)) or s >= first:
            break
    assert s == first or np.any(m32 != _wet(ost["eta"], d32, w.h_min, False))
    m64 = _wet(ost["eta"], d32, w.h_min, False)
    flips = int((m32 != m64).sum())
    # 2. the oracle from the GPU's state one step before the flip takes the GPU's decisions,
    # except at nodes whose wet margin |h - h_min| it leaves within the near-round-off band
    gs = [a.astype(np.float64) for a in gprev]
    r = oracle.run(p, w.x, w.y, d32, gs[0], gs[1], gs[2], nsteps=1, step0=s - 1, record_initial=False)
    mo = _wet(r["eta"], d32, w.h_min, False)
    diff = mo != m32
    margin = np.abs(r["eta"] + d32 - w.h_min)
    band = P.NEAR * np.maximum(1.0, np.abs(d32))
    same_decisions = bool(not diff.any())
    near_only = bool(np.all(margin[diff] < band[diff]))
    jy, jx = np.nonzero(m32 != m64)
    at = [(int(x), int(y), float(d32[y, x]), float(gprev[0][y, x]), float(_eta(g)[y, x]), float(margin[y, x]))
          for y, x in zip(jy, jx)][:4]
    state_diff = max(float(np.abs(gs[i] - oprev[key]).max()) for i, key in enumerate(("eta", "u", "v")))
    pre = s - 1                                     # records 0 .. s-1 precede the flip
    rel_pre, abs_pre = _gauge_rel(g32[: pre + 1], g64[: pre + 1])
    # 3. the FP64 scheme continued from the GPU's state before the flip, against its own run
    c = oracle.run(p, w.x, w.y, d32, gs[0], gs[1], gs[2], nsteps=n - (s - 1), step0=s - 1, record_initial=True, **kw)
    g64c = np.concatenate([g64[: s - 1], c["gauges"][:, :, 0]])
    rel_fp64, _ = _gauge_rel(g64c, g64)
    out.update(flip_step=s, flipped_nodes=flips, flipped_at=at, state_diff_before_flip=state_diff,
               gauge_rel_before_flip=rel_pre, oracle_from_gpu_state_same_decisions=int(same_decisions),
               differing_decisions_near_round_off=int(near_only), fp64_deviation_from_gpu_state=rel_fp64)
    P.report(name, **out)
    g.close()
    assert rel_pre <= P.GAUGE_RTOL and abs_pre <= P.GAUGE_ATOL_SMALL, out
    assert same_decisions or near_only, out
    assert rel <= 3.0 * rel_fp64 + P.GAUGE_RTOL and absol <= P.GAUGE_ATOL_SMALL, out
    return out


def _grid(w, **kw):
    def make():
        g = CliffsGrid.from_workload(w, **kw)
        g.set_bathy(w.x, w.y, w.depth, True, w.filter_alpha, w.filter_min_depth)
        return g
    return make


def test_inversion_1024_full_horizon():
    w = workloads.inversion_1024()
    horizon("horizon_inversion_1024", w, w.eta0, w.steps, _grid(w))


def test_ensemble_scenarios_full_durations():
    """Three scenarios of the ensemble (the longest, the shortest and the median duration):
    all 256 run to their own durations in one persistent launch; each pick equals its own
    single-scenario run bit for bit, and that run is co-stepped with the oracle."""
    w = workloads.ensemble_512()
    order = np.argsort(w.durations)
    picks = [int(order[-1]), int(order[0]), int(order[len(order) // 2])]
    g = CliffsGrid.from_workload(w)
    g.set_bathy(w.x, w.y, w.depth, True, w.filter_alpha, w.filter_min_depth)
    g.set_initial(w.eta0.astype(np.float32))
    g.set_durations(w.durations)
    g.step(int(w.durations.max()), persistent=True)
    batched = {b: (g.state(b)[0], g.gauges(b)[: int(w.durations[b]) // w.gout + 1]) for b in picks}
    g.close()
    for b in picks:
        n = int(w.durations[b])
        w1 = dataclasses.replace(w, eta0=w.eta0[b], steps=n, durations=None)
        make = _grid(w1, batch=1)
        single = make()
        single.set_initial(w.eta0[b].astype(np.float32))
        single.step(n)
        assert np.array_equal(single.state()[0], batched[b][0])
        assert np.array_equal(single.gauges(), batched[b][1])
        single.close()
        horizon("horizon_ensemble_scenario_%d" % b, w1, w.eta0[b], n, make)


def test_spherical_coast_2048_full_horizon():
    w = workloads.spherical_coast()
    horizon("horizon_spherical_2048", w, w.eta0, w.steps, _grid(w, nests=[], maxout=w.steps + 1))
