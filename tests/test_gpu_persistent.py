"""The batched persistent run (cliffs_run_persistent) on the GPU.

One cooperative, graph-captured launch runs many steps of every scenario of a batch; warps
take (scenario, tile) work items of the scenarios still running at each step and meet at a
grid barrier between steps. Each output node is computed by the same arithmetic as in the
one-launch-per-step path, so the results must agree bit for bit with it, and through it with
the oracle, which the last test checks directly for one scenario.
"""
import numpy as np
import pytest

import oracle
import workloads
from paper_1410_0753_gb300 import CliffsError, CliffsGrid, ERR_ARG, ERR_TIMEOUT, cliffs_inject_wait_expiry
from tests import parity as P

pytestmark = pytest.mark.gpu


def _start(w, **kw):
    g = CliffsGrid.from_workload(w, **kw)
    g.set_bathy(w.x, w.y, w.depth, True, w.filter_alpha, w.filter_min_depth)
    g.set_initial(w.eta0.astype(np.float32))
    if w.durations is not None:
        g.set_durations(w.durations)
    return g


def _outputs(g, b, nests=0):
    out = list(g.state(b)) + list(g.maxwave(b))
    if g.n_gauges:
        out.append(g.gauges(b))
    for m in range(nests):
        out += [g.boundary(m, e) for e in range(4)]
    return out


def _same(a, b):
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert x.shape == y.shape
        assert np.array_equal(x, y, equal_nan=True)


def test_persistent_batch_with_uneven_durations_matches_per_step_launches():
    """Scenarios of unequal durations (some end before the first chunk does, one never
    starts) in chunks of steps that straddle the ends; state, maxima and gauge records of
    every scenario equal the per-step path's bit for bit."""
    w = workloads.ensemble_512(batch=9, nx=150, ny=112, dmin=10, dmax=90)
    w.durations[4] = 0
    w.maxout = 3
    w.gout = 2
    total = int(w.durations.max()) + 4
    ref = _start(w)
    ref.step(total)
    run = _start(w)
    done = 0
    for chunk in (7, 1, 25, total):
        n = min(chunk, total - done)
        run.step(n, persistent=True)
        done += n
    assert run.steps_done == ref.steps_done == total
    for b in range(w.batch):
        _same(_outputs(run, b), _outputs(ref, b))
    ref.close()
    run.close()


def test_persistent_spherical_with_nests_and_mixed_calls():
    """Spherical grid with enclosed grids: persistent chunks interleaved with per-step calls
    (the graph is replayed, then re-captured after the record buffers grow) give the same
    boundary series, gauges, maxima and state as per-step launches alone."""
    w = workloads.spherical_coast(260, 220, steps=90)
    ref = _start(w)
    ref.step(w.steps)
    run = _start(w)
    for n, pers in ((10, True), (5, False), (30, True), (1, True), (44, True)):
        run.step(n, persistent=pers)
    assert run.steps_done == w.steps
    _same(_outputs(run, 0, len(w.nests)), _outputs(ref, 0, len(w.nests)))
    ref.close()
    run.close()


def test_persistent_tuned_tile_shape_and_reinitialisation():
    """A tuned tile shape (rows per warp) re-captures the graph and changes nothing; a new
    initial state restarts the step count for the replayed graph."""
    w = workloads.ensemble_512(batch=4, nx=120, ny=100, dmin=15, dmax=60)
    ref = _start(w)
    ref.step(int(w.durations.max()))
    run = _start(w)
    run.step(20, persistent=True)
    run.autotune(1)                           # keeps the fastest shape
    run.set_initial(w.eta0.astype(np.float32))
    run.step(int(w.durations.max()), persistent=True)
    for b in range(w.batch):
        _same(_outputs(run, b), _outputs(ref, b))
    run.close()
    ref.close()


def test_persistent_scenario_against_oracle():
    """One scenario of a persistent batched run against the FP64 oracle directly."""
    w = workloads.ensemble_512(batch=3, nx=96, ny=80, dmin=30, dmax=70)
    g = _start(w)
    g.step(int(w.durations.max()), persistent=True)
    b = int(np.argmin(w.durations))
    d64 = P.oracle_depth(w)
    o = oracle.run(oracle.params_from(w), w.x, w.y, P.f32(d64), w.eta0[b],
                   nsteps=int(w.durations[b]), gout=w.gout, gauges=w.gauges)
    got = g.gauges(b)
    assert got.shape[0] == o["gauges"].shape[0]
    rel, absol = P.gauge_errors(got[:, :, 0], o["gauges"][:, :, 0])
    P.report("persistent_scenario", gauge_rel=rel.max(initial=0.0), gauge_abs=absol.max(initial=0.0))
    assert rel.max(initial=0.0) < P.GAUGE_RTOL
    assert absol.max(initial=0.0) < P.GAUGE_ATOL_SMALL
    g.close()


def test_persistent_wait_expiry_and_errors():
    """Injected ring-wait expiry inside the persistent kernel: the run returns
    CLIFFS_ERR_TIMEOUT, every block leaves through the bounded grid barrier, and the grid
    keeps working. A 1D grid has no persistent path."""
    w = workloads.ensemble_512(batch=3, nx=100, ny=90, dmin=10, dmax=30)
    g = _start(w)
    cliffs_inject_wait_expiry(g.h, 2_000_000)
    with pytest.raises(CliffsError) as e:
        g.step(10, persistent=True)
    assert e.value.code == ERR_TIMEOUT
    g.set_initial(w.eta0.astype(np.float32))
    g.step(int(w.durations.max()), persistent=True)
    ref = _start(w)
    ref.step(int(w.durations.max()))
    for b in range(w.batch):
        _same(_outputs(g, b), _outputs(ref, b))
    g.close()
    ref.close()
    line = CliffsGrid(64, 1, 1.0)
    line.set_bathy(np.arange(64) * 50.0, np.zeros(1), np.full((1, 64), 10.0), False)
    line.set_initial(np.zeros((1, 64), np.float32))
    with pytest.raises(CliffsError) as e:
        line.step(3, persistent=True)
    assert e.value.code == ERR_ARG
    line.close()
