"""Boundary input and the nesting chain on the GPU (section "Running Options": boundary
series for enclosed grids, boundary input, parameter-file fields 5 and 13).

The reading of how input enters the scheme (edge nodes take the input at the current model
time before each step, S and N owning the corners) is the oracle's; here the GPU is checked
against the oracle's forced run, the parent -> child chain is checked bit for bit on the GPU
in open water, the clock (cuke start, stop at the end of the records) is checked, and the
adjoint under input is checked by the dot-product identity against the oracle's forced
tangent model (the imposed edge values carry no sensitivity to the initial state).
"""
import numpy as np
import pytest

import oracle
import workloads
from paper_1410_0753_gb300 import CliffsError, CliffsGrid, ERR_ARG, ERR_STATE
from tests import parity as P

pytestmark = pytest.mark.gpu


def _open_water(nx=150, ny=130):
    x = 100.0 * np.arange(nx)
    y = 100.0 * np.arange(ny)
    X, Y = np.meshgrid(x, y)
    d = 40.0 + 8.0 * np.sin(X / 900.0) * np.cos(Y / 700.0)
    eta0 = 0.8 * np.exp(-((X - 6000.0) ** 2 + (Y - 5000.0) ** 2) / (2 * 700.0 ** 2))
    return x, y, P.f32(d), P.f32(eta0)


def test_nesting_chain_is_bit_exact_on_the_gpu():
    """Parent on the GPU records the series of an enclosed grid on its own nodes; the child,
    driven by them, equals the parent inside its edges bit for bit (open water)."""
    from workloads import Nest
    x, y, d, eta0 = _open_water()
    dt, steps = 1.5, 60
    i0, j0, cx, cy = 41, 33, 70, 64
    nest = Nest(x[i0], y[j0], 100.0, 100.0, cx, cy)
    par = CliffsGrid(len(x), len(y), dt, manning_n2=6.25e-4, nests=[nest], bndout=1)
    par.set_bathy(x, y, d, False)
    par.set_initial(eta0.astype(np.float32))
    par.step(steps)
    series = [par.boundary(0, e) for e in range(4)]
    pe, pu, pv = par.state()
    par.close()
    sub = (slice(j0, j0 + cy), slice(i0, i0 + cx))
    ch = CliffsGrid(cx, cy, dt, manning_n2=6.25e-4)
    ch.set_bathy(x[i0:i0 + cx], y[j0:j0 + cy], d[sub], False)
    ch.set_initial(eta0[sub].astype(np.float32))
    times = dt * np.arange(steps + 1)
    for e in range(4):
        ch.set_boundary_input(e, times, series[e])
    assert ch.set_boundary_clock() == 0.0
    ch.step(steps)
    ce, cu, cv = ch.state()
    for a, b in ((ce, pe), (cu, pu), (cv, pv)):
        assert np.array_equal(a[1:-1, 1:-1], b[sub][1:-1, 1:-1])
    ch.close()


@pytest.mark.parametrize("alternate", [0, 1])
def test_forced_run_against_the_oracle_on_a_beach(alternate):
    """A child straddling the shoreline of a beach, driven by the oracle parent's series:
    the GPU's forced run against the oracle's forced run (both sweep orders)."""
    from workloads import Nest
    w = workloads.beach_200(200, 120, steps=400)
    d64 = P.f32(P.oracle_depth(w))
    i0, j0, cx, cy = 110, 30, 90, 64                       # covers the shoreline (column 182)
    nest = Nest(float(w.x[i0]), float(w.y[j0]), 100.0, 100.0, cx, cy)
    p = oracle.params_from(w)
    par = oracle.run(p, w.x, w.y, d64, w.eta0, nsteps=w.steps, bndout=1, nests=[nest])
    times = w.dt * np.arange(w.steps + 1)
    series = {e: (times, par["boundary"][0][e]) for e in range(4)}
    sub = (slice(j0, j0 + cy), slice(i0, i0 + cx))
    gauges = np.array([(0, 32), (10, 32), (40, 32), (70, 32), (85, 20)], np.int32)   # one on the W input edge
    pc = oracle.params(cx, cy, w.dt, h_min=w.h_min, manning_n2=w.manning_n2, alternate=alternate)
    o = oracle.run_forced(pc, w.x[i0:i0 + cx], w.y[j0:j0 + cy], d64[sub], w.eta0[sub], series,
                          nsteps=w.steps, gout=1, gauges=gauges)
    g = CliffsGrid(cx, cy, w.dt, h_min=w.h_min, manning_n2=w.manning_n2, gauges=[tuple(q) for q in gauges],
                   alternate=alternate)
    g.set_bathy(w.x[i0:i0 + cx], w.y[j0:j0 + cy], d64[sub], False)
    g.set_initial(w.eta0[sub].astype(np.float32))
    for e in range(4):
        g.set_boundary_input(e, times, series[e][1])
    g.step(w.steps)
    rel, absol = P.gauge_errors(g.gauges()[:, :, 0], o["gauges"][:, :, 0])
    P.report("forced_beach_child_alt%d" % alternate, gauge_rel_max=rel.max(initial=0.0),
             gauge_abs_max=absol.max(initial=0.0))
    assert rel.max(initial=0.0) <= P.GAUGE_RTOL and absol.max(initial=0.0) <= P.GAUGE_ATOL_SMALL
    e32 = g.state()[0]
    wet32, wet64, near = P.wet_masks(e32, o["eta"], d64[sub], d64[sub], w.h_min)
    assert np.array_equal(wet32 & ~near, wet64 & ~near)
    assert np.abs(e32 - o["eta"])[wet64].max() <= 1e-4 * np.abs(w.eta0).max()
    g.close()


def test_boundary_clock_cuke_and_stop_at_end():
    """Start at the first record whose |eta| exceeds cuke; with stop_at_end the run ends at
    the last record; without it the last record holds."""
    x = 50.0 * np.arange(120)
    d = np.full((1, 120), 10.0)
    dt = 1.0
    times = np.arange(0.0, 41.0, 2.0)                       # 21 records, 40 s
    eta_w = np.where(times >= 10.0, 0.05 * np.sin(0.2 * (times - 10.0)) + 0.002, 0.0)
    vals = np.zeros((len(times), 3, 1))
    vals[:, 2, 0] = eta_w
    g = CliffsGrid(120, 1, dt, manning_n2=0.0)
    g.set_bathy(x, np.zeros(1), d, False)
    g.set_initial(np.zeros((1, 120), np.float32))
    with pytest.raises(CliffsError) as e:
        g.set_boundary_clock(0.001)
    assert e.value.code == ERR_STATE
    with pytest.raises(CliffsError) as e:
        g.set_boundary_input(2, times, np.zeros((len(times), 3, 120)))    # S runs along the line
    assert e.value.code == ERR_ARG
    g.set_boundary_input(0, times, vals)
    assert g.set_boundary_clock(0.001, stop_at_end=True) == 10.0
    g.step(1000)
    assert g.steps_done == 30                                # 10 s .. 40 s at dt = 1 s
    e1 = g.state()[0]
    assert np.abs(e1).max() > 0.01                           # the wave came in from the west
    # the same input from t = 0 without stopping: runs all steps, the last record holds
    g.set_initial(np.zeros((1, 120), np.float32))
    assert g.set_boundary_clock(0.0, stop_at_end=False) == 0.0
    g.step(60)
    assert g.steps_done == 60
    # the oracle's forced run from t = 10 s matches the first run
    o = oracle.run_forced(oracle.params(120, 1, dt, manning_n2=0.0), x, np.zeros(1), d, np.zeros((1, 120)),
                          {0: (times, vals)}, nsteps=30, t0=10.0)
    assert np.abs(e1 - o["eta"]).max() <= 1e-4 * 0.05
    g.close()


def test_initial_conditions_interpolated_from_a_source_grid():
    """A coarser source grid covering part of the master grid: the GPU's interpolated initial
    state against the oracle's interpolation (both FP64, rounded to FP32), zero outside."""
    w = workloads.beach_200(140, 110, steps=10)
    rng = np.random.default_rng(21)
    sx = np.sort(rng.uniform(1500.0, 11000.0, 37))
    sy = np.sort(rng.uniform(-500.0, 8000.0, 29))
    SX, SY = np.meshgrid(sx, sy)
    eta = (0.4 * np.exp(-((SX - 6000.0) ** 2 + (SY - 4000.0) ** 2) / (2 * 2000.0 ** 2))).astype(np.float32)
    u = (0.1 * np.sin(SX / 3000.0)).astype(np.float32)
    g = CliffsGrid.from_workload(w)
    g.set_bathy(w.x, w.y, w.depth, False)
    g.set_initial_interp(sx, sy, eta, u)
    e32, u32, v32 = g.state()
    g.close()
    for got, src in ((e32, eta), (u32, u)):
        want = P.f32(oracle.interp_initial(w.x, w.y, sx, sy, src))
        assert np.all(np.abs(got - want) <= 2.5e-7 * np.abs(want) + 1e-12)
    assert not v32.any()
    MX, MY = np.meshgrid(w.x, w.y)
    outside = (MX < sx[0]) | (MX > sx[-1]) | (MY < sy[0]) | (MY > sy[-1])
    assert outside.any() and not e32[outside].any() and not u32[outside].any()


@pytest.mark.parametrize("alternate", [0, 1])
def test_adjoint_under_boundary_input_dot_product_against_oracle_tlm(alternate):
    """The beach child driven by the parent's series: <dL/d eta0, delta> from the GPU adjoint
    against the oracle's forced tangent model, with gauges on an input edge and inside, for
    both sweep orders. Same bound as the unforced dot-product tests (1e-4 of the largest
    term)."""
    from workloads import Nest
    w = workloads.beach_200(200, 120, steps=300)
    d64 = P.f32(P.oracle_depth(w))
    i0, j0, cx, cy = 110, 30, 90, 64
    nest = Nest(float(w.x[i0]), float(w.y[j0]), 100.0, 100.0, cx, cy)
    p = oracle.params_from(w)
    par = oracle.run(p, w.x, w.y, d64, w.eta0, nsteps=w.steps, bndout=1, nests=[nest])
    times = w.dt * np.arange(w.steps + 1)
    series = {e: (times, par["boundary"][0][e]) for e in range(4)}
    sub = (slice(j0, j0 + cy), slice(i0, i0 + cx))
    cxs, cys = w.x[i0:i0 + cx], w.y[j0:j0 + cy]
    gauges = np.array([(0, 32), (3, 40), (40, 32), (70, 20), (85, 32)], np.int32)
    n = w.steps
    g = CliffsGrid(cx, cy, w.dt, h_min=w.h_min, manning_n2=w.manning_n2, gauges=[tuple(q) for q in gauges],
                   alternate=alternate)
    g.set_bathy(cxs, cys, d64[sub], False)
    g.set_initial(w.eta0[sub].astype(np.float32))
    for e in range(4):
        g.set_boundary_input(e, times, series[e][1])
    rng = np.random.default_rng(23)
    seed = rng.standard_normal((n + 1, len(gauges))).astype(np.float32)
    grad = g.adjoint(n, seed, checkpoint_every=37).astype(np.float64)
    assert np.isfinite(grad).all()
    pc = oracle.params(cx, cy, w.dt, h_min=w.h_min, manning_n2=w.manning_n2, alternate=alternate)
    yy, xx = np.meshgrid(np.arange(cy), np.arange(cx), indexing="ij")
    worst = 0.0
    for k, (gx, gy, sig) in enumerate(((6.0, 30.0, 8.0), (45.0, 25.0, 10.0), (20.0, 40.0, 14.0))):
        delta = np.exp(-((xx - gx) ** 2 + (yy - gy) ** 2) / (2 * sig ** 2))
        if k == 2:
            delta = delta + 0.1 * rng.standard_normal(delta.shape)
        _, gtan = oracle.run_tlm_forced(pc, cxs, cys, d64[sub], w.eta0[sub], delta, series, nsteps=n,
                                        gauges=gauges)
        terms = seed.astype(np.float64) * gtan
        want = terms.sum()
        got = float((grad * delta).sum())
        scale = max(np.abs(terms).max(), 1e-12)
        err = abs(got - want) / scale
        worst = max(worst, err)
        assert err <= 1e-4, (k, got, want, scale)
    P.report("adjoint_dot_forced_beach_child_alt%d" % alternate, rel_err=worst)
    # an edge node under input reaches the loss only through its own record at step 0
    assert grad[32, 0] == pytest.approx(float(seed[0, 0]), rel=1e-6)
    assert not grad[1:31, 0].any() and not grad[:, -1][1:-1].any()
    g.close()


@pytest.mark.parametrize("alternate", [0, 1])
def test_persistent_run_under_boundary_input_equals_per_step(alternate):
    """The persistent run imposes the input itself before each step (its blocks write the
    edges, then meet at a grid barrier) from the host's interpolation table: state, maxima and
    records equal the per-step path bit for bit, across calls, with the cuke start and the
    stop at the end of the records."""
    from workloads import Nest
    x, y, d, eta0 = _open_water()
    dt, steps = 1.5, 60
    i0, j0, cx, cy = 41, 33, 70, 64
    nest = Nest(x[i0], y[j0], 100.0, 100.0, cx, cy)
    par = CliffsGrid(len(x), len(y), dt, manning_n2=6.25e-4, nests=[nest], bndout=1)
    par.set_bathy(x, y, d, False)
    par.set_initial(eta0.astype(np.float32))
    par.step(steps)
    series = [par.boundary(0, e) for e in range(4)]
    par.close()
    sub = (slice(j0, j0 + cy), slice(i0, i0 + cx))
    times = 10.0 + dt * np.arange(steps + 1) * 0.8         # records every 1.2 s: interpolated
    runs = []
    for pers in (False, True):
        ch = CliffsGrid(cx, cy, dt, manning_n2=6.25e-4, gauges=[(0, 20), (5, 30), (35, 32)], alternate=alternate)
        ch.set_bathy(x[i0:i0 + cx], y[j0:j0 + cy], d[sub], False)
        ch.set_initial(eta0[sub].astype(np.float32))
        for e in range(4):
            ch.set_boundary_input(e, times, series[e])
        ch.set_boundary_clock(1e-4, stop_at_end=True)
        ch.step(17, persistent=pers)
        ch.step(1000, persistent=pers)                     # stops at the end of the records
        runs.append((ch.steps_done, ch.state() + ch.maxwave() + (ch.gauges(),)))
        ch.close()
    assert runs[0][0] == runs[1][0] and 17 < runs[0][0] < 1000
    for p, q in zip(runs[0][1], runs[1][1]):
        assert np.array_equal(p, q)


def test_input_edges_with_open_edges_against_the_oracle():
    """Input on the west and east edges, the south and north edges open: the GPU's forced run
    against the oracle's (the open ghosts act on the edges without input)."""
    from workloads import Nest
    x, y, d, eta0 = _open_water()
    dt, steps = 1.5, 80
    i0, j0, cx, cy = 41, 33, 70, 64
    nest = Nest(x[i0], y[j0], 100.0, 100.0, cx, cy)
    par = CliffsGrid(len(x), len(y), dt, manning_n2=6.25e-4, nests=[nest], bndout=1)
    par.set_bathy(x, y, d, False)
    par.set_initial(eta0.astype(np.float32))
    par.step(steps)
    series = {e: (dt * np.arange(steps + 1), par.boundary(0, e).astype(np.float64)) for e in (0, 1)}
    par.close()
    sub = (slice(j0, j0 + cy), slice(i0, i0 + cx))
    gauges = np.array([(0, 20), (35, 0), (35, 63), (30, 30)], np.int32)
    d64 = d[sub].astype(np.float64)
    pc = oracle.params(cx, cy, dt, manning_n2=6.25e-4, open_edges=12)
    o = oracle.run_forced(pc, x[i0:i0 + cx], y[j0:j0 + cy], d64, eta0[sub], series, nsteps=steps, gout=1,
                          gauges=gauges)
    g = CliffsGrid(cx, cy, dt, manning_n2=6.25e-4, open_edges=12, gauges=[tuple(q) for q in gauges])
    g.set_bathy(x[i0:i0 + cx], y[j0:j0 + cy], d[sub], False)
    g.set_initial(eta0[sub].astype(np.float32))
    for e in (0, 1):
        g.set_boundary_input(e, series[e][0], series[e][1])
    g.step(steps)
    rel, absol = P.gauge_errors(g.gauges()[:, :, 0], o["gauges"][:, :, 0])
    P.report("forced_with_open_edges", gauge_rel_max=rel.max(initial=0.0), gauge_abs_max=absol.max(initial=0.0))
    assert rel.max(initial=0.0) <= P.GAUGE_RTOL and absol.max(initial=0.0) <= P.GAUGE_ATOL_SMALL
    assert np.abs(g.state()[0] - o["eta"]).max() <= 1e-4 * np.abs(eta0).max()
    # the open edges matter: with walls there the run differs
    w = oracle.run_forced(oracle.params(cx, cy, dt, manning_n2=6.25e-4), x[i0:i0 + cx], y[j0:j0 + cy], d64,
                          eta0[sub], series, nsteps=steps)
    assert np.abs(w["eta"] - o["eta"]).max() > 1e-3
    g.close()
