"""Scheme variants on the GPU against the FP64 oracle: the alternating sweep order (y first on
the odd steps, the alternating reading of section "Numerics").

Tolerances as in test_gpu_parity.py: gauge traces within 1e-4 of the oracle's max|eta| (1e-7
m absolute for traces below 1e-3 m), wet/dry masks equal except near round-off.
"""
import numpy as np
import pytest

import oracle
import workloads
from paper_1410_0753_gb300 import CliffsError, CliffsGrid, ERR_ARG
from tests import parity as P

pytestmark = pytest.mark.gpu


def _assert_gauges(name, g32, g64):
    rel, absol = P.gauge_errors(g32[:, :, 0], g64[:, :, 0])
    P.report(name, gauge_rel_max=rel.max(initial=0.0), gauge_abs_max=absol.max(initial=0.0))
    assert rel.max(initial=0.0) <= P.GAUGE_RTOL, rel
    assert absol.max(initial=0.0) <= P.GAUGE_ATOL_SMALL, absol


def _run_both(w, n, **kw):
    d64 = P.f32(P.oracle_depth(w))
    g = P.gpu_run(w, n, **kw)
    o = oracle.run(oracle.params_from(w, **{k: v for k, v in kw.items() if k in ("solver", "alternate")}),
                   w.x, w.y, d64, w.eta0, nsteps=n, maxout=w.maxout, gout=w.gout,
                   gauges=w.gauges if len(w.gauges) else None)
    return g, o, d64


@pytest.mark.parametrize("case", ["beach", "spherical"])
def test_alternating_order_against_oracle(case):
    if case == "beach":
        w = workloads.beach_200(200, 96, steps=400)          # the wave runs up the shore
    else:
        w = workloads.spherical_coast(220, 190, steps=160)
        w.nests = []
    n = w.steps
    g, o, d64 = _run_both(w, n, alternate=1)
    _assert_gauges("alternate_" + case, g["gauges"], o["gauges"])
    wet32, wet64, near = P.wet_masks(g["eta"], o["eta"], g["depth"], d64, w.h_min)
    assert np.array_equal(wet32 & ~near, wet64 & ~near)
    amp = np.abs(w.eta0).max()
    assert np.abs(g["eta"] - o["eta"])[wet64].max() <= 1e-4 * amp
    # the order matters: x-then-y differs from the alternating run
    g0 = P.gpu_run(w, n)
    assert not np.array_equal(g0["eta"], g["eta"])
    g["grid"].close()
    g0["grid"].close()


def test_alternating_order_keeps_1d_equal_2d():
    """With y-invariant data the y-sweep is the identity whichever sweep goes first, so the
    alternating 2D run still equals the 1D run row by row, bit for bit."""
    n, m, dt, steps = 130, 9, 1.5, 200
    x = np.arange(n) * 50.0
    d1 = 8.0 - 10.0 * x / x[-1]
    e1 = 0.6 * np.exp(-(x - 1500.0) ** 2 / (2 * 300.0 ** 2))
    kw = dict(h_min=0.01, manning_n2=6.25e-4)
    g1 = CliffsGrid(n, 1, dt, **kw)
    g1.set_bathy(x, np.zeros(1), d1[None, :], False)
    g1.set_initial(e1[None, :].astype(np.float32))
    g1.step(steps)
    g2 = CliffsGrid(n, m, dt, alternate=1, **kw)
    g2.set_bathy(x, np.arange(m) * 50.0, np.tile(d1, (m, 1)), False)
    g2.set_initial(np.tile(e1, (m, 1)).astype(np.float32))
    g2.step(steps)
    assert np.array_equal(g2.state()[0], np.tile(g1.state()[0], (m, 1)))
    assert np.array_equal(g2.state()[1], np.tile(g1.state()[1], (m, 1)))
    assert not np.any(g2.adjoint(4, None))      # the adjoint takes the alternating order too
    g1.close()
    g2.close()


@pytest.mark.parametrize("case", ["beach", "spherical_alternate", "line_x", "line_y"])
def test_solver1_against_oracle(case):
    """eq. (solver1) (the original VTCS-2 first-order term over the double interval) on wet/dry
    and spherical grids, with the alternating order, and on 1D lines along x and along y."""
    alt = 0
    if case == "beach":
        w = workloads.beach_200(200, 96, steps=400)          # the wave runs up the shore
    elif case == "spherical_alternate":
        w = workloads.spherical_coast(220, 190, steps=160)
        w.nests = []
        alt = 1
    else:
        b = workloads.beach_200(200, 3, steps=300)
        w = b
        row = 1
        w.depth = b.depth[row:row + 1]
        w.eta0 = b.eta0[row:row + 1]
        w.y = b.y[row:row + 1]
        w.ny = 1
        w.gauges = np.array([(ix, 0) for ix in (40, 100, 150, 180)], dtype=np.int32)
        if case == "line_y":
            w.depth, w.eta0 = w.depth.T.copy(), w.eta0.T.copy()
            w.x, w.y = w.y, b.x
            w.nx, w.ny = 1, 200
            w.gauges = w.gauges[:, ::-1].copy()
    n = w.steps
    g, o, d64 = _run_both(w, n, solver=1, alternate=alt)
    _assert_gauges("solver1_" + case, g["gauges"], o["gauges"])
    wet32, wet64, near = P.wet_masks(g["eta"], o["eta"], g["depth"], d64, w.h_min)
    assert np.array_equal(wet32 & ~near, wet64 & ~near)
    amp = np.abs(w.eta0).max()
    assert np.abs(g["eta"] - o["eta"])[wet64].max() <= 1e-4 * amp
    g0 = P.gpu_run(w, n, alternate=alt)                 # solver2 gives a different answer
    assert not np.array_equal(g0["eta"], g["eta"])
    g["grid"].close()
    g0["grid"].close()


def test_solver1_persistent_equals_per_step():
    w = workloads.ensemble_512(batch=4, nx=120, ny=100, dmin=20, dmax=60)
    runs = []
    for pers in (False, True):
        g = CliffsGrid.from_workload(w, solver=1)
        g.set_bathy(w.x, w.y, w.depth, True, w.filter_alpha, w.filter_min_depth)
        g.set_initial(w.eta0.astype(np.float32))
        g.set_durations(w.durations)
        g.step(int(w.durations.max()), persistent=pers)
        runs.append([g.state(b) for b in range(w.batch)] + [g.gauges(b) for b in range(w.batch)])
        g.close()
    for x, y in zip(runs[0], runs[1]):
        for p, q in zip(x if isinstance(x, tuple) else (x,), y if isinstance(y, tuple) else (y,)):
            assert np.array_equal(p, q)


def test_alternating_order_island_in_the_window_halo():
    """With y first, a warp's y-sweep results in the three columns past its outputs feed the
    x-sweep that follows, so they must be exact too. A small island in columns 56-58 lies in
    the halo of the first strip of columns (outputs 0-55) while that strip's own columns are
    open water; its north and south edges are walls in the y-sweep. Checked against the
    oracle next to the island, where column 55 reads columns 56-58."""
    nx, ny, dx, dt, steps = 120, 80, 50.0, 1.8, 120
    x, y = dx * np.arange(nx), dx * np.arange(ny)
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    d = np.full((ny, nx), 15.0)
    d[30:46, 56:59] = -1.0
    eta0 = 0.5 * np.exp(-((X - 30.0) ** 2 + (Y - 38.0) ** 2) / (2 * 6.0 ** 2))
    gauges = np.array([(55, 29), (55, 46), (55, 38), (53, 30), (59, 28), (20, 38)], np.int32)
    kw = dict(h_min=0.01, manning_n2=6.25e-4)
    g = CliffsGrid(nx, ny, dt, alternate=1, gauges=[tuple(q) for q in gauges], **kw)
    g.set_bathy(x, y, d, False)
    d64 = P.f32(g.depth())
    g.set_initial(eta0.astype(np.float32))
    g.step(steps)
    o = oracle.run(oracle.params(nx, ny, dt, alternate=1, **kw), x, y, d64, eta0, nsteps=steps, gout=1,
                   gauges=gauges)
    _assert_gauges("alternate_island_halo", g.gauges(), o["gauges"])
    e32 = g.state()[0]
    wet32, wet64, near = P.wet_masks(e32, o["eta"], d64, d64, 0.01)
    assert np.array_equal(wet32 & ~near, wet64 & ~near)
    assert np.abs(e32 - o["eta"])[wet64].max() <= 1e-4 * 0.5
    g.close()


@pytest.mark.parametrize("opts", [dict(), dict(solver=1), dict(open_edges=15)])
def test_alternating_order_persistent_equals_per_step(opts):
    """The persistent batched run with the alternating order (y first on the odd steps, a
    second worker of the y-first kind sharing each warp's ring) equals per-step launches bit
    for bit: state, maxima and gauge records of every scenario, uneven durations, calls that
    start on an odd step."""
    w = workloads.ensemble_512(batch=4, nx=120, ny=100, dmin=20, dmax=60)
    runs = []
    for pers in (False, True):
        g = CliffsGrid.from_workload(w, alternate=1, **opts)
        g.set_bathy(w.x, w.y, w.depth, True, w.filter_alpha, w.filter_min_depth)
        g.set_initial(w.eta0.astype(np.float32))
        g.set_durations(w.durations)
        g.step(7, persistent=pers)                       # the next call starts on an odd step
        g.step(int(w.durations.max()) - 7, persistent=pers)
        runs.append([g.state(b) + g.maxwave(b) + (g.gauges(b),) for b in range(w.batch)])
        g.close()
    for x, y in zip(runs[0], runs[1]):
        for p, q in zip(x, y):
            assert np.array_equal(p, q)
    # and the order matters: the same persistent run without alternation differs
    g = CliffsGrid.from_workload(w, **opts)
    g.set_bathy(w.x, w.y, w.depth, True, w.filter_alpha, w.filter_min_depth)
    g.set_initial(w.eta0.astype(np.float32))
    g.set_durations(w.durations)
    g.step(int(w.durations.max()), persistent=True)
    assert not np.array_equal(g.state(0)[0], runs[1][0][0])
    g.close()
