"""The wide fused step (four nodes per lane, 120 output columns per warp) against the two-node
fused step, bit for bit.

Both kernels apply the same per-node sequence of operations of the split step (section
"Numerics", steps (a)-(e) of section "Inundation algorithm"), so every output must be
identical: the state, the max-wave fields, the gauge records and the enclosed-grid boundary
series, on grids that flood and dry, on geographic and Cartesian metrics, with friction on
and off, at ragged sizes whose last strip is partial, on batched grids and with tile heights
that leave short items. The oracle parity tests run the wide kernel by default.
"""
import math

import numpy as np
import pytest

import workloads
from paper_1410_0753_gb300 import CliffsError, CliffsGrid, ERR_ARG

pytestmark = pytest.mark.gpu


def _run(w, kind, steps, rows=None, **kw):
    g = CliffsGrid.from_workload(w, **kw)
    g.set_bathy(w.x, w.y, w.depth, True, w.filter_alpha, w.filter_min_depth)
    g.set_step_kernel(kind)
    if rows:
        g.set_rows_per_warp(rows)
    g.set_initial(w.eta0.astype(np.float32))
    if w.durations is not None:
        g.set_durations(w.durations)
    g.step(steps)
    out = {}
    for b in range(w.batch):
        out["state%d" % b] = g.state(b)
        out["max%d" % b] = g.maxwave(b)
        if g.n_gauges:
            out["gauges%d" % b] = g.gauges(b)
    for m in range(len(w.nests) if w.batch == 1 else 0):
        for e in range(4):
            out["bnd%d_%d" % (m, e)] = g.boundary(m, e)
    g.close()
    return out


def _same(a, b):
    assert a.keys() == b.keys()
    for k in a:
        for x, y in zip(a[k] if isinstance(a[k], tuple) else (a[k],), b[k] if isinstance(b[k], tuple) else (b[k],)):
            assert np.array_equal(x, y), k


def _ragged(nx, ny, fric):
    rng = np.random.default_rng(nx * 7 + ny)
    x = np.sort(np.arange(nx) * 80.0 + rng.random(nx) * 10.0)
    y = np.arange(ny) * 90.0
    X, Y = np.meshgrid(x, y)
    d = 20.0 - 26.0 * (X / x[-1]) + 2.0 * np.sin(Y / 500.0)
    d -= 30.0 * np.exp(-((X - 0.4 * x[-1]) ** 2 + (Y - 0.5 * y[-1]) ** 2) / (2 * 400.0 ** 2))
    eta = 0.4 * np.exp(-((X - 0.3 * x[-1]) ** 2 + (Y - 0.4 * y[-1]) ** 2) / (2 * 500.0 ** 2))
    gauges = np.array([(k * 37 % nx, k * 23 % ny) for k in range(12)], np.int32)
    dt = 0.8 * 70.0 / math.sqrt(9.81 * 26.0)
    return workloads.Workload("ragged_%dx%d" % (nx, ny), nx, ny, 1, x, y, d, eta, dt, 200,
                              manning_n2=6.25e-4 if fric else 0.0, maxout=3, gout=2, gauges=gauges)


CASES = {
    "beach_runup": lambda: workloads.beach_200(200, 90, steps=400),
    "spherical_nests": lambda: workloads.spherical_coast(300, 260, steps=200),
    "ragged_131x97": lambda: _ragged(131, 97, True),
    "ragged_241x60_no_friction": lambda: _ragged(241, 60, False),
    "ragged_3x40": lambda: _ragged(3, 40, True),
    "ragged_121x5": lambda: _ragged(121, 5, True),
    "shelf_islands_600": lambda: workloads.shelf_islands(600, 520, steps=150),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_wide_step_equals_two_node_step(case):
    w = CASES[case]()
    _same(_run(w, 0, w.steps), _run(w, 1, w.steps))


@pytest.mark.parametrize("rows", [8, 34, 130])
def test_wide_step_equals_two_node_step_tile_heights(rows):
    w = workloads.spherical_coast(260, 300, steps=90)
    _same(_run(w, 0, w.steps, rows=rows), _run(w, 1, w.steps, rows=rows))


def test_wide_step_batched_per_step_launches():
    w = workloads.ensemble_512(batch=3, nx=250, ny=130, dmin=30, dmax=70)
    _same(_run(w, 0, int(w.durations.max())), _run(w, 1, int(w.durations.max())))


def test_wide_step_alternating_order():
    """With the alternating order the wide kernel takes the x-first steps and the two-node
    kernel the y-first ones."""
    w = workloads.beach_200(200, 90, steps=120)
    _same(_run(w, 0, w.steps, alternate=1), _run(w, 1, w.steps, alternate=1))


def test_step_kernel_argument():
    w = workloads.beach_200(40, 30, steps=5)
    g = CliffsGrid.from_workload(w)
    with pytest.raises(CliffsError) as e:
        g.set_step_kernel(2)
    assert e.value.code == ERR_ARG
    g.close()
