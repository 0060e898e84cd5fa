"""CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances: gauge traces within 1e-4 of the oracle's max |eta| per gauge (1e-7 m absolute
for traces that stay below 1e-3 m), the bound the FP32 step is held to over the runs here
(each step's FP32 rounding is a few 1e-7 of the state, accumulated over hundreds of steps,
and the perturbation form keeps the c = sqrt(g h) differences free of cancellation); wet/dry masks equal
except for cells whose oracle height or flooding margin lies within 1e-5 max(1, |d|) of
h_min (counted); the depth filter and every branch-free identity (lake at rest, 1D == 2D)
bit for bit.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
import workloads
from paper_1410_0753_gb300 import (CliffsError, CliffsGrid, ERR_ARG, ERR_STATE, ERR_TIMEOUT,
                                   ERR_UNSTABLE, cliffs_inject_wait_expiry)
from tests import parity as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1410_0753_gb300 import _build
    _build.build()
    oracle.threads(0)


def assert_gauges(name, g32, g64):
    rel, absol = P.gauge_errors(g32[:, :, 0], g64[:, :, 0])
    P.report(name, gauge_rel_max=rel.max() if len(rel) else 0.0,
             gauge_abs_max=absol.max() if len(absol) else 0.0, n_rel=len(rel), n_abs=len(absol))
    assert len(rel) == 0 or rel.max() <= P.GAUGE_RTOL, rel
    assert len(absol) == 0 or absol.max() <= P.GAUGE_ATOL_SMALL, absol


# ---------------------------------------------------------------------------- S0 filter

@pytest.mark.parametrize("case", ["beach", "spherical", "spiky"])
def test_depth_filter_bit_exact(case):
    if case == "beach":
        w = workloads.beach_200()
        x, y, d = w.x, w.y, w.depth
    elif case == "spherical":
        w = workloads.spherical_coast(300, 260)
        x, y, d = w.x, w.y, w.depth
    else:
        rng = np.random.default_rng(7)
        d = 50.0 + 40.0 * rng.standard_normal((97, 131))
        d[rng.random(d.shape) < 0.05] = 0.05
        d[:, :7] = -2.0
        d[40:50, 60:70] = -1.0
        x = np.arange(131) * 100.0
        y = np.arange(97) * 100.0
    ny, nx = d.shape
    g = CliffsGrid(nx, ny, 0.01, coords=1 if case != "spherical" else 0)
    g.set_bathy(x, y, d, True, 2.0, 0.1)
    got = g.depth()
    want, _ = oracle.depth_filter(d, 2.0, 0.1)
    P.report("filter_" + case, changed=int((want != d).sum()), mismatch=int((got != want).sum()))
    assert np.array_equal(got, want)
    g.close()


# ---------------------------------------------------------------------------- config 1

def test_beach_200_full_run():
    """2D Cartesian 200 x 200, 1000 steps, Manning n = 0.025, 8 gauges, max-wave each step."""
    w = workloads.beach_200()
    d64 = P.oracle_depth(w)
    g = P.gpu_run(w, w.steps)
    assert np.array_equal(g["depth"], d64)
    o = P.oracle_run(w, w.steps, P.f32(d64))
    assert_gauges("beach_200", g["gauges"], o["gauges"])
    # max-wave over wet nodes
    wet_ever = o["eta_max"] > -1e30
    emax_err = np.abs(g["eta_max"][wet_ever] - o["eta_max"][wet_ever]).max()
    smax_err = np.abs(g["speed_max"] - o["speed_max"]).max()
    wet32, wet64, near = P.wet_masks(g["eta"], o["eta"], P.f32(d64), P.f32(d64), w.h_min)
    mism = wet32 != wet64
    P.report("beach_200", emax_abs=emax_err, smax_abs=smax_err, eta_abs=np.abs(g["eta"] - o["eta"]).max(),
             mask_mismatch=int(mism.sum()), mask_mismatch_not_near=int((mism & ~near).sum()),
             wet_cells=int(wet64.sum()))
    assert emax_err <= 1e-4 * 0.5
    assert smax_err <= 1e-3
    assert (mism & ~near).sum() == 0
    g["grid"].close()


# ---------------------------------------------------------------------------- identities

def test_lake_at_rest_is_exact():
    nx, ny = 150, 90
    x = np.arange(nx) * 100.0
    y = np.arange(ny) * 100.0
    X, Y = np.meshgrid(x, y)
    d = 30.0 - 40.0 * X / x[-1] + 3.0 * np.sin(Y / 400.0)
    d -= 50.0 * np.exp(-((X - 5000) ** 2 + (Y - 4000) ** 2) / (2 * 600.0 ** 2))
    for itopo in (1, 0):
        g = CliffsGrid(nx, ny, 1.0, h_min=0.01, manning_n2=6.25e-4, itopo=itopo, dwall=2.0)
        g.set_bathy(x, y, d)
        g.set_initial(np.zeros((ny, nx), np.float32))
        g.step(500)
        e, u, v = g.state()
        assert not e.any() and not u.any() and not v.any()
        g.close()


def beach_line(n=130):
    x = np.arange(n) * 50.0
    d = 8.0 - 10.0 * x / x[-1]
    eta = 0.6 * np.exp(-(x - 1500.0) ** 2 / (2 * 300.0 ** 2))
    return x, d, eta


def test_1d_equals_2d_bit_exact():
    """Dimensional splitting: y-invariant data between reflecting walls leaves the y-sweep
    the identity, so every row of the fused 2D step equals the 1D x-sweep (and transposed)."""
    x, d1, e1 = beach_line()
    n, m, dt, steps = len(x), 9, 1.5, 300
    kw = dict(h_min=0.01, manning_n2=6.25e-4)
    g1 = CliffsGrid(n, 1, dt, **kw)
    g1.set_bathy(x, np.zeros(1), d1[None, :], False)
    g1.set_initial(e1[None, :].astype(np.float32))
    g1.step(steps)
    r1 = g1.state()
    g2 = CliffsGrid(n, m, dt, **kw)
    g2.set_bathy(x, np.arange(m) * 50.0, np.tile(d1, (m, 1)), False)
    g2.set_initial(np.tile(e1, (m, 1)).astype(np.float32))
    g2.step(steps)
    r2 = g2.state()
    assert np.array_equal(r2[0], np.tile(r1[0], (m, 1)))
    assert np.array_equal(r2[1], np.tile(r1[1], (m, 1)))
    assert not r2[2].any()
    # transposed: 1D along y against x-invariant 2D
    g3 = CliffsGrid(1, n, dt, **kw)
    g3.set_bathy(np.zeros(1), x, d1[:, None], False)
    g3.set_initial(e1[:, None].astype(np.float32))
    g3.step(steps)
    r3 = g3.state()
    g4 = CliffsGrid(m, n, dt, **kw)
    g4.set_bathy(np.arange(m) * 50.0, x, np.tile(d1[:, None], (1, m)), False)
    g4.set_initial(np.tile(e1[:, None], (1, m)).astype(np.float32))
    g4.step(steps)
    r4 = g4.state()
    assert np.array_equal(r4[0], np.tile(r3[0], (1, m)))
    assert np.array_equal(r4[2], np.tile(r3[2], (1, m)))
    assert not r4[1].any()
    # and the 1D runs agree with the oracle
    o = oracle.run(oracle.params(n, 1, dt, **kw), x, np.zeros(1), P.f32(d1)[None, :],
                   P.f32(e1)[None, :], nsteps=steps)
    wet = (o["eta"][0] + P.f32(d1)) >= 0.01
    err = np.abs(r1[0][0] - o["eta"][0])[wet].max()
    P.report("line_130", eta_abs=err)
    assert err <= 1e-4 * 0.6
    for g in (g1, g2, g3, g4):
        g.close()


# ---------------------------------------------------------------------------- window edges

@pytest.mark.parametrize("shape", [(64, 40), (120, 33), (176, 21), (61, 45)])
def test_windows_ending_at_the_domain_edge_against_oracle(shape):
    """All-wet grids whose x-sweep windows end exactly at the domain's edges (64: one window,
    both edges; 120 and 176: the last window's edge is the domain's) or one window past it
    (61): a wave reflected by the walls inside those windows against the oracle."""
    nx, ny = shape
    x = np.arange(nx) * 60.0
    y = np.arange(ny) * 75.0
    X, Y = np.meshgrid(x, y)
    d = 20.0 + 5.0 * np.sin(X / 700.0) * np.cos(Y / 900.0)
    eta = 0.5 * np.exp(-((X - 0.1 * x[-1]) ** 2 + (Y - 0.6 * y[-1]) ** 2) / (2 * 300.0 ** 2)) \
        - 0.3 * np.exp(-((X - 0.95 * x[-1]) ** 2 + (Y - 0.3 * y[-1]) ** 2) / (2 * 250.0 ** 2))
    gauges = [(0, ny // 2), (nx - 1, ny // 3), (min(nx - 1, 59), 1), (min(nx - 1, 60), ny - 2), (nx // 2, 0)]
    dt = 0.8 * 60.0 / math.sqrt(9.81 * 26.0)
    kw = dict(h_min=0.01, manning_n2=6.25e-4, maxout=1, gout=1)
    steps = 200
    g = CliffsGrid(nx, ny, dt, gauges=gauges, **kw)
    g.set_bathy(x, y, d)
    d64, _ = oracle.depth_filter(d)
    g.set_initial(eta.astype(np.float32))
    g.step(steps)
    e32, u32, v32 = g.state()
    p = oracle.params(nx, ny, dt, **{k: v for k, v in kw.items() if k not in ("maxout", "gout")})
    o = oracle.run(p, x, y, P.f32(d64), P.f32(eta), nsteps=steps, maxout=1, gout=1, gauges=gauges)
    err = np.abs(e32 - o["eta"]).max()
    uerr = np.abs(u32 - o["u"]).max()
    P.report("window_edges_%dx%d" % shape, eta_abs=err, u_abs=uerr)
    assert err <= 1e-4 * 0.5
    assert uerr <= 1e-4 * 0.5
    assert_gauges("window_edges_%dx%d" % shape, g.gauges(), o["gauges"])
    g.close()


# ---------------------------------------------------------------------------- ragged sizes

@pytest.mark.parametrize("shape", [(131, 97), (57, 203), (3, 3), (200, 1), (1, 150), (345, 17)])
def test_ragged_shapes_against_oracle(shape):
    nx, ny = shape
    rng = np.random.default_rng(nx * 1000 + ny)
    x = np.arange(nx) * 80.0 + (rng.random(nx) * 10.0 if nx > 1 else 0.0)
    x = np.sort(x) if nx > 1 else np.zeros(1)
    y = np.arange(ny) * 90.0
    X, Y = np.meshgrid(x, y)
    d = 20.0 - 26.0 * (X / max(x[-1], 1.0)) + 2.0 * np.sin(Y / 500.0)
    if nx > 20 and ny > 20:
        d -= 30.0 * np.exp(-((X - 0.4 * x[-1]) ** 2 + (Y - 0.5 * y[-1]) ** 2) / (2 * 400.0 ** 2))
    eta = 0.4 * np.exp(-((X - 0.3 * x[-1]) ** 2 + (Y - 0.4 * y[-1]) ** 2) / (2 * 500.0 ** 2))
    gauges = [(min(nx - 1, k * 7 % nx), min(ny - 1, k * 5 % ny)) for k in range(5)]
    dt = 0.8 * 70.0 / math.sqrt(9.81 * 26.0)
    kw = dict(h_min=0.01, manning_n2=6.25e-4, maxout=3, gout=2)
    steps = 240
    g = CliffsGrid(nx, ny, dt, gauges=gauges, **kw)
    g.set_bathy(x, y, d)
    d64, _ = oracle.depth_filter(d)
    assert np.array_equal(g.depth(), d64)
    g.set_initial(eta.astype(np.float32))
    g.step(steps)
    e32, u32, v32 = g.state()
    p = oracle.params(nx, ny, dt, **{k: v for k, v in kw.items() if k not in ("maxout", "gout")})
    o = oracle.run(p, x, y, P.f32(d64), P.f32(eta), nsteps=steps, maxout=3, gout=2, gauges=gauges)
    wet32, wet64, near = P.wet_masks(e32, o["eta"], P.f32(d64), P.f32(d64), 0.01)
    both = wet32 & wet64
    err = np.abs(e32 - o["eta"])[both].max() if both.any() else 0.0
    uerr = np.abs(u32 - o["u"])[both].max() if both.any() else 0.0
    P.report("ragged_%dx%d" % shape, eta_abs=err, u_abs=uerr,
             mask_mismatch=int((wet32 != wet64).sum()))
    assert err <= 1e-4 * 0.4 + 1e-6
    assert ((wet32 != wet64) & ~near).sum() == 0
    assert_gauges("ragged_%dx%d" % shape, g.gauges(), o["gauges"])
    em, sm = g.maxwave()
    ok = o["eta_max"] > -1e30
    assert np.abs(em[ok] - o["eta_max"][ok]).max() <= 1e-4 * 0.4 + 1e-6
    assert np.array_equal(em[~ok], o["eta_max"][~ok].astype(np.float32))
    g.close()


# ---------------------------------------------------------------------------- spherical + nests

def test_spherical_coast_small_with_nests():
    w = workloads.spherical_coast(300, 260, steps=400)
    d64 = P.oracle_depth(w)
    g = P.gpu_run(w, w.steps)
    assert np.array_equal(g["depth"], d64)
    o = P.oracle_run(w, w.steps, P.f32(d64))
    assert_gauges("spherical_300x260", g["gauges"], o["gauges"])
    worst = 0.0
    for m in range(len(w.nests)):
        for e in range(4):
            b32, b64 = g["boundary"][m][e], o["boundary"][m][e]
            assert b32.shape == b64.shape
            scale = max(np.abs(b64[:, 2]).max(), 1e-3)
            worst = max(worst, np.abs(b32[:, 2] - b64[:, 2]).max() / scale)
    wet32, wet64, near = P.wet_masks(g["eta"], o["eta"], P.f32(d64), P.f32(d64), w.h_min)
    P.report("spherical_300x260", boundary_eta_rel=worst, mask_mismatch=int((wet32 != wet64).sum()),
             mask_mismatch_not_near=int(((wet32 != wet64) & ~near).sum()))
    assert worst <= 1e-4
    assert ((wet32 != wet64) & ~near).sum() == 0
    g["grid"].close()


def test_spherical_coast_high_latitude():
    """The same coast moved to 55-57 N, where cos(phi) is 0.57 instead of 0.94, with its
    enclosed grids and a time step shortened for the narrower cells (Courant 0.8)."""
    w = workloads.spherical_coast(200, 160, steps=300)
    w.y = np.asarray(w.y, np.float64) + 35.0
    w.nests = [dataclasses.replace(n, y0=n.y0 + 35.0) for n in w.nests]
    w.dt = 0.6 * w.dt
    d64 = P.oracle_depth(w)
    g = P.gpu_run(w, w.steps)
    o = P.oracle_run(w, w.steps, P.f32(d64))
    assert_gauges("spherical_high_latitude", g["gauges"], o["gauges"])
    worst = 0.0
    for m in range(len(w.nests)):
        for e in range(4):
            b32, b64 = g["boundary"][m][e], o["boundary"][m][e]
            scale = max(np.abs(b64[:, 2]).max(), 1e-3)
            worst = max(worst, np.abs(b32[:, 2] - b64[:, 2]).max() / scale)
    wet32, wet64, near = P.wet_masks(g["eta"], o["eta"], P.f32(d64), P.f32(d64), w.h_min)
    P.report("spherical_high_latitude", boundary_eta_rel=worst, mask_mismatch=int((wet32 != wet64).sum()))
    assert worst <= 1e-4
    assert ((wet32 != wet64) & ~near).sum() == 0
    g["grid"].close()


# ---------------------------------------------------------------------------- quake, batch

@pytest.mark.parametrize("itopo,dwall", [(1, 0.0), (0, 45.0)])
def test_quake_initial_condition(itopo, dwall):
    w = workloads.beach_200(120, 90, steps=150)
    w.itopo, w.dwall = itopo, dwall                          # with itopo = 0: the slope is walls
    d64 = P.oracle_depth(w)
    zeta = w.eta0.astype(np.float32)
    g = CliffsGrid.from_workload(w)
    g.set_bathy(w.x, w.y, w.depth)
    g.set_initial(zeta, quake=1)
    dq, eq = oracle.quake_init(d64, zeta.astype(np.float64), w.h_min, itopo=itopo, dwall=dwall)
    assert np.array_equal(g.depth(), dq)
    assert np.array_equal(g.state()[0], eq.astype(np.float32))
    if not itopo:                                            # some walls carry a deformation
        walls = (d64 >= w.h_min) & (d64 < dwall)
        assert walls.any() and np.abs(zeta[walls]).max() > 0
    g.step(w.steps)
    o = oracle.run(oracle.params_from(w), w.x, w.y, P.f32(dq), eq, nsteps=w.steps, gout=1,
                   gauges=w.gauges)
    assert_gauges("quake", g.gauges(), o["gauges"])
    g.close()


@pytest.mark.parametrize("alternate", [0, 1])
def test_exact_resume_from_the_read_state(alternate):
    """Checkpoint and resume: the state (eta, u, v) is the whole state of the method, so a run
    continued from the state read after 50 steps equals the 80-step run bit for bit (state
    and gauge records), and the max-wave of the two parts combines to the whole run's. With
    the alternating order the resume is at an even step, whose order restarts x first."""
    w = workloads.beach_200(steps=80)
    X, Y = np.meshgrid(w.x, w.y)
    w.eta0 = (1.0 * np.exp(-((X - w.x[165]) ** 2 + (Y - w.y[100]) ** 2) / (2 * 800.0 ** 2))).astype(np.float32)
    w.eta0 = np.maximum(w.eta0, -w.depth).astype(np.float32)

    def grid():
        g = CliffsGrid.from_workload(w, alternate=alternate)
        g.set_bathy(w.x, w.y, w.depth)
        return g

    full = grid()
    full.set_initial(w.eta0)
    full.step(80)
    first = grid()
    first.set_initial(w.eta0)
    first.step(50)
    second = grid()
    second.set_initial(*first.state())
    second.step(30)
    for a, b in zip(full.state(), second.state()):
        assert np.array_equal(a, b)
    assert np.array_equal(full.gauges()[50:], second.gauges())
    (ea, sa), (eb, sb), (ec, sc) = full.maxwave(), first.maxwave(), second.maxwave()
    assert np.array_equal(ea, np.maximum(eb, ec))
    # the resumed grid's initial speed is sqrt(u^2 + v^2) in IEEE form, the step's an
    # approximate-reciprocal form: a maximum reached exactly at the resume step may differ
    # in the last bits
    assert np.allclose(sa, np.maximum(sb, sc), rtol=1e-6, atol=0.0)
    # the run floods land, so the wet/dry logic takes part
    d = full.depth()
    assert ((d < 0) & (full.maxwave()[0] + d > w.h_min)).any()
    for g in (full, first, second):
        g.close()


def _control_widths(c):
    c = np.asarray(c, np.float64)
    if len(c) < 2:
        return np.ones(len(c))
    w = np.empty(len(c))
    w[0], w[-1] = c[1] - c[0], c[-1] - c[-2]
    w[1:-1] = 0.5 * (c[2:] - c[:-2])
    return w


@pytest.mark.parametrize("name", ["beach", "spherical"])
def test_diagnostics_against_their_definition_and_the_oracle(name):
    w = workloads.beach_200(steps=60) if name == "beach" else workloads.spherical_coast(96, 80, steps=60)
    g = CliffsGrid.from_workload(w)
    g.set_bathy(w.x, w.y, w.depth, True, w.filter_alpha, w.filter_min_depth)
    g.set_initial(w.eta0.astype(np.float32))
    g.step(w.steps)
    dg = g.diagnostics()
    e, u, v = g.state()
    d64 = g.depth()
    d32 = d64.astype(np.float32)
    wall = -np.float32(3.402823466e38) if w.itopo else np.float32(w.dwall)
    wet = (d32 >= wall) & (e + d32 >= np.float32(w.h_min))
    wx, wy = _control_widths(w.x), _control_widths(w.y)
    if w.coords != 1:
        R, deg = 6371000.0, np.pi / 180.0
        wx = wx * R * deg
        wy = wy * R * deg * np.cos(np.asarray(w.y, np.float64) * deg)
    A = wy[:, None] * wx[None, :]
    ea = e.astype(np.float64) * A
    assert abs(dg["volume"] - ea[wet].sum()) <= 1e-9 * np.abs(ea[wet]).sum()
    assert dg["wet"] == wet.sum() and 0 < dg["wet"] < w.nx * w.ny
    assert dg["eta_abs_max"] == np.abs(e[wet]).max()
    assert np.isclose(dg["speed_max"], np.sqrt(u * u + v * v)[wet].max(), rtol=1e-6, atol=0.0)
    # the same volume over the FP64 oracle's state after the same steps
    o = oracle.run(oracle.params_from(w), w.x, w.y, P.oracle_depth(w), w.eta0, nsteps=w.steps)
    wo = (o["eta"] + P.oracle_depth(w) >= w.h_min)
    vo = (o["eta"] * A)[wo].sum()
    assert abs(dg["volume"] - vo) <= 1e-4 * np.abs(o["eta"] * A)[wo].sum()
    g.close()


def test_batch_with_durations_matches_single_runs():
    w = workloads.ensemble_512(batch=5, nx=96, ny=80, dmin=20, dmax=120)
    g = P.gpu_run(w, int(w.durations.max()) + 5)
    grid = g["grid"]
    for b in range(w.batch):
        single = CliffsGrid.from_workload(w, batch=1)
        single.set_bathy(w.x, w.y, w.depth)
        single.set_initial(w.eta0[b].astype(np.float32))
        single.step(int(w.durations[b]))
        e1, _, _ = single.state()
        eb, _, _ = grid.state(b)
        assert np.array_equal(eb, e1)
        gb, g1 = grid.gauges(b), single.gauges()
        assert gb.shape == g1.shape == (int(w.durations[b]) + 1, 16, 3)
        assert np.array_equal(gb, g1)
        # diagnostics of a scenario read its own state plane (block sums add in any order)
        db, d1 = grid.diagnostics(b), single.diagnostics()
        assert math.isclose(db["volume"], d1["volume"], rel_tol=1e-12, abs_tol=1e-6)
        assert (db["wet"], db["eta_abs_max"], db["speed_max"]) == (d1["wet"], d1["eta_abs_max"], d1["speed_max"])
        single.close()
    b = 2
    d64 = P.oracle_depth(w)
    o = oracle.run(oracle.params_from(w), w.x, w.y, P.f32(d64), w.eta0[b],
                   nsteps=int(w.durations[b]), gout=1, gauges=w.gauges)
    assert_gauges("batch_scenario2", grid.gauges(b), o["gauges"])
    grid.close()


# ---------------------------------------------------------------------------- full-size windows

def window_check(w, k, centres, name, eta0=None, half=8):
    """Full-size grid on the GPU for k steps; the oracle re-runs only the domain of dependence
    (3 nodes per sweep in each direction) around each sample, so the central block is exact."""
    d64 = P.oracle_depth(w)
    if eta0 is not None:
        w.eta0 = eta0
    g = P.gpu_run(w, k)
    R = 3 * k + 4 + half
    eta0 = w.eta0 if w.eta0.ndim == 2 else w.eta0[0]
    scale = max(np.abs(eta0).max(), 1e-3)
    worst, moved, wetdry = 0.0, 0.0, 0
    for (cy, cx) in centres:
        j0, j1 = max(0, cy - R), min(w.ny, cy + R + 1)
        i0, i1 = max(0, cx - R), min(w.nx, cx + R + 1)
        p = oracle.params(i1 - i0, j1 - j0, w.dt, w.coords, w.h_min, w.manning_n2, w.itopo,
                          w.dwall, w.transverse)
        dwin = P.f32(d64[j0:j1, i0:i1])
        o = oracle.run(p, w.x[i0:i1], w.y[j0:j1], dwin, eta0[j0:j1, i0:i1], nsteps=k)
        sl64 = (slice(cy - j0 - half, cy - j0 + half + 1), slice(cx - i0 - half, cx - i0 + half + 1))
        sl32 = (slice(cy - half, cy + half + 1), slice(cx - half, cx + half + 1))
        blk64, blk32 = o["eta"][sl64], g["eta"][sl32]
        worst = max(worst, np.abs(blk32 - blk64).max() / scale)
        moved = max(moved, np.abs(blk64 - eta0[sl32]).max() / scale)
        wet32, wet64, near = P.wet_masks(blk32, blk64, dwin[sl64], dwin[sl64], w.h_min)
        assert ((wet32 != wet64) & ~near).sum() == 0
        wetdry += int((~wet64).sum())
    P.report(name, window_eta_rel=worst, moved_rel=moved, dry_cells_sampled=wetdry, steps=k)
    assert moved > 1e-3                    # the sampled blocks do carry the wave
    g["grid"].close()
    return worst, wetdry


def test_full_size_spherical_2048_windows():
    w = workloads.spherical_coast(2048, 2048, steps=150)
    jc, ic = np.unravel_index(np.argmax(w.eta0), w.eta0.shape)
    centres = [(jc, ic), (jc + 40, ic + 60), (jc - 50, ic - 40)]
    worst, _ = window_check(w, 150, centres, "spherical_2048_windows")
    assert worst <= 1e-4


def test_full_size_spherical_2048_shoreline_windows():
    """Same full-size launch, with a 3 m hump on the coast so the sampled blocks flood and dry."""
    w = workloads.spherical_coast(2048, 2048, steps=100)
    j = np.arange(w.ny)
    d = w.depth
    row = 1300
    ic = int(np.argmax(d[row] > 0))                      # first wet node east of the coast
    J, I = np.meshgrid(j, np.arange(w.nx), indexing="ij")
    hump = 3.0 * np.exp(-((J - row) ** 2 + (I - ic - 10) ** 2) / (2 * 12.0 ** 2))
    worst, dry = window_check(w, 100, [(row, ic), (row + 15, ic - 5)], "spherical_2048_shore",
                              eta0=P.f32(hump))
    assert dry > 0 and worst <= 1e-4


def test_full_size_shelf_islands_8192_windows():
    w = workloads.shelf_islands(8192, 8192, steps=40)
    centres = [(4096, 800), (2000, 860), (7000, 760)]
    worst, _ = window_check(w, 40, centres, "shelf_8192_windows")
    assert worst <= 1e-4


def test_full_size_shelf_islands_8192_windows_300_steps():
    """The stress grid in the bench's launch configuration over 300 steps: blocks on both
    fronts of the split N-wave, each against an oracle window holding its whole domain of
    dependence (912 nodes each way)."""
    w = workloads.shelf_islands(8192, 8192, steps=300)
    c = int(round(40.0e3 / 50.0))
    shift = int(np.sqrt(9.81 * 200.0) * w.dt * 300 / 50.0)
    worst, _ = window_check(w, 300, [(4096, c + shift), (2000, c - shift)], "shelf_8192_windows_300")
    assert worst <= 1e-4


def test_full_size_shelf_islands_8192_island_windows():
    w = workloads.shelf_islands(8192, 8192, steps=60)
    land = w.depth < 0
    jj, ii = np.nonzero(land)
    k = len(jj) // 2
    cy, cx = int(jj[k]), int(ii[k])
    J, I = np.ogrid[:w.ny, :w.nx]
    hump = 2.0 * np.exp(-((J - cy) ** 2 + (I - cx) ** 2) / (2 * 60.0 ** 2))
    worst, dry = window_check(w, 60, [(cy, cx), (cy + 30, cx + 30)], "shelf_8192_island",
                              eta0=P.f32(hump))
    assert dry > 0 and worst <= 1e-4


# ---------------------------------------------------------------------------- errors

def test_error_paths():
    x = np.arange(20) * 10.0
    d = np.full((20, 20), 100.0)
    g = CliffsGrid(20, 20, 5.0)
    with pytest.raises(CliffsError) as e:
        g.set_bathy(x, x, d)                         # sqrt(g 100) * 5 / 10 = 15.7 > 1
    assert e.value.code == ERR_ARG and "Courant" in str(e.value)
    g.close()
    g = CliffsGrid(20, 20, 0.1)
    with pytest.raises(CliffsError) as e:
        g.step(1)
    assert e.value.code == ERR_STATE
    g.set_bathy(x, x, d)
    # host-side fault injection: a NaN velocity in a wet cell (a NaN surface would read as
    # a dry cell, which step (b) refills at h_min)
    u = np.zeros((20, 20), np.float32)
    u[5, 5] = np.nan
    g.set_initial(np.zeros((20, 20), np.float32), u)
    with pytest.raises(CliffsError) as e:
        g.step(3)
    assert e.value.code == ERR_UNSTABLE
    g.set_initial(np.zeros((20, 20), np.float32))    # the handle stays usable
    g.step(3)
    # a finite velocity far past any physical one
    u = np.zeros((20, 20), np.float32)
    u[5, 5] = 4e5
    g.set_initial(np.zeros((20, 20), np.float32), u)
    with pytest.raises(CliffsError) as e:
        g.step(1)
    assert e.value.code == ERR_UNSTABLE
    g.close()
    # the same on the 1D kernels (a line along x, a line along y)
    for nx, ny in ((20, 1), (1, 20)):
        g = CliffsGrid(nx, ny, 0.1)
        g.set_bathy(x[:nx], x[:ny], d[:ny, :nx])
        w0 = np.zeros((ny, nx), np.float32)
        w0.flat[7] = np.nan
        g.set_initial(np.zeros((ny, nx), np.float32), w0 if nx > 1 else None, None if nx > 1 else w0)
        with pytest.raises(CliffsError) as e:
            g.step(2)
        assert e.value.code == ERR_UNSTABLE
        g.close()
    with pytest.raises(CliffsError) as e:
        CliffsGrid(20, 20, 0.1, gauges=[(25, 3)])
    assert e.value.code == ERR_ARG


def test_zero_and_negative_step_counts():
    """n = 0 steps is a no-op (no launch, no record); a negative count is an argument error
    that leaves the grid as it was."""
    w = workloads.beach_200(120, 90, steps=10)
    g = CliffsGrid.from_workload(w)
    g.set_bathy(w.x, w.y, w.depth)
    g.set_initial(w.eta0.astype(np.float32))
    g.step(3)
    before = g.state(), g.gauges(), g.steps_done
    g.step(0)
    with pytest.raises(CliffsError) as e:
        g.step(-1)
    assert e.value.code == ERR_ARG
    with pytest.raises(CliffsError) as e:
        g.set_initial(w.eta0.astype(np.float32), scenario=1)    # batch 1: no scenario 1
    assert e.value.code == ERR_ARG
    after = g.state(), g.gauges(), g.steps_done
    for a, b in zip(before[0], after[0]):
        assert np.array_equal(a, b)
    assert np.array_equal(before[1], after[1]) and before[2] == after[2] == 3
    g.close()


def test_bounded_wait_expiry_reports_timeout_and_recovers():
    """A ring wait that can never complete (injected: the slots expect bytes no copy
    delivers) expires after its cycle limit; the step reports CLIFFS_ERR_TIMEOUT, the later
    launches of the call return at once, and the grid keeps working."""
    w = workloads.beach_200(120, 90, steps=20)
    g = CliffsGrid.from_workload(w)
    g.set_bathy(w.x, w.y, w.depth)
    g.set_initial(w.eta0.astype(np.float32))
    cliffs_inject_wait_expiry(g.h, 2_000_000)           # ~1 ms per wait
    with pytest.raises(CliffsError) as e:
        g.step(5)
    assert e.value.code == ERR_TIMEOUT
    g.set_initial(w.eta0.astype(np.float32))
    g.step(w.steps)
    ref = CliffsGrid.from_workload(w)
    ref.set_bathy(w.x, w.y, w.depth)
    ref.set_initial(w.eta0.astype(np.float32))
    ref.step(w.steps)
    assert np.array_equal(g.state()[0], ref.state()[0])
    g.close()
    ref.close()


def test_autotuned_tile_shape_gives_identical_results():
    """The rows-per-warp tile shape changes only how the work is split: every output node is
    computed by the same arithmetic, so any shape gives the same bits."""
    w = workloads.spherical_coast(300, 260, steps=80)
    runs = []
    for tune in ("default", "autotune", 1, 7, 300):     # fixed shapes: one row, odd, taller than the grid
        g = CliffsGrid.from_workload(w)
        g.set_bathy(w.x, w.y, w.depth)
        g.set_initial(w.eta0.astype(np.float32))
        if tune == "autotune":
            table = g.autotune(2)
            assert len(table) >= 3 and all(t > 0 for t in table.values())
        elif tune != "default":
            g.set_rows_per_warp(tune)
        g.step(w.steps)
        runs.append((g.state(), g.gauges(), g.maxwave(), g.boundary(0, 2)))
        g.close()
    s0, g0, m0, b0 = runs[0]
    for s1, g1, m1, b1 in runs[1:]:
        for x, y in zip(s0 + m0, s1 + m1):
            assert np.array_equal(x, y)
        assert np.array_equal(g0, g1) and np.array_equal(b0, b1)
    g1d = CliffsGrid(50, 1, 1.0)
    with pytest.raises(CliffsError) as e:
        g1d.set_rows_per_warp(8)                           # before set_bathy
    assert e.value.code == ERR_STATE
    g1d.set_bathy(np.arange(50) * 10.0, np.zeros(1), np.full((1, 50), 5.0), False)
    with pytest.raises(CliffsError) as e:
        g1d.set_rows_per_warp(8)                           # a 1D grid has no tile
    assert e.value.code == ERR_ARG
    g1d.close()


def test_state_views_are_zero_copy():
    """cliffs_state_ptrs: torch views of the library's current state buffers equal
    read_state, follow the alternating buffers, and writes through them are the state."""
    w = workloads.beach_200(100, 70, steps=6)
    g = CliffsGrid.from_workload(w)
    g.set_bathy(w.x, w.y, w.depth)
    g.set_initial(w.eta0.astype(np.float32))
    for n in (3, 1):                                   # both buffers of the pair
        g.step(n)
        views = g.state_views()
        for v, s in zip(views, g.state()):
            assert v.shape == (70, 100) and np.array_equal(v.cpu().numpy(), s)
    e, u, v = g.state_views()
    e.fill_(0.25)
    u.zero_()
    assert np.all(g.state()[0] == 0.25) and not g.state()[1].any()
    g.close()


# ---------------------------------------------------------------------------- degenerate cases

def _run_pair(x, y, d, eta, steps, u=None, **kw):
    """GPU and oracle on the same small grid (no depth filter); returns (gpu state, oracle run)."""
    nx, ny = len(x), len(y)
    dt = kw.pop("dt")
    g = CliffsGrid(nx, ny, dt, **kw)
    g.set_bathy(x, y, d, False)
    g.set_initial(eta.astype(np.float32), None if u is None else u.astype(np.float32))
    g.step(steps)
    st = g.state()
    g.close()
    p = oracle.params(nx, ny, dt, **{k: v for k, v in kw.items() if k in ("h_min", "manning_n2", "itopo", "dwall")})
    o = oracle.run(p, x, y, P.f32(d), P.f32(eta), None if u is None else P.f32(u), None, nsteps=steps)
    return st, o


@pytest.mark.parametrize("case", ["all_land", "single_wet_cell", "exact_threshold", "flood_tie", "walls_only"])
def test_degenerate_cases_against_oracle(case):
    """Inputs at the method's edges, with dyadic values so that FP32 and FP64 take the same
    decisions: an all-dry grid (nothing moves, velocities forced to zero), a single wet cell
    in a dry basin, a node exactly at h = h_min (wet, reading 1), a dry node between two wet
    neighbours of equal eta (reading 2: the left one wins, visible in the copied velocity),
    and a grid of vertical walls only (itopo = 0)."""
    n = 24
    x = 8.0 * np.arange(n)
    y = 8.0 * np.arange(n)
    kw = dict(dt=0.25, h_min=0.125, manning_n2=0.0)
    u = None
    if case == "all_land":
        d = np.full((n, n), -2.0)
        eta = np.full((n, n), 0.5)
        u = np.full((n, n), 0.75)
    elif case == "single_wet_cell":
        d = np.full((n, n), -1.0)
        d[12, 12] = 4.0
        eta = np.zeros((n, n))
        eta[12, 12] = 0.5
    elif case == "exact_threshold":
        d = np.full((n, n), 4.0)
        d[:, 16:] = -0.125
        eta = np.zeros((n, n))
        eta[:, 16] = 0.25                         # h = 0.25 - 0.125 = h_min exactly: wet
    elif case == "flood_tie":
        d = np.full((n, n), 4.0)
        d[:, 12] = -1.0                           # a dry column between two wet ones
        eta = np.full((n, n), 0.5)                # equal eta both sides: eta + d_i = -0.5 ...
        d[:, 12] = 0.0                            # ... make it floodable: eta_j + d_i = 0.5 > h_min
        eta[:, 12] = -0.5                         # dry: h = -0.5 < h_min
        u = np.zeros((n, n))
        u[:, 11] = 0.25                           # left neighbour moves right, right one left
        u[:, 13] = -0.5
    else:                                         # walls only
        d = np.full((n, n), 2.0)
        eta = 0.25 * np.ones((n, n))
        kw.update(itopo=0, dwall=3.0)
    st, o = _run_pair(x, y, d, eta, 6, u, **kw)
    for a, b in zip(st, (o["eta"], o["u"], o["v"])):
        assert np.allclose(a, b, rtol=0, atol=1e-6), np.abs(a - b).max()
    if case == "all_land" or case == "walls_only":
        assert np.array_equal(st[0], eta.astype(np.float32)) and not st[1].any() and not st[2].any()
    if case == "flood_tie":
        s1, o1 = _run_pair(x, y, d, eta, 1, u, **dict(kw))
        assert np.all(o1["u"][:, 12] != 0.0)     # the flooded column took a neighbour's velocity
        assert np.allclose(s1[1][:, 12], o1["u"][:, 12], rtol=0, atol=1e-6)
