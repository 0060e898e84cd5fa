"""Open (radiating) outer edges on the GPU against the FP64 oracle.

The paper gives no condition for an open edge; the reading (the ghost beyond a wet edge node
carries the node's outgoing Riemann invariant and still water's incoming one) is the
oracle's, pinned there by an outgoing simple wave, a draining raised level and a radial wave
leaving a square. Here the fused, persistent and 1D kernels with open edges are checked
against it with the tolerances of test_gpu_parity.py: gauge traces within 1e-4 of the
oracle's max|eta| (1e-7 m absolute below 1e-3 m), wet masks equal except near round-off.
"""
import numpy as np
import pytest

import oracle
import workloads
from paper_1410_0753_gb300 import CliffsError, CliffsGrid, ERR_ARG
from tests import parity as P

pytestmark = pytest.mark.gpu


def _basin(nx, ny):
    """Water of 30 m falling to a beach along the south edge (dry there), an island, one hump
    by the NW corner and one by the east edge: waves cross the W, N and E edges."""
    x, y = 100.0 * np.arange(nx), 100.0 * np.arange(ny)
    X, Y = np.meshgrid(x, y)
    d = 30.0 - 34.0 * np.clip((0.25 * y[-1] - Y) / (0.25 * y[-1]), 0.0, 1.0)
    d = d - 35.0 * np.exp(-((X - 0.5 * x[-1]) ** 2 + (Y - 0.5 * y[-1]) ** 2) / (2 * 600.0 ** 2))
    eta0 = 0.6 * np.exp(-((X - 0.25 * x[-1]) ** 2 + (Y - 0.7 * y[-1]) ** 2) / (2 * 900.0 ** 2)) + \
        0.4 * np.exp(-((X - 0.85 * x[-1]) ** 2 + (Y - 0.55 * y[-1]) ** 2) / (2 * 700.0 ** 2))
    gauges = [(0, int(0.65 * ny)), (2, int(0.6 * ny)), (nx // 4, ny - 1), (nx - 1, ny // 2), (nx - 2, int(0.6 * ny)),
              (nx // 2, ny - 2), (nx // 2, ny // 5), (nx // 2, int(0.7 * ny))]
    return x, y, P.f32(d), eta0, np.array(gauges, np.int32)


def _run(x, y, d64, eta0, gauges, steps, dt, **kw):
    nx, ny = len(x), len(y)
    opts = dict(h_min=0.01, manning_n2=6.25e-4)
    opts.update({k: v for k, v in kw.items() if k in ("h_min", "manning_n2", "coords")})
    g = CliffsGrid(nx, ny, dt, gauges=[tuple(q) for q in gauges], open_edges=kw.get("open_edges", 15),
                   solver=kw.get("solver", 2), alternate=kw.get("alternate", 0), **opts)
    g.set_bathy(x, y, d64, False)
    g.set_initial(eta0.astype(np.float32))
    g.step(steps)
    p = oracle.params(nx, ny, dt, opts.get("coords", 1), opts["h_min"], opts["manning_n2"],
                      solver=kw.get("solver", 2), alternate=kw.get("alternate", 0),
                      open_edges=kw.get("open_edges", 15))
    o = oracle.run(p, x, y, d64, eta0, nsteps=steps, gout=1, gauges=gauges)
    return g, o


def _check(name, g, o, d64, amp, hmin=0.01):
    rel, absol = P.gauge_errors(g.gauges()[:, :, 0], o["gauges"][:, :, 0])
    P.report(name, gauge_rel_max=rel.max(initial=0.0), gauge_abs_max=absol.max(initial=0.0))
    assert rel.max(initial=0.0) <= P.GAUGE_RTOL, rel
    assert absol.max(initial=0.0) <= P.GAUGE_ATOL_SMALL, absol
    e32, u32, v32 = g.state()
    wet32, wet64, near = P.wet_masks(e32, o["eta"], d64, d64, hmin)
    assert np.array_equal(wet32 & ~near, wet64 & ~near)
    assert np.abs(e32 - o["eta"])[wet64].max() <= 1e-4 * amp
    assert np.abs(u32 - o["u"])[wet64].max() <= 1e-4 * np.abs(o["u"]).max() + 1e-7
    assert np.abs(v32 - o["v"])[wet64].max() <= 1e-4 * np.abs(o["v"]).max() + 1e-7


@pytest.mark.parametrize("nx", [150, 151])           # the east edge in node B, then node A, of its lane
@pytest.mark.parametrize("variant", ["solver2", "solver1", "alternate"])
def test_open_edges_against_oracle(nx, variant):
    x, y, d64, eta0, gauges = _basin(nx, 128)
    kw = {"solver1": dict(solver=1), "alternate": dict(alternate=1)}.get(variant, {})
    g, o = _run(x, y, d64, eta0, gauges, 260, 1.0, **kw)
    # the wave has reached the open edges: something went out through them
    assert min(np.abs(o["gauges"][:, k, 0]).max() for k in (0, 2, 3)) > 1e-2   # W, N and E edge nodes
    _check("open_%s_%d" % (variant, nx), g, o, d64, 0.6)
    g.close()


def test_open_edges_spherical_coast():
    w = workloads.spherical_coast(220, 190, steps=160)
    d64 = P.f32(P.oracle_depth(w))
    g, o = _run(w.x, w.y, d64, w.eta0, w.gauges, w.steps, w.dt, coords=w.coords, h_min=w.h_min,
                manning_n2=w.manning_n2)
    _check("open_spherical", g, o, d64, np.abs(w.eta0).max(), w.h_min)
    g.close()


@pytest.mark.parametrize("axis", ["x", "y"])
def test_open_edges_1d_lines(axis):
    """A right-going wave leaving a flat channel through its open far end, on the 1D x and y
    kernels; the state against the oracle, and almost nothing left behind."""
    n, dx, d0 = 300, 50.0, 10.0
    s = dx * np.arange(n)
    c0 = np.sqrt(9.81 * d0)
    eta = 0.05 * np.exp(-((s - 6000.0) ** 2) / (2 * 700.0 ** 2))
    vel = eta * c0 / d0
    dt = 0.5 * dx / c0
    steps = int((s[-1] - 6000.0 + 4200.0) / c0 / dt)
    if axis == "x":
        nx, ny, x, y, d, e0, u0, v0, edges = n, 1, s, np.zeros(1), np.full((1, n), d0), eta[None, :], vel[None, :], None, 3
    else:
        nx, ny, x, y, d, e0, u0, v0, edges = 1, n, np.zeros(1), s, np.full((n, 1), d0), eta[:, None], None, vel[:, None], 12
    g = CliffsGrid(nx, ny, dt, manning_n2=0.0, open_edges=edges)
    g.set_bathy(x, y, d, False)
    g.set_initial(e0.astype(np.float32), None if u0 is None else u0.astype(np.float32),
                  None if v0 is None else v0.astype(np.float32))
    g.step(steps)
    o = oracle.run(oracle.params(nx, ny, dt, manning_n2=0.0, open_edges=edges), x, y, d, e0, u0, v0, nsteps=steps)
    e32 = g.state()[0]
    assert np.abs(e32 - o["eta"]).max() <= 1e-4 * 0.05
    assert np.abs(e32).max() < 0.01 * 0.05
    g.close()


def test_open_edges_keep_a_lake_at_rest_exactly():
    x, y, d64, _, gauges = _basin(150, 128)
    g = CliffsGrid(150, 128, 1.0, h_min=0.01, manning_n2=6.25e-4, open_edges=15)
    g.set_bathy(x, y, d64, False)
    g.set_initial(np.zeros((128, 150), np.float32))
    g.step(50)
    e, u, v = g.state()
    assert not e.any() and not u.any() and not v.any()
    g.close()


def test_open_edges_persistent_run_equals_per_step():
    w = workloads.ensemble_512(batch=4, nx=120, ny=100, dmin=20, dmax=60)
    runs = []
    for pers in (False, True):
        g = CliffsGrid.from_workload(w, open_edges=15)
        g.set_bathy(w.x, w.y, w.depth, True, w.filter_alpha, w.filter_min_depth)
        g.set_initial(w.eta0.astype(np.float32))
        g.set_durations(w.durations)
        g.step(int(w.durations.max()), persistent=pers)
        runs.append([g.state(b) for b in range(w.batch)])
        g.close()
    for a, b in zip(runs[0], runs[1]):
        for p, q in zip(a, b):
            assert np.array_equal(p, q)
    # and the open edges did something: the same run with walls differs
    g = CliffsGrid.from_workload(w)
    g.set_bathy(w.x, w.y, w.depth, True, w.filter_alpha, w.filter_min_depth)
    g.set_initial(w.eta0.astype(np.float32))
    g.set_durations(w.durations)
    g.step(int(w.durations.max()))
    assert not np.array_equal(g.state(0)[0], runs[0][0][0])
    g.close()


def test_open_edges_argument_checks():
    with pytest.raises(CliffsError) as e:
        CliffsGrid(40, 30, 1.0, open_edges=16)
    assert e.value.code == ERR_ARG
    with pytest.raises(CliffsError) as e:
        CliffsGrid(40, 30, 1.0, open_edges=-1)
    assert e.value.code == ERR_ARG


@pytest.mark.parametrize("variant", ["solver2", "solver1", "alternate"])
def test_adjoint_with_open_edges_dot_product_against_oracle_tlm(variant):
    """<dL/d eta0, delta> from the GPU adjoint against the oracle's tangent model through the
    open ghosts (1e-4 of the largest term, as in test_gpu_adjoint.py), gauges on the W, N and
    E edge nodes and inside, directions that reach the edges."""
    nx, ny, steps = 150, 128, 200
    x, y, d64, eta0, gauges = _basin(nx, ny)
    kw = {"solver1": dict(solver=1), "alternate": dict(alternate=1)}.get(variant, {})
    g = CliffsGrid(nx, ny, 1.0, h_min=0.01, manning_n2=6.25e-4, gauges=[tuple(q) for q in gauges],
                   open_edges=15, **kw)
    g.set_bathy(x, y, d64, False)
    g.set_initial(eta0.astype(np.float32))
    rng = np.random.default_rng(29)
    seed = rng.standard_normal((steps + 1, len(gauges))).astype(np.float32)
    grad = g.adjoint(steps, seed, checkpoint_every=37).astype(np.float64)
    assert np.isfinite(grad).all()
    p = oracle.params(nx, ny, 1.0, h_min=0.01, manning_n2=6.25e-4, open_edges=15, **kw)
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    worst = 0.0
    for k, (cx, cy, sig) in enumerate(((8.0, 85.0, 10.0), (40.0, 120.0, 9.0), (140.0, 70.0, 10.0), (75.0, 64.0, 30.0))):
        delta = np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * sig ** 2))
        if k == 3:
            delta = delta + 0.1 * rng.standard_normal(delta.shape)
        _, gtan, _, _ = oracle.run_tlm(p, x, y, d64, eta0, delta, nsteps=steps, gauges=gauges)
        terms = seed.astype(np.float64) * gtan
        want = terms.sum()
        got = float((grad * delta).sum())
        scale = max(np.abs(terms).max(), 1e-12)
        err = abs(got - want) / scale
        worst = max(worst, err)
        assert err <= 1e-4, (variant, k, got, want, scale)
    P.report("adjoint_dot_open_" + variant, rel_err=worst)
    g.close()
