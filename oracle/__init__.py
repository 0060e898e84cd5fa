"""FP64 CPU oracle for the Cliffs shallow-water step (arXiv 1410.0753, section "Numerics").

TEST INFRASTRUCTURE ONLY. The tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may call this package; the CUDA library never does, and the two share no code.

The arithmetic lives in ``cliffs_oracle.cpp`` (plain C++, FP64, optional OpenMP over the
independent lines of a sweep). This module compiles it with the host compiler and exposes it
through ctypes:

* ``depth_filter``  - the depth-jump filter (eqs. dstab, newdw, newdc)
* ``sweep_line``    - one 1D sweep of one line with the record of steps (a)-(e)
* ``run``           - time steps with max-wave, gauges and enclosed-grid boundary series
* ``run_tlm``       - the tangent-linear model of ``run`` (branches frozen on the primal), with
  the gauge tangents of eta or of (eta, u, v)
* ``run_forced``    - ``run`` under boundary input on the domain edges
* ``run_tlm_forced`` - the tangent-linear model under boundary input
* ``interp_initial`` - initial conditions from a source grid onto the master grid
``params(..., open_edges=...)`` makes outer edges open (radiating) instead of walls.

Parity status of each part (what pins it) is listed in the tests under ``tests/test_oracle_*``.
The spherical metric (reading 7) is pinned by its Cartesian limit at the equator, the
propagation speed in longitude and the area-weighted volume with the continuity term; the
metric momentum terms, which the paper leaves to another reference, are not modelled, and
that part of its parity is unpinned.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cliffs_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/liboracle.so (host C++ compiler, no CUDA)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
               "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class OracleParams(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("coords", C.c_int32),
                ("h_min", C.c_double), ("manning_n2", C.c_double),
                ("itopo", C.c_int32), ("dwall", C.c_double), ("dt", C.c_double),
                ("transverse", C.c_int32), ("solver", C.c_int32), ("form", C.c_int32),
                ("alternate", C.c_int32), ("open_edges", C.c_int32)]


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = _bind(C.CDLL(_LIB))
    return _lib


def swap_library(path: Optional[str]):
    """Point this module at another build of the oracle source (``None`` restores the
    default). Used only by the tests that plant mistakes in a copy of the oracle."""
    global _lib
    _lib = None if path is None else _bind(C.CDLL(path))


def _bind(L):
    P = C.POINTER
    dp, ip, lp = P(C.c_double), P(C.c_int), P(C.c_long)
    L.oracle_threads.argtypes = [C.c_int]
    L.oracle_threads.restype = C.c_int
    L.oracle_depth_filter.argtypes = [C.c_int, C.c_int, dp, C.c_double, C.c_double, C.c_int]
    L.oracle_depth_filter.restype = C.c_int
    L.oracle_sweep_line.argtypes = [P(OracleParams), C.c_int, dp, dp, dp, dp, dp, dp,
                                    ip, ip, ip, dp, dp, dp, dp, dp, dp]
    L.oracle_sweep_line.restype = C.c_int
    L.oracle_run.argtypes = [P(OracleParams), dp, dp, dp, dp, dp, dp, C.c_long, C.c_long,
                             C.c_int, C.c_int,
                             C.c_int, dp, dp,
                             C.c_int, C.c_int, ip, dp, C.c_long, lp,
                             C.c_int, C.c_int, dp, dp, C.c_long, lp]
    L.oracle_run.restype = C.c_int
    L.oracle_run_tlm.argtypes = [P(OracleParams), dp, dp, dp, dp, dp, dp, dp, dp, dp,
                                 C.c_long, C.c_long, C.c_int,
                                 C.c_int, C.c_int, ip, dp, dp, C.c_long, lp]
    L.oracle_run_tlm.restype = C.c_int
    L.oracle_run_forced.argtypes = [P(OracleParams), dp, dp, dp, dp, dp, dp, C.c_long, C.c_long, C.c_double,
                                    P(dp), lp, P(dp), C.c_int, C.c_int, ip, dp, C.c_long, lp]
    L.oracle_run_forced.restype = C.c_int
    L.oracle_run_tlm_forced.argtypes = [P(OracleParams), dp, dp, dp, dp, dp, dp, dp, dp, dp,
                                        C.c_long, C.c_long, C.c_int, C.c_int, ip, dp, dp, C.c_long, lp,
                                        C.c_double, P(dp), lp, P(dp)]
    L.oracle_run_tlm_forced.restype = C.c_int
    L.oracle_run_tlm_uv.argtypes = [P(OracleParams), dp, dp, dp, dp, dp, dp, dp, dp, dp,
                                    C.c_long, C.c_long, C.c_int, C.c_int, C.c_int, ip, dp, dp, dp, C.c_long, lp]
    L.oracle_run_tlm_uv.restype = C.c_int
    return L


def threads(n: int = 0) -> int:
    """Set (n > 0) and return the number of OpenMP threads the oracle uses."""
    return lib().oracle_threads(int(n))


def _d(a):
    # the C side reads every array in row-major order
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    if a is None:
        return None
    assert a.dtype.itemsize == 4 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_int))


def params(nx, ny, dt, coords=1, h_min=0.01, manning_n2=0.0, itopo=1, dwall=0.0, transverse=1,
           solver=2, form=0, alternate=0, open_edges=0) -> OracleParams:
    """open_edges: bits W 1, E 2, S 4, N 8 mark open (radiating) outer edges; the others are
    reflecting walls."""
    return OracleParams(nx, ny, coords, h_min, manning_n2, itopo, dwall, dt, transverse,
                        solver, form, alternate, open_edges)


def params_from(w, form=0, solver=2, alternate=0, open_edges=0) -> OracleParams:
    return params(w.nx, w.ny, w.dt, w.coords, w.h_min, w.manning_n2, w.itopo, w.dwall,
                  w.transverse, solver, form, alternate, open_edges)


def depth_filter(depth, alpha=2.0, min_depth=0.1, max_passes=100):
    """Return (filtered copy, passes); passes = -1 if the cap was reached."""
    d = np.ascontiguousarray(depth, dtype=np.float64).copy()
    ny, nx = d.shape
    n = lib().oracle_depth_filter(nx, ny, _d(d), float(alpha), float(min_depth), int(max_passes))
    return d, n


def sweep_line(p: OracleParams, ds, d, eta, w, t, src=None):
    """One sweep of one line; returns the final state and the record of steps (a)-(e)."""
    n = len(d)
    ds = np.ascontiguousarray(ds, np.float64)
    d = np.ascontiguousarray(d, np.float64)
    eta = np.array(eta, np.float64, order="C")
    w = np.array(w, np.float64, order="C")
    t = np.array(t, np.float64, order="C")
    src = None if src is None else np.ascontiguousarray(src, np.float64)
    r = {k: np.zeros(n, np.int32) for k in ("wet0", "wet1", "src")}
    r.update({k: np.zeros(n) for k in ("eta_b", "w_b", "t_b", "eta_d", "w_d", "t_d")})
    rc = lib().oracle_sweep_line(C.byref(p), n, _d(ds), _d(d), _d(src), _d(eta), _d(w), _d(t),
                                 _i(r["wet0"]), _i(r["wet1"]), _i(r["src"]),
                                 _d(r["eta_b"]), _d(r["w_b"]), _d(r["t_b"]),
                                 _d(r["eta_d"]), _d(r["w_d"]), _d(r["t_d"]))
    if rc != 0:
        raise ValueError("oracle_sweep_line: bad arguments (%d)" % rc)
    r.update(eta=eta, w=w, t=t)
    return r


def nest_points(nests):
    """Boundary nodes of each enclosed grid, in master coordinates, ordered per nest as
    west (south to north), east, south (west to east), north. Returns (pts[P,2], sizes)
    with sizes[m] = (ny, ny, nx, nx) for the four edges of nest m."""
    pts, sizes = [], []
    for n in nests:
        xs = n.x0 + np.arange(n.nx) * n.dx
        ys = n.y0 + np.arange(n.ny) * n.dy
        xe = n.x0 + (n.nx - 1) * n.dx
        ye = n.y0 + (n.ny - 1) * n.dy
        pts += [(n.x0, yy) for yy in ys]
        pts += [(xe, yy) for yy in ys]
        pts += [(xx, n.y0) for xx in xs]
        pts += [(xx, ye) for xx in xs]
        sizes.append((n.ny, n.ny, n.nx, n.nx))
    return np.array(pts, dtype=np.float64).reshape(-1, 2), sizes


def run(p: OracleParams, x, y, depth, eta, u=None, v=None, nsteps=0, step0=0,
        record_initial=True, fold_final=True, maxout=0, gout=0, gauges=None, bndout=0,
        nests=None, max_records=None):
    """Advance ``nsteps`` steps from step index ``step0`` and return a dict with the final
    state, the max-wave fields, the gauge records [nrec][G][3] (eta, u, v) and, per nest and
    edge, the boundary series [nt][3][np] (u, v, eta)."""
    L = lib()
    ny, nx = depth.shape
    assert (p.nx, p.ny) == (nx, ny)
    x = np.ascontiguousarray(x, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    depth = np.ascontiguousarray(depth, np.float64)
    eta = np.array(eta, np.float64, order="C").reshape(ny, nx)
    u = np.zeros_like(eta) if u is None else np.array(u, np.float64, order="C").reshape(ny, nx)
    v = np.zeros_like(eta) if v is None else np.array(v, np.float64, order="C").reshape(ny, nx)
    nrec_cap = (nsteps + 1) if max_records is None else max_records
    eta_max = speed_max = None
    if maxout > 0:
        eta_max = np.full((ny, nx), -np.finfo(np.float32).max, np.float64)
        speed_max = np.zeros((ny, nx), np.float64)
    G = 0 if gauges is None else len(gauges)
    gix = None
    grec = None
    ng = C.c_long(0)
    if G and gout > 0:
        gix = np.ascontiguousarray(np.asarray(gauges, np.int32).reshape(-1))
        grec = np.zeros((nrec_cap, G, 3))
    pts, sizes = (None, [])
    brec = None
    nb = C.c_long(0)
    NP = 0
    if nests and bndout > 0:
        pts, sizes = nest_points(nests)
        NP = len(pts)
        pts = np.ascontiguousarray(pts.reshape(-1))
        brec = np.zeros((nrec_cap, NP, 3))
    rc = L.oracle_run(C.byref(p), _d(x), _d(y), _d(depth), _d(eta), _d(u), _d(v),
                      int(step0), int(nsteps), int(record_initial), int(fold_final),
                      int(maxout), _d(eta_max), _d(speed_max),
                      int(gout), G if gix is not None else 0, _i(gix), _d(grec), nrec_cap, C.byref(ng),
                      int(bndout), NP, _d(pts), _d(brec), nrec_cap, C.byref(nb))
    if rc != 0:
        raise ValueError("oracle_run failed (%d)" % rc)
    out = dict(eta=eta, u=u, v=v, eta_max=eta_max, speed_max=speed_max)
    out["gauges"] = grec[: ng.value] if grec is not None else None
    if brec is not None:
        series = []
        b = brec[: nb.value]
        o = 0
        for s4 in sizes:
            edges = []
            for npnt in s4:
                edges.append(np.ascontiguousarray(b[:, o:o + npnt, :].transpose(0, 2, 1)))
                o += npnt
            series.append(edges)
        out["boundary"] = series
    return out


def run_forced(p: OracleParams, x, y, depth, eta, boundary, u=None, v=None, nsteps=0, step0=0,
               t0=0.0, gout=1, gauges=None):
    """A run under boundary input: ``boundary`` maps an edge (0 W, 1 E, 2 S, 3 N) to
    (times[nt], vals[nt][3][np]) with vals ordered (u, v, eta); before each step the edge
    nodes take the input at model time t0 + (k - step0) dt. Returns the final state and the
    gauge records [nrec][G][3]."""
    L = lib()
    ny, nx = depth.shape
    x = np.ascontiguousarray(x, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    depth = np.ascontiguousarray(depth, np.float64)
    eta = np.array(eta, np.float64, order="C").reshape(ny, nx)
    u = np.zeros_like(eta) if u is None else np.array(u, np.float64, order="C").reshape(ny, nx)
    v = np.zeros_like(eta) if v is None else np.array(v, np.float64, order="C").reshape(ny, nx)
    keep = []
    tp = (C.POINTER(C.c_double) * 4)()
    vp = (C.POINTER(C.c_double) * 4)()
    nt = (C.c_long * 4)()
    for e in range(4):
        if e in boundary:
            t, vals = boundary[e]
            t = np.ascontiguousarray(t, np.float64)
            vals = np.ascontiguousarray(vals, np.float64)
            npnt = ny if e < 2 else nx
            assert vals.shape == (len(t), 3, npnt), (e, vals.shape)
            keep += [t, vals]
            tp[e], vp[e], nt[e] = _d(t), _d(vals), len(t)
    G = 0 if gauges is None else len(gauges)
    gix = np.ascontiguousarray(np.asarray(gauges, np.int32).reshape(-1)) if G else None
    cap = nsteps + 1
    grec = np.zeros((cap, max(G, 1), 3))
    ng = C.c_long(0)
    rc = L.oracle_run_forced(C.byref(p), _d(x), _d(y), _d(depth), _d(eta), _d(u), _d(v), int(step0),
                             int(nsteps), float(t0), tp, nt, vp, int(gout), G, _i(gix), _d(grec), cap,
                             C.byref(ng))
    if rc != 0:
        raise ValueError("oracle_run_forced failed (%d)" % rc)
    return dict(eta=eta, u=u, v=v, gauges=grec[: ng.value, :G] if G else None)


def interp_initial(mx, my, sx, sy, field):
    """Initial conditions from a source grid (section "Running Options", "The input to the
    computations"): on master nodes inside the source grid the bilinear interpolation of the
    four surrounding source nodes, zero outside. A source dimension of one node covers only
    master nodes at exactly its coordinate."""
    mx, my, sx, sy = (np.asarray(a, np.float64) for a in (mx, my, sx, sy))
    field = np.asarray(field, np.float64).reshape(len(sy), len(sx))
    out = np.zeros((len(my), len(mx)))

    def cell(c, xp):
        if len(c) == 1:
            return (0, 0.0) if xp == c[0] else None
        if xp < c[0] or xp > c[-1]:
            return None
        k = int(np.searchsorted(c, xp, side="right")) - 1
        k = min(max(k, 0), len(c) - 2)
        return k, (xp - c[k]) / (c[k + 1] - c[k])

    for r, yp in enumerate(my):
        cr = cell(sy, yp)
        if cr is None:
            continue
        j, b = cr
        j1 = j + 1 if b > 0 else j
        for c_, xp in enumerate(mx):
            cc = cell(sx, xp)
            if cc is None:
                continue
            i, a = cc
            i1 = i + 1 if a > 0 else i
            out[r, c_] = ((1 - b) * ((1 - a) * field[j, i] + a * field[j, i1]) +
                          b * ((1 - a) * field[j1, i] + a * field[j1, i1]))
    return out


def run_tlm_forced(p: OracleParams, x, y, depth, eta, deta, boundary, nsteps=0, t0=0.0, gout=1, gauges=None):
    """Tangent-linear run under boundary input (see ``run_forced``): the imposed edge values
    carry no tangent. Returns (gauge values [nrec][G], gauge tangents [nrec][G])."""
    L = lib()
    ny, nx = depth.shape
    x = np.ascontiguousarray(x, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    depth = np.ascontiguousarray(depth, np.float64)
    eta = np.array(eta, np.float64, order="C").reshape(ny, nx)
    deta = np.array(deta, np.float64, order="C").reshape(ny, nx)
    z = [np.zeros_like(eta) for _ in range(4)]
    keep = []
    tp = (C.POINTER(C.c_double) * 4)()
    vp = (C.POINTER(C.c_double) * 4)()
    nt = (C.c_long * 4)()
    for e in range(4):
        if e in boundary:
            t, vals = boundary[e]
            t = np.ascontiguousarray(t, np.float64)
            vals = np.ascontiguousarray(vals, np.float64)
            keep += [t, vals]
            tp[e], vp[e], nt[e] = _d(t), _d(vals), len(t)
    gix = np.ascontiguousarray(np.asarray(gauges, np.int32).reshape(-1))
    G = len(gix) // 2
    cap = nsteps + 1
    gval = np.zeros((cap, G))
    gtan = np.zeros((cap, G))
    n = C.c_long(0)
    rc = L.oracle_run_tlm_forced(C.byref(p), _d(x), _d(y), _d(depth), _d(eta), _d(z[0]), _d(z[1]), _d(deta),
                                 _d(z[2]), _d(z[3]), 0, int(nsteps), int(gout), G, _i(gix), _d(gval), _d(gtan),
                                 cap, C.byref(n), float(t0), tp, nt, vp)
    if rc != 0:
        raise ValueError("oracle_run_tlm_forced failed (%d)" % rc)
    return gval[: n.value], gtan[: n.value]


def run_tlm(p: OracleParams, x, y, depth, eta, deta, u=None, v=None, du=None, dv=None,
            nsteps=0, step0=0, record_initial=True, gout=1, gauges=None, uv=False):
    """Tangent-linear run. Returns (gauge values [nrec][G], gauge tangents [nrec][G],
    final primal state, final tangent state); with uv=True the gauge tangents are those of
    (eta, u, v), [nrec][G][3]."""
    L = lib()
    ny, nx = depth.shape
    x = np.ascontiguousarray(x, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    depth = np.ascontiguousarray(depth, np.float64)
    eta = np.array(eta, np.float64, order="C").reshape(ny, nx)
    deta = np.array(deta, np.float64, order="C").reshape(ny, nx)
    z = np.zeros_like(eta)
    u = z.copy() if u is None else np.array(u, np.float64, order="C").reshape(ny, nx)
    v = z.copy() if v is None else np.array(v, np.float64, order="C").reshape(ny, nx)
    du = z.copy() if du is None else np.array(du, np.float64, order="C").reshape(ny, nx)
    dv = z.copy() if dv is None else np.array(dv, np.float64, order="C").reshape(ny, nx)
    gix = np.ascontiguousarray(np.asarray(gauges, np.int32).reshape(-1))
    G = len(gix) // 2
    cap = nsteps + 1
    gval = np.zeros((cap, G))
    gtan = np.zeros((cap, G))
    n = C.c_long(0)
    if uv:
        guv = np.zeros((cap, G, 2))
        rc = L.oracle_run_tlm_uv(C.byref(p), _d(x), _d(y), _d(depth), _d(eta), _d(u), _d(v),
                                 _d(deta), _d(du), _d(dv), int(step0), int(nsteps), int(record_initial),
                                 int(gout), G, _i(gix), _d(gval), _d(gtan), _d(guv), cap, C.byref(n))
        gtan = np.concatenate([gtan[:, :, None], guv], axis=2)
    else:
        rc = L.oracle_run_tlm(C.byref(p), _d(x), _d(y), _d(depth), _d(eta), _d(u), _d(v),
                              _d(deta), _d(du), _d(dv), int(step0), int(nsteps), int(record_initial),
                              int(gout), G, _i(gix), _d(gval), _d(gtan), cap, C.byref(n))
    if rc != 0:
        raise ValueError("oracle_run_tlm failed (%d)" % rc)
    return gval[: n.value], gtan[: n.value], (eta, u, v), (deta, du, dv)


def run_workload(w, nsteps=None, form=0, solver=2, alternate=0, filtered_depth=None,
                 scenario=None, record=True):
    """Run a ``workloads.Workload`` from its initial state: filter the depth (unless a
    filtered depth is given), then step with the workload's outputs."""
    depth = filtered_depth
    if depth is None:
        depth, _ = depth_filter(w.depth, w.filter_alpha, w.filter_min_depth)
    eta0 = w.eta0 if w.eta0.ndim == 2 else w.eta0[scenario or 0]
    p = params_from(w, form=form, solver=solver, alternate=alternate)
    n = w.steps if nsteps is None else nsteps
    return run(p, w.x, w.y, depth, eta0, w.u0, w.v0, nsteps=n,
               maxout=w.maxout if record else 0, gout=w.gout if record else 0,
               gauges=w.gauges if record else None, bndout=w.bndout if record else 0,
               nests=w.nests if record else None)


def quake_init(depth, zeta, h_min, itopo=1, dwall=0.0):
    """Parameter-file field 12, quake = 1: the sea-floor deformation zeta lifts the bottom,
    d <- d - zeta, and the free surface with it on nodes that were wet (d >= h_min and, when
    itopo = 0, not a wall): eta <- zeta there, 0 elsewhere."""
    depth = np.asarray(depth, np.float64)
    zeta = np.asarray(zeta, np.float64)
    wet = (depth >= h_min) & ((itopo != 0) | (depth >= dwall))
    return depth - zeta, np.where(wet, zeta, 0.0)
