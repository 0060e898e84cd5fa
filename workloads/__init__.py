"""Seeded synthetic workloads for the shallow-water step (bathymetry, sources, gauges, nests).

This module is the one piece shared by the CUDA path's tests/bench and the FP64 oracle's
tests. It holds none of the method's arithmetic: no sweep, no depth filter, no output
recording. It only draws inputs.

The paper's own data (the Okushiri grids, the Synolakis beach files) are not available, so
these generators stand in for them, on the scales the paper's examples use (30 arc-second
/ ~930 m grids, metre-scale sources, Manning n^2 of order 1e-3, cadences of 1-500 steps;
Examples section, Tables 1-6). Every array is seeded from ``default_rng(SEED + k)`` for
workload k, and every floating-point input is rounded to an FP32-representable value
(stored as float64) so that the FP32 device path and the FP64 oracle read identical inputs.

Layout conventions (Running Options, "Netcdf structure"): 2D fields are ``[ny][nx]`` with
x (longitude) fastest; batched fields are ``[B][ny][nx]``. Gauge indices are 0-based
``(ix, iy)`` pairs (the paper's parameter file uses 1-based node numbers).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

G = 9.81                 # gravity, m s^-2
R_EARTH = 6371000.0      # sphere radius used for geographic grids, m
SEED = 14100753


def f32(a):
    """Round to FP32-representable values, keep float64 storage."""
    return np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float64)


@dataclass
class Nest:
    """An enclosed (nested) grid given in master coordinates: uniform spacing (dx, dy)."""
    x0: float
    y0: float
    dx: float
    dy: float
    nx: int
    ny: int


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    coords: int                      # 1 = Cartesian, otherwise geographic spherical
    x: np.ndarray                    # [nx] node x (m) or longitude (deg)
    y: np.ndarray                    # [ny] node y (m) or latitude (deg)
    depth: np.ndarray                # [ny][nx] undisturbed depth, positive down (m)
    eta0: np.ndarray                 # [ny][nx] or [B][ny][nx] initial free surface (m)
    dt: float
    steps: int
    u0: Optional[np.ndarray] = None
    v0: Optional[np.ndarray] = None
    h_min: float = 0.01              # 'ground', minimal flow depth
    manning_n2: float = 0.025 ** 2   # 'crough'
    itopo: int = 1
    dwall: float = 0.0
    transverse: int = 1
    maxout: int = 1
    gout: int = 1
    bndout: int = 1
    gauges: np.ndarray = field(default_factory=lambda: np.zeros((0, 2), np.int32))
    nests: List[Nest] = field(default_factory=list)
    durations: Optional[np.ndarray] = None   # [B] steps per scenario (batched form)
    filter_alpha: float = 2.0
    filter_min_depth: float = 0.1
    extra: dict = field(default_factory=dict)

    @property
    def batch(self) -> int:
        return 1 if self.eta0.ndim == 2 else self.eta0.shape[0]

    @property
    def cells(self) -> int:
        return self.nx * self.ny


# --------------------------------------------------------------------------- noise

def fractal_noise_2d(shape, rng, beta=3.0):
    """White Gaussian noise filtered to a power spectrum P(k) ~ |k|^-beta;
    zero mean, unit standard deviation, clipped at +-3."""
    ny, nx = shape
    w = rng.standard_normal((ny, nx))
    W = np.fft.rfft2(w)
    ky = np.fft.fftfreq(ny)[:, None]
    kx = np.fft.rfftfreq(nx)[None, :]
    k = np.sqrt(kx * kx + ky * ky)
    k[0, 0] = np.inf
    W *= k ** (-beta / 2.0)
    n = np.fft.irfft2(W, s=(ny, nx))
    n -= n.mean()
    n /= n.std()
    np.clip(n, -3.0, 3.0, out=n)
    return n


def fractal_noise_1d(n, rng, beta=3.0):
    w = rng.standard_normal(n)
    W = np.fft.rfft(w)
    k = np.fft.rfftfreq(n)
    k[0] = np.inf
    W *= k ** (-beta / 2.0)
    s = np.fft.irfft(W, n=n)
    s -= s.mean()
    s /= max(np.abs(s).max(), 1e-300)
    return s                                   # max |s| = 1


def cfl_dt(cfl, ds_min, dmax):
    return cfl * ds_min / math.sqrt(G * dmax)


# --------------------------------------------------------------------------- config 1

def beach_200(nx=200, ny=200, steps=1000):
    """2D Cartesian beach: dx = dy = 100 m; 50 m offshore for x <= 10 km, then a plane beach
    rising to +10 m dry land at x = 19.9 km (the shoreline near i = 182.5). A 0.5 m Gaussian
    hump (sigma 1.5 km) at the grid centre, zero velocity, CFL 0.5, Manning n = 0.025,
    reflective outer walls, 8 gauges on row ny/2 running toward the shore."""
    dx = 100.0
    x = np.arange(nx) * dx
    y = np.arange(ny) * dx
    xmax = (200 - 1) * dx
    d1 = np.where(x <= 10000.0, 50.0, 50.0 - 60.0 * (x - 10000.0) / (xmax - 10000.0))
    depth = np.broadcast_to(d1[None, :], (ny, nx)).copy()
    xc, yc = 0.5 * (nx - 1) * dx, 0.5 * (ny - 1) * dx
    X, Y = np.meshgrid(x, y)
    eta0 = 0.5 * np.exp(-((X - xc) ** 2 + (Y - yc) ** 2) / (2 * 1500.0 ** 2))
    gx = np.clip(np.round(np.linspace(0.5 * nx, 0.885 * nx, 8)).astype(np.int32), 0, nx - 1)
    gauges = np.stack([gx, np.full(8, ny // 2, np.int32)], axis=1).astype(np.int32)
    dt = cfl_dt(0.5, dx, 50.0)
    return Workload("beach_200", nx, ny, 1, f32(x), f32(y), f32(depth), f32(eta0), dt, steps,
                    gauges=gauges, maxout=1, gout=1, bndout=1)


# --------------------------------------------------------------------------- config 2

def spherical_coast(nx=2048, ny=2048, steps=3600, seed_offset=2):
    """Geographic grid at 1 arc-minute: lon 140 + i/60, lat 20 + j/60. A meandering coast at
    ix_c(j) = nx/8 + (nx/32) sin(2 pi j/(ny/2)) plus a fractal meander of +-nx/128 cells; land
    rising 0.5 m/km to +50 m; a 0-5 km ramp to a 150 m shelf out to 80 km; a slope to a
    4000 m plain at 180 km; all times (1 + 0.05 N) with fractal noise N. Source: a 2 m
    elliptical Gaussian (300 x 100 km taken as 4 sigma), rotated 30 deg CCW from east,
    centred on row ny/2 at 150 km offshore. 64 gauges, max-wave every step, four enclosed
    grids at 20 arc-seconds straddling the coast, boundary series every step; CFL 0.8."""
    rng = np.random.default_rng(SEED + seed_offset)
    lon = 140.0 + np.arange(nx) / 60.0
    lat = 20.0 + np.arange(ny) / 60.0
    sc = nx / 2048.0
    j = np.arange(ny)
    meander = fractal_noise_1d(ny, rng)
    ixc = 256.0 * sc + 64.0 * sc * np.sin(2 * np.pi * j / (1024.0 * ny / 2048.0)) + 16.0 * sc * meander
    dxrow = R_EARTH * np.cos(np.radians(lat)) * np.radians(1.0 / 60.0)     # m per cell along a row
    s_km = (np.arange(nx)[None, :] - ixc[:, None]) * dxrow[:, None] / 1000.0
    d = np.empty((ny, nx))
    land = s_km < 0
    d[land] = -np.minimum(0.5 * -s_km[land], 50.0)
    m = (s_km >= 0) & (s_km < 5)
    d[m] = 150.0 * s_km[m] / 5.0
    m = (s_km >= 5) & (s_km < 80)
    d[m] = 150.0
    m = (s_km >= 80) & (s_km < 180)
    d[m] = 150.0 + (4000.0 - 150.0) * (s_km[m] - 80.0) / 100.0
    d[s_km >= 180] = 4000.0
    noise = fractal_noise_2d((ny, nx), rng)
    d *= 1.0 + 0.05 * noise
    # source
    jc = ny // 2
    latc = lat[jc]
    lonc = lon[0] + (ixc[jc] + 150.0e3 / dxrow[jc]) / 60.0
    LON, LAT = np.meshgrid(lon, lat)
    ex = np.radians(LON - lonc) * R_EARTH * np.cos(np.radians(latc))
    ey = np.radians(LAT - latc) * R_EARTH
    th = np.radians(30.0)
    a = ex * math.cos(th) + ey * math.sin(th)
    b = -ex * math.sin(th) + ey * math.cos(th)
    eta0 = 2.0 * np.exp(-a * a / (2 * 75.0e3 ** 2) - b * b / (2 * 25.0e3 ** 2))
    # gauges: 8 rows x 8 offshore distances
    rows = (np.array([128 + 256 * k for k in range(8)]) * ny / 2048.0).astype(int)
    dists = [2, 10, 30, 60, 100, 150, 250, 400]
    gl = []
    for r in rows:
        for s in dists:
            ix = int(round(ixc[r] + s * 1000.0 / dxrow[r]))
            gl.append((min(max(ix, 0), nx - 1), r))
    gauges = np.array(gl, dtype=np.int32)
    # nests: 20 arc-second grids, 100 master cells across (scaled), centred on the coast
    nn = max(31, int(round(300 * sc)) + 1)
    span = (nn - 1) / 180.0
    nests = []
    for r in (np.array([256, 768, 1280, 1792]) * ny / 2048.0).astype(int):
        lc = lon[0] + ixc[r] / 60.0
        y0 = min(max(lat[r] - span / 2, lat[0]), lat[-1] - span)
        x0 = min(max(lc - span / 2, lon[0]), lon[-1] - span)
        nests.append(Nest(x0, y0, 1.0 / 180.0, 1.0 / 180.0, nn, nn))
    dsmin = R_EARTH * math.cos(math.radians(lat[-1])) * math.radians(1.0 / 60.0)
    dt = cfl_dt(0.8, dsmin, float(d.max()))
    return Workload("spherical_coast_%dx%d" % (nx, ny), nx, ny, 0, f32(lon), f32(lat), f32(d),
                    f32(eta0), dt, steps, gauges=gauges, nests=nests, maxout=1, gout=1, bndout=1)


# --------------------------------------------------------------------------- config 3

def shelf_islands(nx=8192, ny=8192, steps=2000, seed_offset=3, maxout=None):
    """Cartesian 50 m grid: a 200 m shelf times (1 + 0.02 N) with 10 conical islands (centres
    uniform in [0.3 L, 0.95 L]^2, base radius 1-5 km, summit 20-80 m above sea level), so the
    domain carries several wet/dry shorelines; an N-wave line source with +1 m peak,
    x0 = 40 km (scaled with the domain), L = 3 km; CFL 0.8."""
    rng = np.random.default_rng(SEED + seed_offset)
    dx = 50.0
    x = np.arange(nx) * dx
    y = np.arange(ny) * dx
    Lx, Ly = (nx - 1) * dx, (ny - 1) * dx
    noise = fractal_noise_2d((ny, nx), rng)
    d = 200.0 * (1.0 + 0.02 * noise)
    sc = nx / 8192.0
    for _ in range(10):
        cx = rng.uniform(0.3, 0.95) * Lx
        cy = rng.uniform(0.3, 0.95) * Ly
        rb = rng.uniform(1.0e3, 5.0e3) * max(sc, 0.05)
        top = rng.uniform(20.0, 80.0)
        i0, i1 = max(0, int((cx - rb) / dx) - 1), min(nx, int((cx + rb) / dx) + 2)
        j0, j1 = max(0, int((cy - rb) / dx) - 1), min(ny, int((cy + rb) / dx) + 2)
        if i0 >= i1 or j0 >= j1:
            continue
        XX, YY = np.meshgrid(x[i0:i1], y[j0:j1])
        r = np.sqrt((XX - cx) ** 2 + (YY - cy) ** 2)
        cone = -top + (200.0 + top) * r / rb
        d[j0:j1, i0:i1] = np.minimum(d[j0:j1, i0:i1], cone)
    x0 = 40.0e3 * sc
    Ln = 3.0e3 * max(sc, 0.05)
    s = (x - x0) / Ln
    eta1 = s * np.exp(0.5 - 0.5 * s * s)
    eta0 = np.broadcast_to(eta1[None, :], (ny, nx)).copy()
    dt = cfl_dt(0.8, dx, float(d.max()))
    mo = steps + 1 if maxout is None else maxout
    return Workload("shelf_islands_%dx%d" % (nx, ny), nx, ny, 1, f32(x), f32(y), f32(d),
                    f32(eta0), dt, steps, maxout=mo, gout=steps + 1, bndout=steps + 1)


# --------------------------------------------------------------------------- config 4

def basin_slope_depth(x, xs_deep, xs_shore, d0, land_top):
    """Constant depth d0 to xs_deep, linear to 0 at xs_shore, then land rising linearly to
    land_top (m above sea level) at the last node."""
    xe = x[-1]
    d = np.where(x <= xs_deep, d0, d0 * (xs_shore - x) / (xs_shore - xs_deep))
    land = x > xs_shore
    if xe > xs_shore:
        d = np.where(land, -land_top * (x - xs_shore) / (xe - xs_shore), d)
    return d


def ensemble_512(batch=256, nx=512, ny=512, seed_offset=4, dmin=500, dmax=4000):
    """256 scenarios on one shared Cartesian 200 m bathymetry (3000 m to x = 50 km, linear to
    0 at 95 km, land up to +20 m at the east edge); each scenario a 1 m Gaussian with sigma
    uniform in 5-20 km centred uniformly in [10,60] x [10,92] km (scaled to the domain);
    durations uniform in {500..4000} steps; 16 shared gauges on a 4 x 4 lattice."""
    rng = np.random.default_rng(SEED + seed_offset)
    dx = 200.0
    sx, sy = nx / 512.0, ny / 512.0
    x = np.arange(nx) * dx
    y = np.arange(ny) * dx
    d1 = basin_slope_depth(x, 50.0e3 * sx, 95.0e3 * sx, 3000.0, 20.0)
    depth = np.broadcast_to(d1[None, :], (ny, nx)).copy()
    X, Y = np.meshgrid(x, y)
    eta0 = np.empty((batch, ny, nx))
    sig = rng.uniform(5.0e3, 20.0e3, batch) * min(sx, sy)
    cx = rng.uniform(10.0e3, 60.0e3, batch) * sx
    cy = rng.uniform(10.0e3, 92.0e3, batch) * sy
    for b in range(batch):
        eta0[b] = np.exp(-((X - cx[b]) ** 2 + (Y - cy[b]) ** 2) / (2 * sig[b] ** 2))
    durations = rng.integers(dmin, dmax + 1, batch).astype(np.int64)
    gx = (np.array([55.0e3, 65.0e3, 75.0e3, 85.0e3]) * sx / dx).astype(np.int32)
    gy = (np.array([20.0e3, 40.0e3, 60.0e3, 80.0e3]) * sy / dx).astype(np.int32)
    gauges = np.array([(a, b) for b in gy for a in gx], dtype=np.int32)
    dt = cfl_dt(0.8, dx, 3000.0)
    return Workload("ensemble_%dx%dx%d" % (batch, nx, ny), nx, ny, 1, f32(x), f32(y), f32(depth),
                    f32(eta0), dt, int(durations.max()), gauges=gauges, durations=durations,
                    maxout=int(durations.max()) + 1, gout=1, bndout=int(durations.max()) + 1)


# --------------------------------------------------------------------------- config 5

def unit_sources(nx, ny, dx, sx=1.0, sy=1.0):
    """64 unit Gaussians (sigma 8 km) on an 8 x 8 lattice, x = 20..160 km, y = 32..256 km."""
    xs = np.array([20.0e3 + 20.0e3 * k for k in range(8)]) * sx
    ys = np.array([32.0e3 + 32.0e3 * k for k in range(8)]) * sy
    cx = np.array([a for b in ys for a in xs])
    cy = np.array([b for b in ys for a in xs])
    sig = np.full(64, 8.0e3 * min(sx, sy))
    return cx, cy, sig


def gaussian_basis(x, y, cx, cy, sig):
    X, Y = np.meshgrid(x, y)
    return np.stack([np.exp(-((X - cx[k]) ** 2 + (Y - cy[k]) ** 2) / (2 * sig[k] ** 2))
                     for k in range(len(cx))])


def inversion_1024(nx=1024, ny=1024, steps=2000, seed_offset=5):
    """Source inversion: Cartesian 250 m grid, 2000 m to x = 120 km, linear to 0 at 240 km,
    land up to +20 m at the east edge. eta0 = sum_k theta_k G_k over 64 unit Gaussians;
    truth theta* ~ N(0, 0.5^2) (seed + 100); evaluation point theta0 = theta* + N(0, 0.25^2)
    (seed + 200). 32 gauges at x = 180 and 220 km by 16 y positions, every step."""
    dx = 250.0
    sx, sy = nx / 1024.0, ny / 1024.0
    x = np.arange(nx) * dx
    y = np.arange(ny) * dx
    d1 = basin_slope_depth(x, 120.0e3 * sx, 240.0e3 * sx, 2000.0, 20.0)
    depth = np.broadcast_to(d1[None, :], (ny, nx)).copy()
    cx, cy, sig = unit_sources(nx, ny, dx, sx, sy)
    theta_true = np.random.default_rng(SEED + seed_offset + 100).normal(0.0, 0.5, 64)
    theta0 = theta_true + np.random.default_rng(SEED + seed_offset + 200).normal(0.0, 0.25, 64)
    gxs = (np.array([180.0e3, 220.0e3]) * sx / dx).astype(np.int32)
    gys = ((np.arange(16) + 0.5) * 16.0e3 * sy / dx).astype(np.int32)
    gauges = np.array([(a, b) for a in gxs for b in gys], dtype=np.int32)
    dt = cfl_dt(0.8, dx, 2000.0)
    basis = f32(gaussian_basis(x, y, cx, cy, sig))
    eta0 = f32(np.tensordot(f32(theta0), basis, axes=1))
    w = Workload("inversion_%dx%d" % (nx, ny), nx, ny, 1, f32(x), f32(y), f32(depth), eta0, dt,
                 steps, gauges=gauges, maxout=steps + 1, gout=1, bndout=steps + 1)
    w.extra.update(dict(src_x=cx, src_y=cy, src_sigma=sig, theta_true=f32(theta_true),
                        theta0=f32(theta0), basis=basis))
    return w


# --------------------------------------------------------------------------- run-up (E1)

def runup_1d(H_over_d=0.0185, d=1.0, slope=19.85, dt=0.03, steps=2000):
    """Solitary-wave run-up on a plane beach (section "Examples", "Runup on a sloping beach"),
    reconstructed: the paper's grid and initial-condition files are not available. A 1D
    Cartesian line from deep water at depth d to dry land, slope 1:slope from the toe up
    through the still shoreline; node spacing d in the deep part, narrowing linearly to
    0.1 d twenty depths before the toe and 0.1 d from there over the beach. Initial wave
    eta = H sech^2(gamma (x - X1)), gamma = sqrt(3H/(4 d^3)), centred half a wavelength
    (arccosh(sqrt 20)/gamma) seaward of the toe, moving shoreward with u = eta sqrt(g/d).
    Parameters of the paper's table: h_min 0.003 m, no friction, inundation on, dt 0.03 s,
    2000 steps; max-wave every step. The wave travels toward +x; the still shoreline is at
    x = 0. The beach is used unfiltered: it has no depth jumps, and raising depths below
    min_depth would flatten the swash zone."""
    H = H_over_d * d
    gamma = math.sqrt(3.0 * H / (4.0 * d ** 3))
    half = math.acosh(math.sqrt(20.0)) / gamma
    x_toe = -slope * d
    x1 = x_toe - half
    x_deep = x1 - 2.0 * half
    x_fine = x_toe - 20.0 * d
    x_land = 3.0 * d
    xs = [x_deep]
    while xs[-1] < x_land:
        xc = xs[-1]
        if xc < x_fine:
            f = min(1.0, (x_fine - xc) / (x_fine - x_deep))
            dx = d * (0.1 + 0.9 * f)
        else:
            dx = 0.1 * d
        xs.append(xc + dx)
    x = np.array(xs)
    depth = np.where(x <= x_toe, d, -x / slope)
    eta0 = H / np.cosh(gamma * (x - x1)) ** 2
    eta0 = np.where(depth > 0.0, eta0, 0.0)
    u0 = eta0 * math.sqrt(G / d)
    n = len(x)
    w = Workload("runup_1d_%.4f" % H_over_d, n, 1, 1, f32(x), f32(np.zeros(1)), f32(depth[None, :]),
                 f32(eta0[None, :]), dt, steps, u0=f32(u0[None, :]), h_min=0.003, manning_n2=0.0,
                 maxout=1, gout=steps + 1, bndout=steps + 1)
    w.extra.update(dict(H=H, d=d, slope=slope,
                        runup_law=2.831 * math.sqrt(slope) * H_over_d ** 1.25 * d))
    return w


WORKLOADS = {
    "beach_200": beach_200,
    "spherical_coast": spherical_coast,
    "shelf_islands": shelf_islands,
    "ensemble_512": ensemble_512,
    "inversion_1024": inversion_1024,
    "runup_1d": runup_1d,
}
