"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU).

Each test names the passage of the Cliffs manual (arXiv 1410.0753) it checks. None of them
compares the oracle with itself: the expected values come from the paper's closed forms,
from exact solutions of the linear equations, from conservation and symmetry, or from the
algorithm's rules applied by hand to tiny inputs.
"""
import math
import os

import numpy as np
import pytest

import oracle
import workloads

G = 9.81


def line_params(n, dt, **kw):
    return oracle.params(n, 1, dt, **kw)


# ----------------------------------------------------------------------------------------
# Section "Numerical stability", eqs. (eq:uet2), (eq:f), (eq:uet): one-step response of a
# single-node pulse (eta_j, u_j) in a still basin on an uneven bottom, uniform spacing.

def pulse_residual(eps, solver, form):
    dx, dt = 100.0, 1.0
    d = np.array([40.0, 40.0, 30.0, 20.0, 35.0, 60.0, 60.0, 60.0, 60.0])
    j = 4
    n = len(d)
    eta = np.zeros(n)
    u = np.zeros(n)
    eta[j] = eps
    u[j] = 0.3 * eps
    p = line_params(n, dt, manning_n2=0.0, solver=solver, form=form, h_min=0.01)
    r = oracle.sweep_line(p, np.full(n - 1, dx), d, eta, u, np.zeros(n))
    beta = dt * math.sqrt(G * d[j]) / dx                                        # Courant number
    f = (6 * math.sqrt(d[j]) - math.sqrt(d[j - 1]) - math.sqrt(d[j + 1])) / (4 * math.sqrt(d[j]))
    u_exp = (1 - beta ** 2 * f) * u[j]                                          # eq. (eq:u2)
    eta_exp = (1 - beta ** 2) * eta[j]                                          # eq. (eq:et)
    if solver == 2:                                                             # eq. (eq:et2)
        eta_exp -= beta / (4 * math.sqrt(G)) * (math.sqrt(d[j + 1]) - math.sqrt(d[j - 1])) * u[j]
    return abs(r["w"][j] - u_exp), abs(r["eta"][j] - eta_exp), abs(eta_exp - eta[j])


@pytest.mark.parametrize("solver", [2, 1])
@pytest.mark.parametrize("form", [0, 1])
def test_pulse_closed_form(solver, form):
    """The residual against the closed form is second order in the pulse size: halving
    the pulse quarters it (a wrong first-order term would only halve it)."""
    ru1, re1, shift = pulse_residual(1e-4, solver, form)
    ru2, re2, _ = pulse_residual(5e-5, solver, form)
    for a, b in ((ru1, ru2), (re1, re2)):
        assert a < 1e-7
        assert 3.3 < a / b < 4.7, (a, b)
    assert shift > 50 * re1          # the one-step change itself is far above the residual


def test_pulse_solvers_differ_by_the_printed_term():
    """eq. (eq:et2) minus eq. (eq:et): solver2 adds -beta/(4 sqrt g)(sqrt d_{j+1} - sqrt d_{j-1}) u."""
    _, re2, _ = pulse_residual(1e-4, 2, 0)
    # evaluating solver1 against the solver2 closed form leaves the printed term as residual
    dx, dt, j = 100.0, 1.0, 4
    d = np.array([40.0, 40.0, 30.0, 20.0, 35.0, 60.0, 60.0, 60.0, 60.0])
    eta = np.zeros(9); u = np.zeros(9); eta[j] = 1e-4; u[j] = 3e-5
    r1 = oracle.sweep_line(line_params(9, dt, solver=1), np.full(8, dx), d, eta, u, np.zeros(9))
    r2 = oracle.sweep_line(line_params(9, dt, solver=2), np.full(8, dx), d, eta, u, np.zeros(9))
    beta = dt * math.sqrt(G * d[j]) / dx
    term = beta / (4 * math.sqrt(G)) * (math.sqrt(d[j + 1]) - math.sqrt(d[j - 1])) * u[j]
    assert abs((r1["eta"][j] - r2["eta"][j]) - term) < 1e-3 * abs(term)


# ----------------------------------------------------------------------------------------
# eq. (eqQ): "In the steady state, Q = 0". Lake at rest over wet/dry steps, with land,
# a shoreline, an island, friction and both shoreline modes (itopo).

def lake_bathy(nx=40, ny=30):
    x = np.arange(nx) * 100.0
    y = np.arange(ny) * 100.0
    X, Y = np.meshgrid(x, y)
    d = 20.0 - 25.0 * X / x[-1] + 3.0 * np.sin(Y / 300.0)
    d -= 30.0 * np.exp(-((X - 1500) ** 2 + (Y - 1500) ** 2) / (2 * 250.0 ** 2))   # island
    d, _ = oracle.depth_filter(d)
    return x, y, d


@pytest.mark.parametrize("itopo", [1, 0])
def test_lake_at_rest(itopo):
    x, y, d = lake_bathy()
    assert (d < 0).any() and (d > 0).any()
    for solver in (2, 1):
        for form, tol in ((0, 1e-9), (1, 0.0)):
            p = oracle.params(d.shape[1], d.shape[0], 2.0, h_min=0.01, manning_n2=6.25e-4,
                              itopo=itopo, dwall=1.0, form=form, solver=solver)
            r = oracle.run(p, x, y, d, np.zeros_like(d), nsteps=1000)
            for k in ("eta", "u", "v"):
                assert np.abs(r[k]).max() <= tol, (solver, form, k, np.abs(r[k]).max())


# ----------------------------------------------------------------------------------------
# Linear long waves travel at sqrt(g h): on a flat bottom a still Gaussian hump splits
# into two halves moving at +-sqrt(gH) (d'Alembert). The scheme is second order in space
# (section "Difference Scheme": "second-order accurate in space for a uniform grid").

def dalembert_error(dx, solver=2):
    H, sigma, A = 10.0, 150.0, 1e-3
    L = 6000.0
    n = int(round(L / dx)) + 1
    x = np.arange(n) * dx
    c = math.sqrt(G * H)
    dt = 0.5 * 10.0 / c * (dx / 10.0)
    T = 1500.0 / c
    steps = int(round(T / dt))
    t = steps * dt
    x0 = 3000.0
    eta0 = A * np.exp(-(x - x0) ** 2 / (2 * sigma ** 2))
    p = oracle.params(n, 1, dt, manning_n2=0.0, h_min=0.01, solver=solver)
    r = oracle.run(p, x, np.zeros(1), np.full((1, n), H), eta0[None, :], nsteps=steps)
    exact = 0.5 * A * (np.exp(-(x - x0 - c * t) ** 2 / (2 * sigma ** 2)) +
                       np.exp(-(x - x0 + c * t) ** 2 / (2 * sigma ** 2)))
    return np.abs(r["eta"][0] - exact).max() / A


@pytest.mark.parametrize("solver", [2, 1])
def test_dalembert_speed_and_second_order(solver):
    e10 = dalembert_error(10.0, solver)   # sigma / dx = 15
    e20 = dalembert_error(20.0, solver)   # sigma / dx = 7.5
    assert e10 < 0.01, e10
    assert e20 / e10 > 3.0, (e20, e10)


# ----------------------------------------------------------------------------------------
# eq. (eqQ) in the Riemann invariants r = w +- 2c, and the same flux rewritten in
# perturbation variables: with c^2 = g (eta + d),
#   1/2 (lam_a + lam_b)(r_a - r_b) - g (d_a - d_b)
#     = 1/2 (lam_a + lam_b)(w_a - w_b) +- (w_a + w_b)(c_a - c_b) + g (eta_a - eta_b),
# c_a - c_b = g ((eta_a - eta_b) + (d_a - d_b)) / (c_a + c_b). The oracle computes both; on a
# moving flow over an uneven bottom they must agree to rounding, under either solver.

@pytest.mark.parametrize("solver", [2, 1])
def test_literal_and_perturbation_forms_agree(solver):
    rng = np.random.default_rng(17)
    n = 80
    x = np.concatenate([[0.0], np.cumsum(rng.uniform(40.0, 60.0, n - 1))])
    d = 12.0 + 8.0 * np.sin(x / 300.0) + 3.0 * rng.random(n)
    eta = 0.8 * np.exp(-(x - x[30]) ** 2 / (2 * 200.0 ** 2))
    u = 0.4 * np.sin(x / 170.0)
    out = []
    for form in (0, 1):
        p = oracle.params(n, 1, 1.0, h_min=0.01, manning_n2=6.25e-4, solver=solver, form=form)
        out.append(oracle.run(p, x, np.zeros(1), d[None, :], eta[None, :], u[None, :], nsteps=60))
    for f in ("eta", "u"):
        ref = np.abs(out[0][f]).max()
        assert np.abs(out[0][f] - out[1][f]).max() <= 1e-10 * ref, f
    assert np.abs(out[1]["eta"] - eta).max() > 0.1                 # the flow did move


# ----------------------------------------------------------------------------------------
# Dimensional splitting (eqs. eq2A/eq2B): for y-invariant data between reflecting north and
# south walls the y-sweep is the identity, so every row of a 2D run equals the 1D run.

def beach_1d(n=60):
    x = np.arange(n) * 50.0
    d = 8.0 - 10.0 * x / x[-1]
    eta = 0.6 * np.exp(-(x - 800.0) ** 2 / (2 * 200.0 ** 2))
    return x, d, eta


@pytest.mark.parametrize("form,tol", [(1, 0.0), (0, 1e-12)])
def test_1d_equals_2d_rows(form, tol):
    x, d1, e1 = beach_1d()
    n, ny, dt, steps = len(x), 7, 1.5, 150
    kw = dict(h_min=0.01, manning_n2=6.25e-4, form=form)
    r1 = oracle.run(oracle.params(n, 1, dt, **kw), x, np.zeros(1), d1[None, :], e1[None, :],
                    nsteps=steps)
    y = np.arange(ny) * 50.0
    r2 = oracle.run(oracle.params(n, ny, dt, **kw), x, y, np.tile(d1, (ny, 1)),
                    np.tile(e1, (ny, 1)), nsteps=steps)
    wet = (r1["eta"][0] + d1 >= 0.01)
    assert wet.sum() > 20 and (~wet).sum() > 3
    for k in ("eta", "u"):
        assert np.abs(r2[k] - r1[k][0][None, :]).max() <= tol
    assert np.abs(r2["v"]).max() == 0.0


@pytest.mark.parametrize("form,tol", [(1, 0.0), (0, 1e-12)])
def test_1d_equals_2d_columns(form, tol):
    y, d1, e1 = beach_1d()
    n, nx, dt, steps = len(y), 7, 1.5, 150
    kw = dict(h_min=0.01, manning_n2=6.25e-4, form=form)
    r1 = oracle.run(oracle.params(1, n, dt, **kw), np.zeros(1), y, d1[:, None], e1[:, None],
                    nsteps=steps)
    x = np.arange(nx) * 50.0
    r2 = oracle.run(oracle.params(nx, n, dt, **kw), x, y, np.tile(d1[:, None], (1, nx)),
                    np.tile(e1[:, None], (1, nx)), nsteps=steps)
    assert np.abs(r2["eta"] - r1["eta"]).max() <= tol
    assert np.abs(r2["v"] - r1["v"]).max() <= tol
    assert np.abs(r2["u"]).max() == 0.0


# ----------------------------------------------------------------------------------------
# Mass in a closed, fully wet flat basin: in the linear limit the update telescopes with the
# mirror walls and conserves sum(eta); the scheme is in characteristic (non-conservative)
# form, so the nonlinear drift is of the order of the wave steepness.

def mass_drift(eps, form=0, nsteps=400):
    nx, ny, H = 30, 24, 10.0
    x = np.arange(nx) * 100.0
    y = np.arange(ny) * 100.0
    X, Y = np.meshgrid(x, y)
    eta0 = eps * H * np.exp(-((X - 1200) ** 2 + (Y - 1100) ** 2) / (2 * 300.0 ** 2))
    p = oracle.params(nx, ny, 3.0, manning_n2=0.0, form=form)
    r = oracle.run(p, x, y, np.full((ny, nx), H), eta0, nsteps=nsteps)
    return abs(r["eta"].sum() - eta0.sum()) / np.abs(eta0).sum()


def test_mass_linear_limit():
    lin = mass_drift(1e-6, form=1)
    non = mass_drift(1e-2, form=1)
    assert lin < 1e-6, lin
    assert non > 100 * lin                 # the drift is a nonlinear effect
    assert mass_drift(1e-6, form=0) < 1e-5


# ----------------------------------------------------------------------------------------
# Walls half a node from the last wet node (section "Numerics": "a half-node re-positioning
# of the reflecting wall within a cell"; reading 3): the gravest seiche of a closed basin of
# N nodes has length L = N dx and period 2 L / sqrt(g H) (a wall on the node would give
# (N - 1) dx, 2.5 % shorter for N = 40).

def test_standing_wave_wall_at_half_node():
    N, dx, H, A = 40, 25.0, 10.0, 1e-4
    L = N * dx
    c = math.sqrt(G * H)
    x = np.arange(N) * dx
    dt = 0.25 * dx / c
    T = 2 * L / c
    eta0 = A * np.cos(np.pi * (x + dx / 2) / L)
    p = oracle.params(N, 1, dt, manning_n2=0.0)
    steps = int(2.6 * T / dt)
    r = oracle.run(p, x, np.zeros(1), np.full((1, N), H), eta0[None, :], nsteps=steps,
                   gout=1, gauges=[(0, 0)])
    s = r["gauges"][:, 0, 0]
    t = np.arange(len(s)) * dt
    k = np.where((s[:-1] > 0) & (s[1:] <= 0))[0]         # downward zero crossings
    tc = t[k] + dt * s[k] / (s[k] - s[k + 1])
    period = np.diff(tc).mean()
    assert abs(period / T - 1) < 3e-3, period / T


# ----------------------------------------------------------------------------------------
# Friction (reading 4): in a uniform flow no flux enters the interior, so the interior
# velocity follows the explicit Euler step of u_t = -g n^2 u |u| / h^(4/3), and h is
# untouched; the clamp keeps a thin fast layer from reversing.

@pytest.mark.parametrize("form", [0, 1])
def test_friction_uniform_flow(form):
    n2, H, dt, u0, nx = 6.25e-4, 2.0, 1.0, 1.5, 30
    x = np.arange(nx) * 100.0
    p = oracle.params(nx, nx, dt, manning_n2=n2, form=form)
    r = oracle.run(p, x, x, np.full((nx, nx), H), np.zeros((nx, nx)),
                   np.full((nx, nx), u0), nsteps=5)
    u = u0
    for _ in range(5):
        u = u - dt * G * n2 * u * abs(u) / H ** (4.0 / 3.0)
    c = (15, 15)
    assert abs(r["u"][c] - u) <= 1e-13 * u
    assert r["u"][c] < u0
    assert abs(r["eta"][c]) <= (0.0 if form == 1 else 1e-13)


def test_friction_clamp_never_reverses():
    n, dt = 9, 1.0
    p = line_params(n, dt, manning_n2=6.25e-4, h_min=0.01)
    r = oracle.sweep_line(p, np.full(n - 1, 100.0), np.full(n, 0.02), np.zeros(n),
                          np.full(n, 2.0), np.zeros(n))
    assert abs(r["w"][4]) < 1e-14
    p1 = line_params(n, dt, manning_n2=6.25e-4, h_min=0.01, form=1)
    r1 = oracle.sweep_line(p1, np.full(n - 1, 100.0), np.full(n, 0.02), np.zeros(n),
                           np.full(n, 2.0), np.zeros(n))
    assert r1["w"][4] == 0.0


# ----------------------------------------------------------------------------------------
# Inundation algorithm, steps (a)-(e), applied by hand to 7-node lines.

def sweep7(d, eta, w, t=None, itopo=1, dwall=0.0, dt=0.1):
    n = len(d)
    p = line_params(n, dt, h_min=0.01, manning_n2=0.0, itopo=itopo, dwall=dwall)
    return oracle.sweep_line(p, np.full(n - 1, 10.0), np.array(d, float), np.array(eta, float),
                             np.array(w, float), np.zeros(n) if t is None else np.array(t, float))


def test_step_b_flooding_by_hand():
    d = [5, 5, 5, -0.2, -1, -1, -1]
    r = sweep7(d, [0.5, 0.5, 0.5, 0, 0, 0, 0], [0.3, 0.3, 0.3, 0, 0, 0, 0],
               [0.1, 0.1, 0.1, 0, 0, 0, 0])
    assert list(r["wet0"]) == [1, 1, 1, 0, 0, 0, 0]                 # (a): h = -0.2 < h_min
    assert list(r["wet1"]) == [1, 1, 1, 1, 0, 0, 0]                 # (b): 0.5 - 0.2 > 0.01
    assert r["src"][3] == 2
    assert r["eta_b"][3] == 0.01 - (-0.2)                           # height h_min
    assert r["w_b"][3] == 0.3 and r["t_b"][3] == 0.1                # neighbour's velocities
    assert r["wet1"][4] == 0                                        # one ring per sweep
    assert r["eta"][4] == 0.0 and r["w"][4] == 0.0


def test_step_b_threshold_and_dry_velocity():
    r = sweep7([5, 5, 5, -0.6, -1, -1, -1], [0.5, 0.5, 0.5, 0, 0, 0, 0],
               [0.3, 0.3, 0.3, 0.7, 0.7, 0, 0])
    assert r["wet1"][3] == 0                                        # 0.5 - 0.6 < h_min
    assert r["w_b"][3] == 0.0 and r["w_b"][4] == 0.0                # (a): dry cells at rest


def test_step_b_tie_break():
    d = [5, 5, -0.1, 5, 5, 5, 5]
    r = sweep7(d, [0.5, 0.5, 0, 0.8, 0.8, 0.8, 0.8], [0.2, 0.2, 0, -0.4, -0.4, -0.4, -0.4])
    assert r["src"][2] == 3 and r["w_b"][2] == -0.4                 # larger eta wins
    r = sweep7(d, [0.5, 0.5, 0, 0.5, 0.5, 0.5, 0.5], [0.2, 0.2, 0, -0.4, -0.4, -0.4, -0.4])
    assert r["src"][2] == 1 and r["w_b"][2] == 0.2                  # tie: the left one


def test_step_a_vertical_wall_mode():
    # itopo = 0: nodes shallower than dwall are a permanent wall, even when covered
    r = sweep7([5, 5, 0.5, 5, 5, 5, 5], [0.5, 0.5, 2.0, 0.5, 0.5, 0.5, 0.5],
               [0.3] * 7, itopo=0, dwall=1.0)
    assert r["wet0"][2] == 0 and r["wet1"][2] == 0
    r = sweep7([5, 5, 0.5, 5, 5, 5, 5], [0.5, 0.5, 2.0, 0.5, 0.5, 0.5, 0.5], [0.3] * 7, itopo=1)
    assert r["wet0"][2] == 1


def test_step_e_cushion_limiter():
    # height branch: the new cell (3, filled from 2) ends above half its neighbour after (d)
    d = [0.559, 0.205, 0.142, -0.009, -1, -1, -1]
    r = sweep7(d, [0.038, 0.263, 0.284, 0, 0, 0, 0], [1.73, -1.647, 2.98, 0, 0, 0, 0], dt=1.976)
    assert r["src"][3] == 2
    hj = r["eta"][2] + d[2]
    assert r["eta_d"][3] + d[3] > hj / 2                             # the limiter fires
    assert abs((r["eta"][3] + d[3]) - hj / 2) < 1e-15                # h_i = h_j / 2
    # velocity branch: |u_i| > |u_j| after (d) is cut back to u_j
    d = [1.6228, 1.6228, 1.6228, -0.0436, -1, -1, -1]
    r = sweep7(d, [0.6066, 0.6066, 0.6066, 0, 0, 0, 0], [1.377, 1.377, 1.377, 0, 0, 0, 0],
               dt=0.5664)
    assert r["src"][3] == 2
    assert abs(r["w_d"][3]) > abs(r["w"][2])
    assert r["w"][3] == r["w"][2]
    # no limiter: a new cell below half its neighbour keeps its (d) state
    d = [10, 10, 10, -0.05, -1, -1, -1]
    r = sweep7(d, [1.0, 1.0, 1.0, 0, 0, 0, 0], [3.0, 3.0, 3.0, 0, 0, 0, 0], dt=1.0)
    assert r["src"][3] == 2
    assert r["eta_d"][3] + d[3] <= (r["eta"][2] + d[2]) / 2
    assert r["eta"][3] == r["eta_d"][3]


def test_front_moves_at_most_one_cell_per_sweep():
    # dam break onto a dry flat (section "Inundation algorithm": "the wet area is also
    # expanded by no more than one cell on each side")
    nx, ny = 40, 30
    x = np.arange(nx) * 10.0
    d = np.full((ny, nx), -0.001)
    eta = np.zeros((ny, nx))
    eta[10:20, 15:25] = 1.0
    p = oracle.params(nx, ny, 0.1, h_min=0.01, manning_n2=0.0)
    wet = lambda e: (e + d >= 0.01)
    prev = wet(eta)
    state = (eta, None, None)
    for _ in range(8):
        r = oracle.run(p, x, x, d, state[0], state[1], state[2], nsteps=1)
        now = wet(r["eta"])
        jj, ii = np.where(prev)
        # bounding box grows by at most one cell in each direction per step (x then y sweep)
        j2, i2 = np.where(now)
        assert i2.min() >= ii.min() - 1 and i2.max() <= ii.max() + 1
        assert j2.min() >= jj.min() - 1 and j2.max() <= jj.max() + 1
        prev = now
        state = (r["eta"], r["u"], r["v"])
    assert prev.sum() > 100


# ----------------------------------------------------------------------------------------
# Depth-jump filter (eqs. dstab, newdw, newdc), by hand and by its post-conditions.

def test_depth_filter_by_hand():
    d = np.array([[100.0, 100, 100], [100, 1, 100], [100, 100, 100]])
    out, n = oracle.depth_filter(d)
    assert np.all(out == 100.0) and n == 2          # newdw: (10 + 10)^2 / 4
    out, n = oracle.depth_filter(np.array([[-1.0, 1.0, 100.0]]))
    assert list(out[0]) == [-1.0, 25.0, 100.0]       # newdc next to the coast: 100 / 2^2
    out, _ = oracle.depth_filter(np.array([[-1.0, 0.05, 0.1, 0.1]]))
    assert out[0, 1] == 0.1                          # minimal depth in wet nodes
    out, _ = oracle.depth_filter(np.array([[4.0, 1.0, 4.0]]), alpha=2.0)
    assert out[0, 1] == 1.0                          # ratio exactly alpha^2 is allowed


def test_depth_filter_postconditions():
    rng = np.random.default_rng(5)
    d = 50.0 + 40.0 * rng.standard_normal((60, 50))
    d[rng.random(d.shape) < 0.05] = 0.5              # shallow spikes
    d[:, :5] = -3.0                                  # a coast
    for alpha in (2.0, 2.5):
        out, n = oracle.depth_filter(d, alpha=alpha)
        assert n > 0
        assert np.all(out[d <= 0] == d[d <= 0])      # land untouched
        a2 = alpha * alpha
        for arr in (out, out.T):
            c, l, r = arr[:, 1:-1], arr[:, :-2], arr[:, 2:]
            wet = c > 0
            assert np.all(~(wet & (l > 0)) | (l <= a2 * c * (1 + 1e-12)))
            assert np.all(~(wet & (r > 0)) | (r <= a2 * c * (1 + 1e-12)))
            # eqs. (rr), (rstab), (fcond): with alpha = 3 - 2 eps, dstab gives 1 + r >= eps on
            # both sides of every wet node between wet neighbours, hence f > 0
            eps = (3.0 - alpha) / 2.0
            both = wet & (l > 0) & (r > 0)
            sc, sl, sr = np.sqrt(c[both]), np.sqrt(l[both]), np.sqrt(r[both])
            assert np.all(1 + (sc - sl) / (2 * sc) >= eps - 1e-12)
            assert np.all(1 + (sc - sr) / (2 * sc) >= eps - 1e-12)
            assert np.all(6 * sc > sl + sr)
            assert both.sum() > 1000
        again, n2 = oracle.depth_filter(out, alpha=alpha)
        assert n2 == 1 and np.array_equal(again, out)  # idempotent
    # the unfiltered map breaks eq. (fcond) somewhere, so the check above has teeth
    c, l, r = d[:, 1:-1], d[:, :-2], d[:, 2:]
    both = (c > 0) & (l > 0) & (r > 0)
    assert np.any(6 * np.sqrt(c[both]) <= np.sqrt(l[both]) + np.sqrt(r[both]))
    smooth = np.full((20, 20), 30.0) + np.arange(20)[None, :]
    out, n = oracle.depth_filter(smooth)
    assert n == 1 and np.array_equal(out, smooth)   # untouched where dstab holds


# ----------------------------------------------------------------------------------------
# Spherical metrics (reading 7; the paper defers the equations to Titov & Gonzalez 1997):
# the equatorial limit is the Cartesian grid with dx = R dlambda, and a zonal wave crosses
# longitude 1 / cos(phi) times faster in degrees.

R = 6371000.0


def test_spherical_equator_limit():
    n, m = 80, 11
    dlam = 0.01
    lon = 150.0 + np.arange(n) * dlam
    lat = (np.arange(m) - m // 2) * 0.01
    xs = np.radians(lon - lon[0]) * R
    ys = np.radians(lat - lat[0]) * R
    H = 100.0
    X, Y = np.meshgrid(xs, ys)
    eta0 = 0.5 * np.exp(-((X - xs[40]) ** 2 + (Y - ys[5]) ** 2) / (2 * 3000.0 ** 2))
    dt = 0.5 * xs[1] / math.sqrt(G * H)
    rs = oracle.run(oracle.params(n, m, dt, coords=0, manning_n2=0.0), lon, lat,
                    np.full((m, n), H), eta0, nsteps=40)
    rc = oracle.run(oracle.params(n, m, dt, coords=1, manning_n2=0.0), xs, ys,
                    np.full((m, n), H), eta0, nsteps=40)
    assert np.abs(rs["eta"] - rc["eta"]).max() < 2e-4 * 0.5
    assert np.abs(rs["eta"]).max() > 0.05


def test_spherical_zonal_speed_scales_with_cos_lat():
    n, m, H = 400, 5, 1000.0
    dlam = 0.01
    c = math.sqrt(G * H)
    for phi in (0.0, 60.0):
        lon = np.arange(n) * dlam
        lat = phi + (np.arange(m) - m // 2) * dlam
        dxm = R * math.cos(math.radians(phi)) * math.radians(dlam)
        sig = 8 * dlam
        eta0 = np.tile(1e-3 * np.exp(-(lon - lon[n // 2]) ** 2 / (2 * sig ** 2)), (m, 1))
        dt = 0.4 * dxm / c
        steps = 150
        r = oracle.run(oracle.params(n, m, dt, coords=0, manning_n2=0.0), lon, lat,
                       np.full((m, n), H), eta0, nsteps=steps)
        row = r["eta"][m // 2]
        assert np.isfinite(row).all()
        right = np.argmax(row[n // 2:]) + n // 2
        moved_deg = (right - n // 2) * dlam
        expect_deg = math.degrees(c * steps * dt / (R * math.cos(math.radians(phi))))
        assert abs(moved_deg - expect_deg) <= 1.5 * dlam, (phi, moved_deg, expect_deg)


# ----------------------------------------------------------------------------------------
# Outputs (section "Running Options": maxout, gout, bndout).

def test_gauges_maxwave_and_bilinear_boundary():
    import workloads
    nx, ny = 30, 20
    x = 100.0 * np.arange(nx)
    y = 100.0 * np.arange(ny)
    X, Y = np.meshgrid(x, y)
    d = np.full((ny, nx), 10.0)
    lin = 1e-3 * (0.5 * X - 0.25 * Y + 30.0)          # a linear field is reproduced exactly
    nests = [workloads.Nest(x0=250.0, y0=330.0, dx=40.0, dy=25.0, nx=11, ny=9)]
    p = oracle.params(nx, ny, 2.0, manning_n2=0.0)
    r0 = oracle.run(p, x, y, d, lin, nsteps=0, bndout=1, nests=nests)
    W, E, S, N = r0["boundary"][0]
    n = nests[0]
    ys = n.y0 + n.dy * np.arange(n.ny)
    xs = n.x0 + n.dx * np.arange(n.nx)
    f = lambda a, b: 1e-3 * (0.5 * a - 0.25 * b + 30.0)
    assert np.allclose(W[0, 2], f(n.x0, ys), rtol=0, atol=1e-15)
    assert np.allclose(E[0, 2], f(n.x0 + 10 * n.dx, ys), rtol=0, atol=1e-15)
    assert np.allclose(S[0, 2], f(xs, n.y0), rtol=0, atol=1e-15)
    assert np.allclose(N[0, 2], f(xs, n.y0 + 8 * n.dy), rtol=0, atol=1e-15)
    assert W.shape == (1, 3, 9) and S.shape == (1, 3, 11)          # vals(tim, uvq, pnt)
    # a running case: gauges every step from step 0, max-wave every step
    eta0 = 0.3 * np.exp(-((X - 1500) ** 2 + (Y - 1000) ** 2) / (2 * 300.0 ** 2))
    gauges = [(15, 10), (5, 3), (29, 19)]
    r = oracle.run(p, x, y, d, eta0, nsteps=30, gout=1, gauges=gauges, maxout=1, bndout=3,
                   nests=nests)
    g = r["gauges"]
    assert g.shape == (31, 3, 3)
    assert np.array_equal(g[0, :, 0], [eta0[10, 15], eta0[3, 5], eta0[19, 29]])
    for k, (ix, iy) in enumerate(gauges):
        assert r["eta_max"][iy, ix] == g[:, k, 0].max()
    assert r["boundary"][0][0].shape[0] == 11                      # steps 0, 3, ..., 30
    # cadences: gauges every 4 steps are every 4th record of the run above; max-wave every 5
    # steps is the maximum over steps 0, 5, ..., 30 (the gauges are wet throughout)
    r4 = oracle.run(p, x, y, d, eta0, nsteps=30, gout=4, gauges=gauges, maxout=5)
    assert np.array_equal(r4["gauges"], g[::4])
    for k, (ix, iy) in enumerate(gauges):
        assert r4["eta_max"][iy, ix] == g[::5, k, 0].max()
    assert (r4["eta_max"] <= r["eta_max"]).all() and (r4["eta_max"] < r["eta_max"]).any()
    # every 7 steps: steps 0, 7, ..., 28, and the final state (step 30) folded in at the end
    r7 = oracle.run(p, x, y, d, eta0, nsteps=30, gout=1, gauges=gauges, maxout=7)
    for k, (ix, iy) in enumerate(gauges):
        assert r7["eta_max"][iy, ix] == g[[0, 7, 14, 21, 28, 30], k, 0].max()
    assert any(g[30, k, 0] > g[[0, 7, 14, 21, 28], k, 0].max() for k in range(len(gauges)))
    # record slots: a wave uniform in y moves u only (v stays exactly 0), so gauges hold
    # (eta, u, v) and boundary series (u, v, eta) in that order
    ex = 0.3 * np.exp(-(X - 1500) ** 2 / (2 * 300.0 ** 2))
    rx = oracle.run(p, x, y, d, ex, nsteps=20, gout=1, gauges=gauges, bndout=1, nests=nests)
    gx = rx["gauges"]
    assert np.abs(gx[1:, :, 1]).max() > 1e-6 and not gx[:, :, 2].any()
    Wx = rx["boundary"][0][0]
    assert np.abs(Wx[1:, 0]).max() > 1e-6 and not Wx[:, 1].any()


# ----------------------------------------------------------------------------------------
# Tangent-linear model (branches frozen on the primal) against central differences.

def test_tlm_matches_central_differences():
    nx, ny = 36, 24
    x = 100.0 * np.arange(nx)
    y = 100.0 * np.arange(ny)
    X, Y = np.meshgrid(x, y)
    d = 12.0 - 16.0 * X / x[-1]
    d, _ = oracle.depth_filter(d)
    eta0 = 0.4 * np.exp(-((X - 1000) ** 2 + (Y - 1200) ** 2) / (2 * 250.0 ** 2))
    dirn = np.exp(-((X - 1100) ** 2 + (Y - 1000) ** 2) / (2 * 300.0 ** 2))
    gauges = [(20, 12), (25, 5), (10, 20)]
    p = oracle.params(nx, ny, 2.0, manning_n2=6.25e-4, h_min=0.01)
    steps = 60
    gval, gtan, _, _ = oracle.run_tlm(p, x, y, d, eta0, dirn, nsteps=steps, gauges=gauges)
    h = 1e-3
    rp = oracle.run(p, x, y, d, eta0 + h * dirn, nsteps=steps, gout=1, gauges=gauges)
    rm = oracle.run(p, x, y, d, eta0 - h * dirn, nsteps=steps, gout=1, gauges=gauges)
    fd = (rp["gauges"][:, :, 0] - rm["gauges"][:, :, 0]) / (2 * h)
    scale = np.abs(gtan).max()
    assert scale > 1e-3
    assert np.abs(fd - gtan).max() <= 1e-5 * scale, np.abs(fd - gtan).max() / scale
    r0 = oracle.run(p, x, y, d, eta0, nsteps=steps, gout=1, gauges=gauges)
    assert np.array_equal(r0["gauges"][:, :, 0], gval)
    # the velocity tangents at the gauges against the same differences
    _, g3, _, _ = oracle.run_tlm(p, x, y, d, eta0, dirn, nsteps=steps, gauges=gauges, uv=True)
    assert np.array_equal(g3[:, :, 0], gtan)
    for comp in (1, 2):
        fdc = (rp["gauges"][:, :, comp] - rm["gauges"][:, :, comp]) / (2 * h)
        sc = np.abs(g3[:, :, comp]).max()
        assert sc > 1e-4
        assert np.abs(fdc - g3[:, :, comp]).max() <= 1e-5 * sc, (comp, np.abs(fdc - g3[:, :, comp]).max() / sc)


# ----------------------------------------------------------------------------------------
# eq. (pq3): the transverse velocity is carried by the along-sweep flow, v_t = -u v_x.

def test_transverse_velocity_advected_by_u():
    n, dx, H, U = 400, 10.0, 10.0, 2.0
    x = np.arange(n) * dx
    v0 = 0.1 * np.exp(-(x - 2000.0) ** 2 / (2 * 100.0 ** 2))
    dt = 0.5 * dx / (U + math.sqrt(G * H))
    steps = int(100.0 / dt)
    p = oracle.params(n, 1, dt, manning_n2=0.0)
    r = oracle.run(p, x, np.zeros(1), np.full((1, n), H), np.zeros((1, n)),
                   np.full((1, n), U), v0[None, :], nsteps=steps)
    v = r["v"][0]
    shift = (np.argmax(v) - np.argmax(v0)) * dx
    assert abs(shift - U * steps * dt) <= 1.0 * dx
    assert abs(v.max() / v0.max() - 1) < 0.05
    p0 = oracle.params(n, 1, dt, manning_n2=0.0, transverse=0)
    r0 = oracle.run(p0, x, np.zeros(1), np.full((1, n), H), np.zeros((1, n)),
                    np.full((1, n), U), v0[None, :], nsteps=steps)
    assert np.array_equal(r0["v"][0][1:-1], v0[1:-1])       # switched off: v stays put


# ----------------------------------------------------------------------------------------
# Spherical continuity (reading 7): with the term h v tan(phi)/R the area-weighted volume
# sum(eta cos(phi)) of a closed basin is kept in the linear limit; without it, or with the
# wrong sign, it drifts by the order of the meridional transport.

def test_spherical_area_weighted_mass():
    n, dlat, H = 40, 0.05, 1000.0
    lon = 140 + np.arange(n) * dlat
    lat = 30 + np.arange(n) * dlat
    LON, LAT = np.meshgrid(lon, lat)
    eta0 = 1e-3 * np.exp(-((LON - lon[n // 2]) ** 2 + (LAT - lat[n // 3]) ** 2) / (2 * (4 * dlat) ** 2))
    dsmin = R * math.cos(math.radians(lat[-1])) * math.radians(dlat)
    dt = 0.5 * dsmin / math.sqrt(G * H)
    r = oracle.run(oracle.params(n, n, dt, coords=0, manning_n2=0.0), lon, lat,
                   np.full((n, n), H), eta0, nsteps=300)
    w = np.cos(np.radians(LAT))
    drift_area = abs((r["eta"] * w).sum() - (eta0 * w).sum()) / np.abs(eta0 * w).sum()
    drift_plain = abs(r["eta"].sum() - eta0.sum()) / np.abs(eta0).sum()
    assert drift_area < 1e-4, drift_area
    assert drift_plain > 50 * drift_area


def test_maxwave_ignores_dry_cells():
    nx, ny = 20, 12
    x = 100.0 * np.arange(nx)
    X, Y = np.meshgrid(x, x[:ny])
    d = np.where(X > 1500.0, -2.0, 8.0)
    eta0 = 0.2 * np.exp(-((X - 700) ** 2 + (Y - 500) ** 2) / (2 * 200.0 ** 2))
    r = oracle.run(oracle.params(nx, ny, 2.0, manning_n2=0.0), x, x[:ny], d, eta0, nsteps=5,
                   maxout=1)
    fmax = np.finfo(np.float32).max
    assert np.all(r["eta_max"][d < -1] == -fmax) and np.all(r["speed_max"][d < -1] == 0)
    assert np.all(r["eta_max"][d > 0] >= eta0[d > 0])


# ----------------------------------------------------------------------------------------
# Run-up of a non-breaking solitary wave on a plane beach (section "Examples", "Runup on a
# sloping beach"; the Synolakis 1987 experiment): the run-up law R/d = 2.831 sqrt(cot beta)
# (H/d)^(5/4) holds to about 10 % for H/d = 0.0185 on the 1:19.85 slope. This exercises the
# inundation algorithm (a)-(e) over a whole run-up and run-down.

def test_runup_of_a_solitary_wave_follows_the_runup_law():
    w = workloads.runup_1d()
    p = oracle.params_from(w)
    r = oracle.run(p, w.x, w.y, w.depth.astype(np.float64), w.eta0, w.u0, None, nsteps=w.steps, maxout=1)
    land = w.depth[0] < 0
    em = r["eta_max"][0][land]
    R = em[em > -1e30].max()
    law = w.extra["runup_law"]
    assert abs(R / law - 1.0) <= 0.10, (R, law)


# ----------------------------------------------------------------------------------------
# Nesting chain (section "Running Options": boundary series for enclosed grids, then boundary
# input into such a grid). A child on the parent's own nodes, driven by the parent's series,
# must reproduce the parent inside it exactly in open water: there the update of an
# interior node reads only its neighbours (the 3-node stencil of eq. (solver2) in each
# sweep), and the child's edge nodes carry the parent's values at every step.

def _open_water_parent(nx=60, ny=50, steps=40):
    x = 100.0 * np.arange(nx)
    y = 100.0 * np.arange(ny)
    X, Y = np.meshgrid(x, y)
    d = 40.0 + 8.0 * np.sin(X / 900.0) * np.cos(Y / 700.0)
    eta0 = 0.8 * np.exp(-((X - 2400.0) ** 2 + (Y - 2100.0) ** 2) / (2 * 500.0 ** 2))
    p = oracle.params(nx, ny, 1.5, manning_n2=6.25e-4)
    return x, y, d, eta0, p, steps


def test_nesting_chain_reproduces_the_parent_inside_the_child():
    from workloads import Nest
    x, y, d, eta0, p, steps = _open_water_parent()
    i0, j0, cx, cy = 17, 12, 30, 24
    nest = Nest(x[i0], y[j0], 100.0, 100.0, cx, cy)
    par = oracle.run(p, x, y, d, eta0, nsteps=steps, bndout=1, nests=[nest])
    series = par["boundary"][0]                               # W, E, S, N: [nt][3][np]
    times = 1.5 * np.arange(steps + 1)
    sub = (slice(j0, j0 + cy), slice(i0, i0 + cx))
    pc = oracle.params(cx, cy, 1.5, manning_n2=6.25e-4)
    ch = oracle.run_forced(pc, x[i0:i0 + cx], y[j0:j0 + cy], d[sub], eta0[sub],
                           {e: (times, series[e]) for e in range(4)}, nsteps=steps)
    for f in ("eta", "u", "v"):
        assert np.array_equal(ch[f][1:-1, 1:-1], par[f][sub][1:-1, 1:-1]), f
    # without the input the child's walls reflect the wave and the interior departs
    free = oracle.run(pc, x[i0:i0 + cx], y[j0:j0 + cy], d[sub], eta0[sub], nsteps=steps)
    assert np.abs(free["eta"] - par["eta"][sub]).max() > 1e-3


def test_forced_tlm_matches_central_differences_of_the_forced_run():
    """Under boundary input the edge nodes take the input before each step, so their tangent
    is zero there; the forced tangent model against central differences of the forced run on
    an enclosed grid of a sloping parent (the wave crosses the child's edges)."""
    from workloads import Nest
    x, y, d, eta0, p, steps = _open_water_parent()
    i0, j0, cx, cy = 17, 12, 30, 24
    nest = Nest(x[i0], y[j0], 100.0, 100.0, cx, cy)
    par = oracle.run(p, x, y, d, eta0, nsteps=steps, bndout=1, nests=[nest])
    times = 1.5 * np.arange(steps + 1)
    bnd = {e: (times, par["boundary"][0][e]) for e in range(4)}
    sub = (slice(j0, j0 + cy), slice(i0, i0 + cx))
    pc = oracle.params(cx, cy, 1.5, manning_n2=6.25e-4)
    cxs, cys = x[i0:i0 + cx], y[j0:j0 + cy]
    X, Y = np.meshgrid(cxs, cys)
    dirn = np.exp(-((X - cxs[4]) ** 2 + (Y - cys[12]) ** 2) / (2 * 400.0 ** 2))   # reaches the W edge
    gauges = [(2, 12), (15, 12), (27, 20)]
    gval, gtan = oracle.run_tlm_forced(pc, cxs, cys, d[sub], eta0[sub], dirn, bnd, nsteps=steps, gauges=gauges)
    h = 1e-3
    rp = oracle.run_forced(pc, cxs, cys, d[sub], eta0[sub] + h * dirn, bnd, nsteps=steps, gauges=gauges)
    rm = oracle.run_forced(pc, cxs, cys, d[sub], eta0[sub] - h * dirn, bnd, nsteps=steps, gauges=gauges)
    fd = (rp["gauges"][:, :, 0] - rm["gauges"][:, :, 0]) / (2 * h)
    scale = np.abs(gtan).max()
    assert scale > 1e-3
    assert np.abs(fd - gtan).max() <= 1e-6 * scale, np.abs(fd - gtan).max() / scale
    r0 = oracle.run_forced(pc, cxs, cys, d[sub], eta0[sub], bnd, nsteps=steps, gauges=gauges)
    assert np.array_equal(r0["gauges"][:, :, 0], gval)
    # the unforced tangent differs: the perturbation leaving through the edges is not replaced
    _, free, _, _ = oracle.run_tlm(pc, cxs, cys, d[sub], eta0[sub], dirn, nsteps=steps, gauges=gauges)
    assert np.abs(free - gtan).max() > 1e-3 * scale


# ----------------------------------------------------------------------------------------
# Initial conditions from a source grid (section "Running Options", "The input to the
# computations"): interpolated inside the source grid, zero outside it.

def test_initial_condition_interpolation_exact_for_linear_fields_and_zero_outside():
    rng = np.random.default_rng(9)
    sx = np.sort(rng.uniform(100.0, 900.0, 23))
    sy = np.sort(rng.uniform(-300.0, 500.0, 17))
    SX, SY = np.meshgrid(sx, sy)
    f = 0.3 + 1e-3 * SX - 2e-3 * SY
    mx = np.linspace(0.0, 1000.0, 41)
    my = np.linspace(-400.0, 600.0, 37)
    out = oracle.interp_initial(mx, my, sx, sy, f)
    MX, MY = np.meshgrid(mx, my)
    inside = (MX >= sx[0]) & (MX <= sx[-1]) & (MY >= sy[0]) & (MY <= sy[-1])
    assert np.abs(out - (0.3 + 1e-3 * MX - 2e-3 * MY))[inside].max() < 1e-12
    assert not out[~inside].any()
    # master nodes on source nodes take the source values
    same = oracle.interp_initial(sx, sy, sx, sy, f)
    assert np.array_equal(same, f)


# ----------------------------------------------------------------------------------------
# Open outer edges (the paper gives no condition): the ghost beyond an edge node carries the
# node's outgoing Riemann invariant and still water's incoming one.

def _channel(n=400, dx=50.0, d0=10.0):
    x = dx * np.arange(n)
    return x, np.full((1, n), d0)


def test_open_edges_keep_a_lake_at_rest():
    nx, ny = 40, 30
    x, y = 100.0 * np.arange(nx), 100.0 * np.arange(ny)
    X, Y = np.meshgrid(x, y)
    d = 20.0 + 10.0 * np.sin(X / 700.0) * np.cos(Y / 500.0)
    p = oracle.params(nx, ny, 1.0, manning_n2=6.25e-4, open_edges=15)
    r = oracle.run(p, x, y, d, np.zeros((ny, nx)), nsteps=50)
    assert np.abs(r["eta"]).max() < 1e-12 and np.abs(r["u"]).max() < 1e-12 and np.abs(r["v"]).max() < 1e-12


def test_open_edge_lets_a_simple_wave_leave():
    """A right-going linear wave (u = eta sqrt(g/d)) on a flat channel crossing an open east
    edge: while it goes out, the channel matches a channel twice as long (where nothing has
    come back yet) to within 2 % of the amplitude; a wall instead sends it all back."""
    n = 400
    x, d = _channel(n)
    X, D = _channel(2 * n)
    c0 = np.sqrt(9.81 * 10.0)
    A, x0, sig = 0.05, 15000.0, 800.0
    eta0 = A * np.exp(-((X - x0) ** 2) / (2 * sig ** 2))
    u0 = eta0 * c0 / 10.0
    dt = 0.5 * 50.0 / c0
    worst = 0.0
    for steps in range(150, 400, 50):                        # the crest reaches the edge at ~200
        ro = oracle.run(oracle.params(n, 1, dt, open_edges=2), x, np.zeros(1), d, eta0[None, :n], u0[None, :n],
                        nsteps=steps)
        rl = oracle.run(oracle.params(2 * n, 1, dt), X, np.zeros(1), D, eta0[None, :], u0[None, :], nsteps=steps)
        worst = max(worst, np.abs(ro["eta"][0] - rl["eta"][0, :n]).max())
    assert worst < 0.02 * A, worst / A
    rw = oracle.run(oracle.params(n, 1, dt), x, np.zeros(1), d, eta0[None, :n], u0[None, :n], nsteps=350)
    assert np.abs(rw["eta"]).max() > 0.5 * A


def test_open_edges_drain_a_raised_level_toward_still_water():
    """A uniform raised level at rest in a channel open at both ends runs out toward the
    still-water level of the incoming invariants (a zero-gradient edge would keep it)."""
    x, d = _channel(n=200)
    c0 = np.sqrt(9.81 * 10.0)
    dt = 0.5 * 50.0 / c0
    eta0 = np.full((1, len(x)), 0.2)
    p = oracle.params(len(x), 1, dt, open_edges=3)
    r = oracle.run(p, x, np.zeros(1), d, eta0, nsteps=int(6 * x[-1] / c0 / dt))
    assert np.abs(r["eta"]).max() < 0.02 * 0.2
    closed = oracle.run(oracle.params(len(x), 1, dt), x, np.zeros(1), d, eta0, nsteps=200)
    assert np.abs(closed["eta"] - eta0).max() < 1e-12


def test_open_edges_columns_equal_rows():
    """The S and N bits act on a column exactly as W and E act on a row."""
    x, d = _channel(n=150)
    c0 = np.sqrt(9.81 * 10.0)
    dt = 0.5 * 50.0 / c0
    eta0 = 0.3 * np.exp(-((x - 5000.0) ** 2) / (2 * 600.0 ** 2))
    u0 = 0.2 * np.sin(x / 900.0)
    for ew, sn in ((1, 4), (2, 8), (3, 12)):
        rx = oracle.run(oracle.params(len(x), 1, dt, open_edges=ew), x, np.zeros(1), d, eta0[None, :],
                        u0[None, :], nsteps=180)
        ry = oracle.run(oracle.params(1, len(x), dt, open_edges=sn), np.zeros(1), x, d.T.copy(), eta0[:, None],
                        None, u0[:, None], nsteps=180)
        assert np.array_equal(rx["eta"][0], ry["eta"][:, 0])
        assert np.array_equal(rx["u"][0], ry["v"][:, 0])


def test_open_edges_let_a_radial_wave_leave_a_square():
    """A radial wave in a square open on all four sides: once it has passed the edges little
    is left (oblique incidence reflects a little); with walls it stays in the basin."""
    n = 120
    x = 100.0 * np.arange(n)
    X, Y = np.meshgrid(x, x)
    d = np.full((n, n), 20.0)
    c0 = np.sqrt(9.81 * 20.0)
    dt = 0.5 * 100.0 / c0
    eta0 = 0.1 * np.exp(-((X - 6000.0) ** 2 + (Y - 6000.0) ** 2) / (2 * 700.0 ** 2))
    steps = int(1.6 * 6000.0 / c0 / dt)
    r = oracle.run(oracle.params(n, n, dt, open_edges=15), x, x, d, eta0, nsteps=steps)
    w = oracle.run(oracle.params(n, n, dt), x, x, d, eta0, nsteps=steps)
    E_open = np.sum(r["eta"] ** 2 + (20.0 / 9.81) * (r["u"] ** 2 + r["v"] ** 2))
    E_wall = np.sum(w["eta"] ** 2 + (20.0 / 9.81) * (w["u"] ** 2 + w["v"] ** 2))
    assert E_open < 0.05 * E_wall, (E_open, E_wall)


def test_tlm_with_open_edges_matches_central_differences():
    """The tangent model through the open ghost (a function of the edge node) against central
    differences, with the perturbation crossing the W and N edges."""
    nx, ny = 36, 28
    x, y = 100.0 * np.arange(nx), 100.0 * np.arange(ny)
    X, Y = np.meshgrid(x, y)
    d = 15.0 + 5.0 * np.cos(X / 800.0) * np.sin(Y / 600.0)
    eta0 = 0.3 * np.exp(-((X - 800.0) ** 2 + (Y - 2000.0) ** 2) / (2 * 400.0 ** 2))
    dirn = np.exp(-((X - 500.0) ** 2 + (Y - 2300.0) ** 2) / (2 * 350.0 ** 2))
    gauges = [(0, 20), (1, 24), (10, 27), (20, 14)]
    p = oracle.params(nx, ny, 2.0, manning_n2=6.25e-4, open_edges=15)
    steps = 60
    gval, gtan, _, _ = oracle.run_tlm(p, x, y, d, eta0, dirn, nsteps=steps, gauges=gauges)
    h = 1e-4
    rp = oracle.run(p, x, y, d, eta0 + h * dirn, nsteps=steps, gout=1, gauges=gauges)
    rm = oracle.run(p, x, y, d, eta0 - h * dirn, nsteps=steps, gout=1, gauges=gauges)
    fd = (rp["gauges"][:, :, 0] - rm["gauges"][:, :, 0]) / (2 * h)
    scale = np.abs(gtan).max()
    assert scale > 1e-2
    assert np.abs(fd - gtan).max() <= 1e-6 * scale, np.abs(fd - gtan).max() / scale
    # the tangent sees the open edges: with walls it differs
    _, gw, _, _ = oracle.run_tlm(oracle.params(nx, ny, 2.0, manning_n2=6.25e-4), x, y, d, eta0, dirn,
                                 nsteps=steps, gauges=gauges)
    assert np.abs(gw - gtan).max() > 1e-2 * scale


def _golden(name):
    vals = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", name)):
        line = line.split("#")[0].split()
        if line:
            vals[line[0]] = [float(v) for v in line[1:]]
    return vals


def test_runup_workload_takes_the_printed_parameter_file():
    """The reconstructed run-up example uses the values of the paper's Table 1 where the
    method reads them (Cartesian, h_min, friction, inundation, dt, steps) and the printed
    wave heights and slope; max-wave every step instead of every 500 (the test reads the
    maxima) is the one stated departure."""
    t = _golden("runup_params_table1.txt")
    for H in t["H_over_d"]:
        w = workloads.runup_1d(H_over_d=H)
        assert w.coords == t["coords"][0] and w.ny == 1
        assert w.h_min == t["h_min"][0] and w.manning_n2 == t["manning_n2"][0]
        assert (w.itopo != 0) == (t["itopo"][0] != 0)
        assert w.dt == t["dt"][0] and w.steps == t["steps"][0]
        assert w.extra["slope"] == t["slope"][0] and math.isclose(w.extra["H"] / w.extra["d"], H)
        assert not w.nests and not len(w.gauges)


# ----------------------------------------------------------------------------------------
# Section "Numerics", eqs. (eq2A), (eq2B): the step is the x-problem followed by the
# y-problem; with alternating splitting the odd steps take them in the other order. The
# y-sweep of a grid is the x-sweep of its transpose (x <-> y, u <-> v), so a step in the
# order y then x equals the plain step of the transposed grid, transposed back. That fixes
# what two alternating steps must give without using the alternating code.

def _shore_problem(nx=14, ny=11, seed=31):
    rng = np.random.default_rng(seed)
    x = np.concatenate([[0.0], np.cumsum(rng.uniform(80.0, 120.0, nx - 1))])
    y = np.concatenate([[0.0], np.cumsum(rng.uniform(80.0, 120.0, ny - 1))])
    X, Y = np.meshgrid(x, y)
    d = 15.0 + 45.0 * rng.random((ny, nx))
    d[:3, :4] = -0.4                                               # a low beach in one corner
    eta = 1.2 * np.exp(-((X - x[4]) ** 2 + (Y - y[4]) ** 2) / (2 * 260.0 ** 2))
    eta[d < 0] = -d[d < 0]                                         # dry: h = 0
    u = 0.1 * rng.standard_normal((ny, nx))
    v = 0.1 * rng.standard_normal((ny, nx))
    u[d < 0] = v[d < 0] = 0.0
    return x, y, d, eta, u, v


def _y_then_x(kw, x, y, d, eta, u, v):
    ny, nx = d.shape
    r = oracle.run(oracle.params(ny, nx, 1.0, **kw), y, x, d.T, eta.T, v.T, u.T, nsteps=1)
    return r["eta"].T, r["v"].T, r["u"].T


@pytest.mark.parametrize("form", [0, 1])
def test_alternating_sweeps_take_y_first_on_odd_steps(form):
    x, y, d, eta, u, v = _shore_problem()
    ny, nx = d.shape
    kw = dict(h_min=0.01, manning_n2=6.25e-4, form=form)
    alt = oracle.run(oracle.params(nx, ny, 1.0, alternate=1, **kw), x, y, d, eta, u, v, nsteps=2)
    one = oracle.run(oracle.params(nx, ny, 1.0, **kw), x, y, d, eta, u, v, nsteps=1)   # step 0: x, y
    e2, u2, v2 = _y_then_x(kw, x, y, d, one["eta"], one["u"], one["v"])               # step 1: y, x
    for f, ref in (("eta", e2), ("u", u2), ("v", v2)):
        assert np.abs(alt[f] - ref).max() <= 1e-12 * (1.0 + np.abs(ref).max()), f
    # an odd first step is y then x
    odd = oracle.run(oracle.params(nx, ny, 1.0, alternate=1, **kw), x, y, d, eta, u, v, nsteps=1, step0=1)
    e1, _, _ = _y_then_x(kw, x, y, d, eta, u, v)
    assert np.abs(odd["eta"] - e1).max() <= 1e-12 * (1.0 + np.abs(e1).max())
    # the orders differ by far more than the tolerance on this problem
    plain = oracle.run(oracle.params(nx, ny, 1.0, **kw), x, y, d, eta, u, v, nsteps=2)
    assert np.abs(plain["eta"] - alt["eta"]).max() > 1e-6
    assert np.abs(one["eta"] - e1).max() > 1e-6


# ----------------------------------------------------------------------------------------
# Section "Running Options", the input to the computations: boundary input is a time series
# at the edge nodes. Between records the input is the straight line through the two records
# (before the first and after the last it holds that record), so imposing a series at a time
# between records equals imposing the constant series of the interpolated value.

def test_boundary_input_is_linear_between_records():
    x, y, d, eta0, p, _ = _open_water_parent(nx=12, ny=10)
    rng = np.random.default_rng(5)
    ny = d.shape[0]
    a = 0.3 * rng.standard_normal((3, ny))
    b = 0.3 * rng.standard_normal((3, ny))
    series = {0: (np.array([0.0, 4.0]), np.stack([a, b]))}

    def forced(bnd, t0, nsteps=1, **state):
        return oracle.run_forced(p, x, y, d, state.get("eta", eta0), bnd, u=state.get("u"),
                                 v=state.get("v"), nsteps=nsteps, t0=t0, step0=state.get("step0", 0))

    for t0, val in ((1.0, 0.75 * a + 0.25 * b), (3.0, 0.25 * a + 0.75 * b),
                    (-2.0, a), (9.0, b)):
        got = forced(series, t0)
        ref = forced({0: (np.array([0.0]), val[None])}, 0.0)
        for f in ("eta", "u", "v"):
            assert np.array_equal(got[f], ref[f]), (t0, f)
    # the model clock advances by dt per step: two steps from t = 1 equal one step at t = 1
    # and one at t = 1 + dt (1.5 s) = 2.5 s, each against its interpolated constant input
    two = forced(series, 1.0, nsteps=2)
    first = forced({0: (np.array([0.0]), (0.75 * a + 0.25 * b)[None])}, 0.0)
    second = forced({0: (np.array([0.0]), (0.375 * a + 0.625 * b)[None])}, 0.0,
                    eta=first["eta"], u=first["u"], v=first["v"], step0=1)
    for f in ("eta", "u", "v"):
        assert np.array_equal(two[f], second[f]), f


# ----------------------------------------------------------------------------------------
# Section "Running Options", field quake: with quake = 1 the initial deformation zeta is
# applied to the sea floor. The floor rises by zeta everywhere; over wet nodes the water
# column rises with it (its height is unchanged, the surface stands at zeta); dry nodes and,
# with itopo = 0, walls keep a flat surface.

def test_quake_lifts_the_floor_and_the_water_column_with_it():
    rng = np.random.default_rng(23)
    d = rng.uniform(-20.0, 80.0, (30, 40))
    d[0, :5] = [0.0, 0.005, 0.01, 0.02, 3.0]                       # around h_min and a wall
    zeta = rng.uniform(-1.5, 2.5, d.shape)
    for itopo, dwall in ((1, 0.0), (0, 5.0)):
        dn, eta = oracle.quake_init(d, zeta, 0.01, itopo=itopo, dwall=dwall)
        assert np.allclose(dn + zeta, d, rtol=0.0, atol=1e-12)
        wet = (d >= 0.01) if itopo else (d >= 5.0)
        assert np.array_equal(eta[wet], zeta[wet])
        assert not eta[~wet].any()
        assert np.allclose((eta + dn)[wet], d[wet], rtol=0.0, atol=1e-12)
    # by hand: nodes 50 m, 5 mm (below h_min), land and a 2 m node, h_min = 1 cm
    d4 = np.array([[50.0, 0.005, -3.0, 2.0]])
    z4 = np.array([[1.0, 0.5, 0.25, -0.5]])
    dn, eta = oracle.quake_init(d4, z4, 0.01, itopo=1)
    assert dn.tolist() == [[49.0, -0.495, -3.25, 2.5]] and eta.tolist() == [[1.0, 0.0, 0.0, -0.5]]
    dn, eta = oracle.quake_init(d4, z4, 0.01, itopo=0, dwall=5.0)  # the 2 m node is a wall
    assert eta.tolist() == [[1.0, 0.0, 0.0, 0.0]]


# ----------------------------------------------------------------------------------------
# The lines of a sweep are independent (eqs. eq2A, eq2B), so the oracle's threads over them
# cannot change a bit of the result; and the seeded inputs are the same on every call.

def test_oracle_threads_do_not_change_results():
    w = workloads.spherical_coast(96, 80, steps=40)
    d = oracle.depth_filter(w.depth, w.filter_alpha, w.filter_min_depth)[0]
    p = oracle.params_from(w)
    kw = dict(nsteps=w.steps, maxout=1, gout=1, gauges=w.gauges, bndout=1, nests=w.nests)
    n0 = oracle.threads()
    try:
        oracle.threads(1)
        one = oracle.run(p, w.x, w.y, d, w.eta0, **kw)
        oracle.threads(max(2, os.cpu_count() or 2))
        many = oracle.run(p, w.x, w.y, d, w.eta0, **kw)
    finally:
        oracle.threads(n0)
    for k in ("eta", "u", "v", "eta_max", "speed_max", "gauges"):
        assert np.array_equal(one[k], many[k]), k
    for a, b in zip(one["boundary"][0], many["boundary"][0]):
        assert np.array_equal(a, b)


def test_seeded_inputs_repeat():
    for make in (lambda: workloads.spherical_coast(64, 48, steps=5),
                 lambda: workloads.ensemble_512(batch=3, nx=40, ny=32),
                 lambda: workloads.inversion_1024(64, 48, steps=5),
                 lambda: workloads.shelf_islands(128, 96, steps=5),
                 lambda: workloads.beach_200(40, 30, steps=5)):
        a, b = make(), make()
        for f in ("x", "y", "depth", "eta0"):
            assert np.array_equal(getattr(a, f), getattr(b, f)), f
        assert np.array_equal(a.gauges, b.gauges)


# ----------------------------------------------------------------------------------------
# Section "Numerical stability", the one-step pulse response, on unequal spacings: eq.
# (solver2) applied to a pulse (eta_j, u_j) at node j of a flat basin of depth H, spacings
# dsL to the left and dsR to the right, gives to second order in the pulse
#   eta_j' = (1 - b) eta_j - (H dt / 2) s u_j,   u_j' = (1 - b) u_j - (g dt / 2) s eta_j,
# b = g H dt^2 / (dsL dsR) (the second-order term, k2 = dt^2 / (dsL + dsR)) and
# s = 1/dsL - 1/dsR (the averaged first-order fluxes); eq. (solver1)'s first-order flux spans
# the two neighbours at rest, so s = 0 there. With dsL = dsR this is eq. (eq:uet), f = 1.

def unequal_pulse_residual(eps, solver, form, dsL=80.0, dsR=130.0):
    H, dt, j, n = 30.0, 1.0, 4, 9
    ds = np.array([100.0, 90.0, 110.0, dsL, dsR, 95.0, 105.0, 100.0])
    eta = np.zeros(n); u = np.zeros(n)
    eta[j], u[j] = eps, 0.4 * eps
    p = line_params(n, dt, manning_n2=0.0, solver=solver, form=form, h_min=0.01)
    r = oracle.sweep_line(p, ds, np.full(n, H), eta, u, np.zeros(n))
    b = G * H * dt ** 2 / (dsL * dsR)
    s = (1 / dsL - 1 / dsR) if solver == 2 else 0.0
    eta_exp = (1 - b) * eta[j] - 0.5 * H * dt * s * u[j]
    u_exp = (1 - b) * u[j] - 0.5 * G * dt * s * eta[j]
    return abs(r["eta"][j] - eta_exp), abs(r["w"][j] - u_exp), abs(eta_exp - eta[j])


@pytest.mark.parametrize("solver", [2, 1])
@pytest.mark.parametrize("form", [0, 1])
def test_pulse_closed_form_on_unequal_spacing(solver, form):
    re1, ru1, shift = unequal_pulse_residual(1e-4, solver, form)
    re2, ru2, _ = unequal_pulse_residual(5e-5, solver, form)
    for a, b in ((re1, re2), (ru1, ru2)):
        assert a < 1e-9 and 3.3 < a / b < 4.7, (a, b)
    assert shift > 1e3 * re1
