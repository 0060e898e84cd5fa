"""The hand-written adjoint (cliffs_adjoint_n) on the GPU.

Pinned three ways: (1) the dot-product identity against the FP64 oracle's tangent-linear
model, <dL/d eta0, delta> = sum_r,g seed[r,g] * (TLM delta)[r,g], with branches frozen on the
primal on both sides; (2) central finite differences of the GPU forward on unit-source
coefficients through torch.autograd; (3) checkpoint spacing changes nothing (bit for bit).

Tolerances. The adjoint runs in FP32 against an FP64 tangent model over runs of 60-160
steps; each step's Jacobian coefficients carry FP32 relative errors of a few 1e-7, and the
coefficients are formed in the perturbation form, so no p = w + 2c cancellation enters.
Measured: at most 8e-6 of the largest term of the dot product (shoreline and spherical runs
included). The bound is 1e-4, which a dropped term, a wrong sign or a transposed stencil
exceeds by orders of magnitude. Central differences of the FP32 forward with h = 1e-3 carry
~1e-5 relative rounding noise and O(h^2) truncation; measured 4e-5, bound 1e-3.
"""
import numpy as np
import pytest

import oracle
import workloads
from paper_1410_0753_gb300 import CliffsError, CliffsGrid, ERR_ARG, ERR_STATE
from tests import parity as P

pytestmark = pytest.mark.gpu

DOT_RTOL = 1e-4
FD_RTOL = 1e-3


def _start(w, **kw):
    g = CliffsGrid.from_workload(w, **kw)
    g.set_bathy(w.x, w.y, w.depth, True, w.filter_alpha, w.filter_min_depth)
    g.set_initial(w.eta0.astype(np.float32))
    return g


def _walls():
    w = workloads.beach_200(200, 90, steps=400)
    w.itopo, w.dwall = 0, 5.0                      # a vertical wall where the beach is shallower than 5 m
    return w


def _no_transverse():
    w = workloads.inversion_1024(nx=128, ny=112, steps=120)
    w.transverse, w.manning_n2 = 0, 0.0
    return w


def _solver1():
    w = workloads.beach_200(200, 90, steps=300)
    w.extra["solver"] = 1                          # eq. (solver1), run-up included
    return w


def _alternate():
    w = workloads.spherical_coast(160, 150, steps=61)
    w.extra["alternate"] = 1                       # y first on the odd steps
    return w


def _cases():
    return {
        "solver1_beach": _solver1,
        "alternate_spherical": _alternate,
        "inversion_slope": lambda: workloads.inversion_1024(nx=128, ny=112, steps=160),
        "beach_runup": lambda: workloads.beach_200(200, 90, steps=400),   # the wave runs up the shore
        "spherical_coast": lambda: workloads.spherical_coast(160, 150, steps=60),
        "walls_itopo0": _walls,
        "no_transverse_no_friction": _no_transverse,
    }


@pytest.mark.parametrize("case", sorted(_cases()))
def test_adjoint_dot_product_against_oracle_tlm(case):
    w = _cases()[case]()
    n = w.steps
    solver, alternate = w.extra.get("solver", 2), w.extra.get("alternate", 0)
    g = _start(w, solver=solver, alternate=alternate)
    nrec = n // w.gout + 1
    G = len(w.gauges)
    rng = np.random.default_rng(17)
    seed = rng.standard_normal((nrec, G)).astype(np.float32)
    grad = g.adjoint(n, seed, checkpoint_every=37).astype(np.float64)
    assert np.isfinite(grad).all()
    if case in ("beach_runup", "walls_itopo0", "inversion_slope", "spherical_coast", "solver1_beach",
                "alternate_spherical"):
        assert (w.depth < (w.dwall if w.itopo == 0 else w.h_min)).any()   # dry land or walls in play
    d64 = P.f32(P.oracle_depth(w))
    p = oracle.params_from(w, solver=solver, alternate=alternate)
    yy, xx = np.meshgrid(np.arange(w.ny), np.arange(w.nx), indexing="ij")
    worst = 0.0
    for k in range(3):
        cx, cy = rng.uniform(0.3, 0.7) * w.nx, rng.uniform(0.3, 0.7) * w.ny
        sig = rng.uniform(0.05, 0.12) * min(w.nx, w.ny)
        delta = np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * sig ** 2))
        if k == 2:
            delta = delta + 0.1 * rng.standard_normal(delta.shape)
        _, gtan, _, _ = oracle.run_tlm(p, w.x, w.y, d64, w.eta0, delta, nsteps=n, gout=w.gout,
                                       gauges=w.gauges)
        terms = seed.astype(np.float64) * gtan
        want = terms.sum()
        got = float((grad * delta).sum())
        scale = max(np.abs(terms).max(), 1e-12)
        err = abs(got - want) / scale
        worst = max(worst, err)
        assert err <= DOT_RTOL, (case, k, got, want, scale)
    P.report("adjoint_dot_" + case, rel_err=worst)
    g.close()


def test_adjoint_gradient_matches_finite_differences_through_autograd():
    import torch
    from paper_1410_0753_gb300.autograd import gauge_run
    w = workloads.inversion_1024(nx=128, ny=112, steps=120)
    n = w.steps
    basis = torch.tensor(w.extra["basis"], device="cuda")
    truth = torch.tensor(w.extra["theta_true"], device="cuda")
    g = _start(w)
    with torch.no_grad():
        obs = gauge_run(torch.einsum("k,kyx->yx", truth, basis), g, n)

    def loss(theta):
        eta0 = torch.einsum("k,kyx->yx", theta, basis)
        return 0.5 * ((gauge_run(eta0, g, n, 25) - obs) ** 2).sum(dtype=torch.float64)

    theta = torch.tensor(w.extra["theta0"], device="cuda", requires_grad=True)
    L = loss(theta)
    L.backward()
    grad = theta.grad.detach().cpu().numpy().astype(np.float64)
    assert np.isfinite(grad).all() and np.abs(grad).max() > 0
    h = 1e-3
    worst = 0.0
    rng = np.random.default_rng(5)
    dirs = []
    for k in np.argsort(-np.abs(grad))[:8]:             # 8 coordinates
        e = np.zeros(64)
        e[k] = 1.0
        dirs.append(e)
    for _ in range(4):                                  # and 4 random directions
        v = rng.standard_normal(64)
        dirs.append(v / np.linalg.norm(v))
    with torch.no_grad():
        for v in dirs:
            e = torch.tensor(h * v, dtype=theta.dtype, device="cuda")
            fd = (loss(theta + e).item() - loss(theta - e).item()) / (2 * h)
            want = float(grad @ v)
            err = abs(fd - want) / np.abs(grad).max()
            worst = max(worst, err)
            assert err <= FD_RTOL, (fd, want)
    P.report("adjoint_fd_inversion", rel_err=worst)
    g.close()


def test_adjoint_unit_source_gradient_against_oracle():
    """The gradient of L = sum (eta_g - obs)^2 with respect to all 64 unit-source
    coefficients, obs from the FP64 oracle at the true coefficients: GPU forward + adjoint
    against the oracle's own forward and tangent-linear runs, within 1e-3 relative L2 over
    the 64-vector."""
    w = workloads.inversion_1024(nx=128, ny=112, steps=100)
    n = w.steps
    basis = w.extra["basis"].astype(np.float64)
    d64 = P.f32(P.oracle_depth(w))
    p = oracle.params_from(w)
    eta_true = P.f32(np.tensordot(w.extra["theta_true"].astype(np.float64), basis, axes=1))
    obs = oracle.run(p, w.x, w.y, d64, eta_true, nsteps=n, gout=w.gout, gauges=w.gauges)["gauges"][:, :, 0]
    # GPU: forward at theta0, seed 2 (eta - obs), adjoint, projected on the basis
    g = _start(w)
    g.step(n)
    seed32 = (2.0 * (g.gauges()[:, :, 0].astype(np.float64) - obs)).astype(np.float32)
    g.set_initial(w.eta0.astype(np.float32))
    grad_eta = g.adjoint(n, seed32, checkpoint_every=30).astype(np.float64)
    gpu = basis.reshape(64, -1) @ grad_eta.ravel()
    g.close()
    # oracle: its own forward residual and one tangent-linear run per coefficient
    r64 = oracle.run(p, w.x, w.y, d64, w.eta0, nsteps=n, gout=w.gout, gauges=w.gauges)["gauges"][:, :, 0]
    seed64 = 2.0 * (r64 - obs)
    ref = np.empty(64)
    for k in range(64):
        _, gtan, _, _ = oracle.run_tlm(p, w.x, w.y, d64, w.eta0, basis[k], nsteps=n, gout=w.gout,
                                       gauges=w.gauges)
        ref[k] = float((seed64 * gtan).sum())
    rel = np.linalg.norm(gpu - ref) / np.linalg.norm(ref)
    P.report("adjoint_theta64_vs_oracle", rel_l2=rel)
    assert np.linalg.norm(ref) > 0
    assert rel <= 1e-3, rel


def test_adjoint_checkpoint_spacing_and_state_untouched():
    """Any checkpoint spacing gives the same gradient bit for bit (the forward is recomputed
    by the same kernel), and the grid's own state is left as it was."""
    w = workloads.beach_200(96, 80, steps=70)
    g = _start(w)
    g.step(5)
    before = g.state()
    n = 40
    seed = np.random.default_rng(3).standard_normal((n // w.gout + 1, len(w.gauges))).astype(np.float32)
    ref = g.adjoint(n, seed, checkpoint_every=n)
    # K = 2: 20 segments; the checkpoint pass keeps the states of the last 16, the first 4
    # are recomputed in one batched launch per step. K = 7 and 16: every segment (a shorter
    # last one included) kept by the checkpoint pass. K = 1: every state kept.
    for K in (1, 2, 7, 16):
        assert np.array_equal(g.adjoint(n, seed, checkpoint_every=K), ref)
    for x, y in zip(before, g.state()):
        assert np.array_equal(x, y)
    assert np.count_nonzero(ref) > 0
    assert not np.any(g.adjoint(n, None))
    g.close()


def test_adjoint_argument_errors():
    w = workloads.ensemble_512(batch=2, nx=64, ny=48, dmin=5, dmax=9)
    g = _start(w)
    g.set_durations(w.durations)
    for scen, n in ((2, 4), (-1, 4), (0, int(w.durations[0]) + 1)):     # no such scenario; past its end
        with pytest.raises(CliffsError) as e:
            g.adjoint(n, None, scenario=scen)
        assert e.value.code == ERR_ARG
    assert not np.any(g.adjoint(4, None, scenario=1))
    g.close()
    w = workloads.beach_200(64, 48, steps=10)
    g = _start(w)
    for n, k in ((0, 5), (5, 0)):
        with pytest.raises(CliffsError) as e:
            g.adjoint(n, None, checkpoint_every=k)
        assert e.value.code == ERR_ARG
    g.close()


def test_recorded_run_gradient_equals_the_checkpoint_pass_gradient():
    """A forward recorded by cliffs_step_n (a checkpoint every K steps) gives the adjoint the
    same checkpoints as its own checkpoint pass, so cliffs_adjoint_recorded equals
    cliffs_adjoint_n bit for bit; the autograd binding uses the record, and falls back to a
    fresh start when the grid ran something else in between."""
    import torch
    from paper_1410_0753_gb300.autograd import gauge_run
    w = workloads.inversion_1024(nx=128, ny=112, steps=90)
    n = w.steps
    seed = np.random.default_rng(8).standard_normal((n // w.gout + 1, len(w.gauges))).astype(np.float32)
    g = _start(w)
    ref = g.adjoint(n, seed, checkpoint_every=20)
    with pytest.raises(CliffsError) as e:
        g.adjoint_recorded(seed)
    assert e.value.code == ERR_STATE
    assert np.array_equal(g.adjoint(n, seed, checkpoint_every=1), ref)   # every state kept, read in place
    g.adjoint_record(20)
    g.step(50)
    g.step(40)                                   # the record follows the run across calls
    assert np.array_equal(g.adjoint_recorded(seed), ref)
    g.set_initial(w.eta0.astype(np.float32))     # a record of every state: no recomputation
    g.adjoint_record(1)
    g.step(n)
    assert np.array_equal(g.adjoint_recorded(seed), ref)
    with pytest.raises(CliffsError) as e:
        g.step(2, persistent=True)
    assert e.value.code == ERR_ARG
    g.set_initial(w.eta0.astype(np.float32))     # a new record from the new initial state
    g.step(n)
    assert np.array_equal(g.adjoint_recorded(seed), ref)
    with pytest.raises(CliffsError) as e:
        g.adjoint_record(10)                     # only from an initial state
    assert e.value.code == ERR_STATE
    g.adjoint_record(0)
    # autograd: recorded path, and the fresh-start path after another run on the grid
    eta = torch.tensor(w.eta0, device="cuda", requires_grad=True)
    out = gauge_run(eta, g, n, 20)
    out.backward(torch.tensor(seed, device="cuda"))
    a1 = eta.grad.detach().cpu().numpy()
    eta.grad = None
    out = gauge_run(eta, g, n, 20)
    g.step(3)
    out.backward(torch.tensor(seed, device="cuda"))
    a2 = eta.grad.detach().cpu().numpy()
    eta.grad = None
    out = gauge_run(eta, g, n)                   # default: every state kept (it fits), nothing recomputed
    out.backward(torch.tensor(seed, device="cuda"))
    a3 = eta.grad.detach().cpu().numpy()
    assert np.array_equal(a1, ref) and np.array_equal(a2, ref) and np.array_equal(a3, ref)
    g.close()


def test_adjoint_with_respect_to_initial_velocities():
    """dL/du0 and dL/dv0 from the same adjoint run, against the oracle's tangent-linear model
    along velocity directions (the dot-product identity)."""
    w = workloads.inversion_1024(nx=128, ny=112, steps=100)
    n = w.steps
    g = _start(w)
    with pytest.raises(CliffsError) as e:
        g.adjoint_velocity()
    assert e.value.code == ERR_STATE
    rng = np.random.default_rng(23)
    seed = rng.standard_normal((n // w.gout + 1, len(w.gauges))).astype(np.float32)
    g.adjoint(n, seed, checkpoint_every=30)
    du, dv = g.adjoint_velocity()
    g.close()
    d64 = P.f32(P.oracle_depth(w))
    p = oracle.params_from(w)
    yy, xx = np.meshgrid(np.arange(w.ny), np.arange(w.nx), indexing="ij")
    z = np.zeros((w.ny, w.nx))
    worst = 0.0
    for k in range(2):
        dirn = np.exp(-((xx - rng.uniform(30, 90)) ** 2 + (yy - rng.uniform(30, 80)) ** 2) / (2 * 12.0 ** 2))
        args = (dict(du=dirn, dv=z), dict(du=z, dv=dirn))[k]
        _, gtan, _, _ = oracle.run_tlm(p, w.x, w.y, d64, w.eta0, z, nsteps=n, gout=w.gout, gauges=w.gauges, **args)
        terms = seed.astype(np.float64) * gtan
        got = float(((du, dv)[k].astype(np.float64) * dirn).sum())
        err = abs(got - terms.sum()) / max(np.abs(terms).max(), 1e-12)
        worst = max(worst, err)
        assert err <= DOT_RTOL, (k, got, terms.sum())
    P.report("adjoint_dot_velocity", rel_err=worst)


def _dot_against_tlm(p, w, grad, seed, state, n, step0=0, k=3, rng=None):
    """Worst relative error of <grad, delta> against the oracle's tangent model from the
    GPU state `state` (eta, u, v) over the next n steps."""
    rng = rng or np.random.default_rng(31)
    d64 = P.f32(P.oracle_depth(w))
    yy, xx = np.meshgrid(np.arange(w.ny), np.arange(w.nx), indexing="ij")
    worst, dots = 0.0, []
    for i in range(k):
        cx, cy = rng.uniform(0.3, 0.7) * w.nx, rng.uniform(0.3, 0.7) * w.ny
        sig = rng.uniform(0.05, 0.12) * min(w.nx, w.ny)
        delta = np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * sig ** 2))
        _, gtan, _, _ = oracle.run_tlm(p, w.x, w.y, d64, state[0], delta, u=state[1], v=state[2], nsteps=n,
                                       step0=step0, gout=w.gout, gauges=w.gauges)
        terms = seed.astype(np.float64) * gtan
        got = float((grad * delta).sum())
        worst = max(worst, abs(got - terms.sum()) / max(np.abs(terms).max(), 1e-12))
        dots.append((got, terms.sum(), np.abs(terms).max()))
    return worst, dots


def test_batched_scenario_adjoint_equals_a_single_grid_and_the_oracle():
    """Scenario 1 of a batched grid, 10 steps in: its adjoint equals, bit for bit, the adjoint
    of a single grid started from the same state, and passes the dot-product test against
    the oracle's tangent model from that state."""
    w = workloads.ensemble_512(batch=3, nx=120, ny=100, dmin=60, dmax=90)
    g = _start(w)
    g.set_durations(w.durations)
    g.step(10)
    state = g.state(1)
    n = 40
    rng = np.random.default_rng(37)
    seed = rng.standard_normal((n // w.gout + 1, len(w.gauges))).astype(np.float32)
    grad = g.adjoint(n, seed, checkpoint_every=13, scenario=1)
    others = [g.state(b) for b in (0, 2)]
    g.close()
    s1 = CliffsGrid(w.nx, w.ny, w.dt, coords=w.coords, h_min=w.h_min, manning_n2=w.manning_n2, itopo=w.itopo,
                    dwall=w.dwall, transverse=w.transverse, maxout=w.maxout, gout=w.gout,
                    gauges=[tuple(q) for q in w.gauges])
    s1.set_bathy(w.x, w.y, w.depth, True, w.filter_alpha, w.filter_min_depth)
    s1.set_initial(*state)
    single = s1.adjoint(n, seed, checkpoint_every=13)
    s1.close()
    assert np.array_equal(grad, single)
    assert all(np.isfinite(o[0]).all() for o in others)
    p = oracle.params_from(w)
    worst, _ = _dot_against_tlm(p, w, grad.astype(np.float64), seed, state, n, rng=rng)
    P.report("adjoint_dot_batched_scenario", rel_err=worst)
    assert worst <= DOT_RTOL


def test_alternating_adjoint_keeps_the_forward_parity_after_odd_steps():
    """After 3 steps the next step of the alternating order sweeps y first; the adjoint from
    there must transpose that order: the dot-product test against the oracle's tangent model
    started at step index 3 passes, and the same test at the other parity fails (the two
    splitting orders differ at second order, so that failure is small but far above the
    right parity's error)."""
    w = _alternate()
    g = _start(w, alternate=1)
    g.step(3)
    state = g.state()
    n = 40
    rng = np.random.default_rng(41)
    seed = rng.standard_normal((n // w.gout + 1, len(w.gauges))).astype(np.float32)
    grad = g.adjoint(n, seed, checkpoint_every=17).astype(np.float64)
    g.close()
    p = oracle.params_from(w, alternate=1)
    worst, _ = _dot_against_tlm(p, w, grad, seed, state, n, step0=3, rng=np.random.default_rng(5))
    P.report("adjoint_dot_alternate_odd_start", rel_err=worst)
    assert worst <= DOT_RTOL
    wrong, _ = _dot_against_tlm(p, w, grad, seed, state, n, step0=4, rng=np.random.default_rng(5))
    assert wrong > DOT_RTOL and wrong > 50 * worst, (wrong, worst)       # measured 2.2e-4 vs 5.3e-7


def test_adjoint_of_velocity_records_dot_product_against_oracle_tlm():
    """Seeds on all three recorded fields (eta, u, v) of every gauge: the GPU adjoint against
    the oracle's tangent model of the same records (its u and v tangents pinned by central
    differences), on the beach with run-up and on the spherical coast."""
    for name in ("beach_runup", "spherical_coast"):
        w = _cases()[name]()
        n = w.steps
        g = _start(w)
        nrec = n // w.gout + 1
        rng = np.random.default_rng(43)
        seed = rng.standard_normal((nrec, len(w.gauges), 3)).astype(np.float32)
        grad = g.adjoint(n, seed, checkpoint_every=37).astype(np.float64)
        du, dv = g.adjoint_velocity()
        eta_only = g.adjoint(n, np.ascontiguousarray(seed[:, :, 0]), checkpoint_every=37).astype(np.float64)
        g.close()
        assert not np.array_equal(grad, eta_only)            # the velocity seeds reach eta0
        d64 = P.f32(P.oracle_depth(w))
        p = oracle.params_from(w)
        yy, xx = np.meshgrid(np.arange(w.ny), np.arange(w.nx), indexing="ij")
        worst = 0.0
        for k in range(3):
            cx, cy = rng.uniform(0.3, 0.7) * w.nx, rng.uniform(0.3, 0.7) * w.ny
            sig = rng.uniform(0.05, 0.12) * min(w.nx, w.ny)
            delta = np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * sig ** 2))
            _, g3, _, _ = oracle.run_tlm(p, w.x, w.y, d64, w.eta0, delta, nsteps=n, gout=w.gout,
                                         gauges=w.gauges, uv=True)
            terms = seed.astype(np.float64) * g3
            got = float((grad * delta).sum())
            err = abs(got - terms.sum()) / max(np.abs(terms).max(), 1e-12)
            worst = max(worst, err)
            assert err <= DOT_RTOL, (name, k, got, terms.sum())
        # and along an initial-velocity direction (eta0 fixed): dL/du0
        delta_u = np.exp(-((xx - 0.5 * w.nx) ** 2 + (yy - 0.5 * w.ny) ** 2) / (2 * (0.1 * w.nx) ** 2))
        z = np.zeros_like(delta_u)
        _, g3, _, _ = oracle.run_tlm(p, w.x, w.y, d64, w.eta0, z, du=delta_u, nsteps=n, gout=w.gout,
                                     gauges=w.gauges, uv=True)
        terms = seed.astype(np.float64) * g3
        err = abs(float((du.astype(np.float64) * delta_u).sum()) - terms.sum()) / max(np.abs(terms).max(), 1e-12)
        worst = max(worst, err)
        assert err <= DOT_RTOL, (name, "u0", err)
        P.report("adjoint_dot_records_" + name, rel_err=worst)


def test_autograd_on_whole_records_matches_finite_differences():
    """gauge_run(records=True): a loss on the recorded velocities, gradient through the
    recorded forward and the adjoint against central differences of the GPU forward."""
    import torch
    from paper_1410_0753_gb300.autograd import gauge_run
    w = workloads.inversion_1024(nx=128, ny=112, steps=100)
    n = w.steps
    basis = torch.tensor(w.extra["basis"], device="cuda")
    g = _start(w)

    def loss(theta):
        rec = gauge_run(torch.einsum("k,kyx->yx", theta, basis), g, n, 25, records=True)
        return 0.5 * (rec[:, :, 1] ** 2 + 3.0 * rec[:, :, 2] ** 2 + rec[:, :, 0] ** 2).sum(dtype=torch.float64)

    theta = torch.tensor(w.extra["theta0"], device="cuda", requires_grad=True)
    loss(theta).backward()
    grad = theta.grad.detach().cpu().numpy().astype(np.float64)
    assert np.isfinite(grad).all() and np.abs(grad).max() > 0
    h, worst = 1e-3, 0.0
    with torch.no_grad():
        for k in np.argsort(-np.abs(grad))[:6]:
            e = torch.zeros(64, dtype=theta.dtype, device="cuda")
            e[k] = h
            fd = (loss(theta + e).item() - loss(theta - e).item()) / (2 * h)
            err = abs(fd - grad[k]) / np.abs(grad).max()
            worst = max(worst, err)
            assert err <= FD_RTOL, (k, fd, grad[k])
    P.report("adjoint_fd_records", rel_err=worst)
    g.close()


def test_every_state_kept_with_the_alternating_order():
    """checkpoint_every = 1 (each state read where it is stored) gives the bits of any other
    spacing, also with y-first steps."""
    w = _alternate()
    g = _start(w, alternate=1)
    n = 41
    seed = np.random.default_rng(9).standard_normal((n // w.gout + 1, len(w.gauges))).astype(np.float32)
    a7 = g.adjoint(n, seed, checkpoint_every=7)
    a1 = g.adjoint(n, seed, checkpoint_every=1)
    g.close()
    assert np.array_equal(a1, a7) and np.abs(a1).max() > 0


def test_recorded_batched_run_per_scenario():
    """A recorded batched forward keeps every scenario's states; the recorded adjoint of a
    scenario equals its checkpoint-pass adjoint from the same initial state bit for bit (with
    a checkpoint every 7 steps and with every state kept), for eta and for whole-record
    seeds; a scenario that stopped before the end of the record is refused."""
    w = workloads.ensemble_512(batch=3, nx=96, ny=80, dmin=30, dmax=50)
    n = 30
    rng = np.random.default_rng(47)
    seed = rng.standard_normal((n // w.gout + 1, len(w.gauges))).astype(np.float32)
    seed3 = rng.standard_normal((n // w.gout + 1, len(w.gauges), 3)).astype(np.float32)
    g = _start(w)
    g.set_durations(w.durations)
    refs = {b: (g.adjoint(n, seed, checkpoint_every=7, scenario=b), g.adjoint(n, seed3, checkpoint_every=7, scenario=b))
            for b in (0, 2)}
    for K in (7, 1):
        g.set_initial(w.eta0.astype(np.float32))
        g.adjoint_record(K)
        g.step(n)
        for b in (0, 2):
            assert np.array_equal(g.adjoint_recorded(seed, scenario=b), refs[b][0])
            assert np.array_equal(g.adjoint_recorded(seed3, scenario=b), refs[b][1])
    g.adjoint_record(0)
    g.close()
    short = w.durations.copy()
    short[1] = n - 5
    g = _start(w)
    g.set_durations(short)
    g.adjoint_record(5)
    g.step(n)
    with pytest.raises(CliffsError) as e:
        g.adjoint_recorded(seed, scenario=1)
    assert e.value.code == ERR_ARG
    assert np.array_equal(g.adjoint_recorded(seed, scenario=0), refs[0][0])
    g.close()


def test_adjoint_inversion_1024_at_its_stated_size():
    """The inversion workload at its stated size: 1024^2 nodes, 2000 FP32 steps, a checkpoint
    every 100 steps, 32 gauges, L = sum (eta_g - obs)^2 with obs from the FP64 oracle at the
    true coefficients; the gradient with respect to the 64 unit-source coefficients theta.
    (1) Dot-product identity: <dL/dtheta, dtheta> from the GPU adjoint against the oracle's
        FP64 tangent-linear model with the same (GPU) seed, on 3 seeded directions; the
        sum runs over 2001 records x 32 gauges, so its rounding scales with sum |terms|,
        to which the difference is compared (bound 1e-4).
    (2) The oracle's gradient: the same directional derivatives with the oracle's own FP64
        residual as seed, within 1e-3 of |dL/dtheta|.
    (3) Central differences (h = 1e-3) of the FP64 oracle's loss on the 2 largest
        coordinates and 2 random directions, against the GPU gradient: within 1e-3 of
        max |dL/dtheta| on the directions whose two runs take the same wet/dry history (the
        same nodes ever wet, the same final mask), within 1e-2 on the others; the gradient
        is that of the step with its branches frozen, which a difference across a flooding
        decision does not see (over 2000 steps of run-up most directions flip a shoreline
        node between theta - h and theta + h).
    (4) Central differences of the GPU's FP32 forward on the 8 largest coordinates and 4
        random directions, reported: at this size they carry the
        FP32 forward's rounding, ~2 sum|r| delta_r / 2h with delta_r ~ 1e-6 m over 2000 steps,
        a few 1e-3 of max |dL/dtheta|; bound 2e-2."""
    w = workloads.inversion_1024()
    n = w.steps
    assert (w.nx, w.ny, n, len(w.gauges)) == (1024, 1024, 2000, 32)
    B = w.extra["basis"].reshape(64, -1).astype(np.float64)     # [64][nodes]
    d64 = P.f32(P.oracle_depth(w))
    p = oracle.params_from(w)
    kw = dict(nsteps=n, gout=w.gout, gauges=w.gauges)
    eta_true = P.f32(np.tensordot(w.extra["theta_true"].astype(np.float64), w.extra["basis"], axes=1))
    obs = oracle.run(p, w.x, w.y, d64, eta_true, **kw)["gauges"][:, :, 0]
    g = _start(w)

    def eta_of(theta):
        return (theta @ B).reshape(w.ny, w.nx).astype(np.float32)

    def loss(theta):
        g.set_initial(eta_of(theta))
        g.step(n)
        r = g.gauges()[:, :, 0].astype(np.float64) - obs
        return float((r * r).sum()), r

    def loss64(theta):
        o = oracle.run(p, w.x, w.y, d64, eta_of(theta).astype(np.float64), maxout=1, **kw)
        r = o["gauges"][:, :, 0] - obs
        # the wet/dry history: nodes ever wet (max-wave set) and wet at the end
        return float((r * r).sum()), o["eta_max"] > -1e30, (o["eta"] + d64) >= w.h_min

    theta0 = w.extra["theta0"].astype(np.float64)
    L0, r32 = loss(theta0)
    seed32 = (2.0 * r32).astype(np.float32)
    g.set_initial(eta_of(theta0))
    grad_eta = g.adjoint(n, seed32, checkpoint_every=100).astype(np.float64).ravel()
    gtheta = B @ grad_eta
    assert np.isfinite(gtheta).all() and np.linalg.norm(gtheta) > 0
    h = 1e-3
    rng = np.random.default_rng(41)
    dirs = [np.eye(64)[k] for k in np.argsort(-np.abs(gtheta))[:8]]
    for _ in range(4):
        v = rng.standard_normal(64)
        dirs.append(v / np.linalg.norm(v))
    fd32_worst = 0.0
    for v in dirs:
        fd = (loss(theta0 + h * v)[0] - loss(theta0 - h * v)[0]) / (2 * h)
        fd32_worst = max(fd32_worst, abs(fd - float(gtheta @ v)) / np.abs(gtheta).max())
    g.close()
    fd64 = []
    for v in dirs[:2] + dirs[8:10]:                   # 2 coordinates, 2 random directions
        Lp, evp, wp = loss64(theta0 + h * v)
        Lm, evm, wm = loss64(theta0 - h * v)
        flip_free = bool(np.array_equal(evp, evm) and np.array_equal(wp, wm))
        fd64.append((abs((Lp - Lm) / (2 * h) - float(gtheta @ v)) / np.abs(gtheta).max(), flip_free))
    free = [e for e, f in fd64 if f]
    fd64_worst = max(free, default=0.0)
    fd64_all = max(e for e, _ in fd64)
    eta0 = eta_of(theta0).astype(np.float64)
    r64 = oracle.run(p, w.x, w.y, d64, eta0, **kw)["gauges"][:, :, 0] - obs
    seed64 = 2.0 * r64
    dot_worst, grad_worst = 0.0, 0.0
    for k in range(3):
        v = rng.standard_normal(64)
        v /= np.linalg.norm(v)
        delta = (v @ B).reshape(w.ny, w.nx)
        _, gtan, _, _ = oracle.run_tlm(p, w.x, w.y, d64, eta0, delta, **kw)
        got = float(gtheta @ v)
        terms = seed32.astype(np.float64) * gtan
        dot_worst = max(dot_worst, abs(got - terms.sum()) / np.abs(terms).sum())
        grad_worst = max(grad_worst, abs(got - float((seed64 * gtan).sum())) / np.linalg.norm(gtheta))
    P.report("adjoint_inversion_1024_full", steps=n, dot_rel=dot_worst, oracle_grad_rel=grad_worst,
             fd64_rel_flip_free=fd64_worst, fd64_per_direction=[[float(e), int(f)] for e, f in fd64],
             fd32_rel=fd32_worst, loss=L0, grad_norm=float(np.linalg.norm(gtheta)))
    assert dot_worst <= DOT_RTOL, dot_worst
    assert grad_worst <= 1e-3, grad_worst
    assert fd64_worst <= FD_RTOL and fd64_all <= 1e-2, fd64
    assert fd32_worst <= 2e-2, fd32_worst
