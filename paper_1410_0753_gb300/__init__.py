"""Python binding of libcliffs.so, the GB300 (sm_103a) shallow-water step of the Cliffs model
(arXiv 1410.0753). Argument marshalling only: every step of the method runs in the library's
CUDA kernels. The functions below carry the C ABI's names (include/cliffs.h) and raise
``CliffsError`` on a non-zero status; ``CliffsGrid`` wraps a handle.

Arrays may be NumPy arrays (host) or torch CUDA tensors (device pointers); the library copies
inputs before returning and fills outputs before returning.

The library is built in-tree by ``paper_1410_0753_gb300._build.build()`` (also run by
``__graft_entry__.build()``). Loading fails with an error when it is missing: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from . import _build

__all__ = [
    "CliffsError", "CliffsGrid", "lib", "cliffs_config", "cliffs_nest",
    "cliffs_grid_create", "cliffs_set_bathy", "cliffs_read_depth", "cliffs_set_initial",
    "cliffs_set_durations", "cliffs_step_n", "cliffs_steps_done", "cliffs_read_gauges",
    "cliffs_read_maxwave", "cliffs_read_boundary", "cliffs_read_state", "cliffs_kernel_time",
    "cliffs_destroy", "cliffs_last_error", "cliffs_abi_version", "cliffs_depth_filter_noalloc",
    "cliffs_inject_wait_expiry", "cliffs_autotune", "cliffs_run_persistent", "cliffs_adjoint_n",
    "cliffs_set_boundary_input", "cliffs_set_boundary_clock", "cliffs_set_initial_interp",
    "cliffs_adjoint_record", "cliffs_adjoint_recorded", "cliffs_state_ptrs", "cliffs_adjoint_velocity",
    "cliffs_adjoint_scenario", "cliffs_set_rows_per_warp", "cliffs_adjoint_records",
    "cliffs_adjoint_recorded_records", "cliffs_adjoint_recorded_scenario", "cliffs_diagnostics",
    "EXPORTED",
]

OK, ERR_ARG, ERR_STATE, ERR_CUDA, ERR_UNSTABLE, ERR_TIMEOUT, ERR_NOMEM = 0, -1, -2, -3, -4, -5, -6
EDGE_WEST, EDGE_EAST, EDGE_SOUTH, EDGE_NORTH = 0, 1, 2, 3

# every function include/cliffs.h declares
EXPORTED = [
    "cliffs_grid_create", "cliffs_set_bathy", "cliffs_read_depth", "cliffs_set_initial",
    "cliffs_set_durations", "cliffs_step_n", "cliffs_steps_done", "cliffs_read_gauges",
    "cliffs_read_maxwave", "cliffs_read_boundary", "cliffs_read_state", "cliffs_kernel_time",
    "cliffs_destroy", "cliffs_last_error", "cliffs_abi_version", "cliffs_depth_filter_noalloc",
    "cliffs_inject_wait_expiry", "cliffs_autotune", "cliffs_run_persistent", "cliffs_adjoint_n",
    "cliffs_set_boundary_input", "cliffs_set_boundary_clock", "cliffs_set_initial_interp",
    "cliffs_adjoint_record", "cliffs_adjoint_recorded", "cliffs_state_ptrs", "cliffs_adjoint_velocity",
    "cliffs_adjoint_scenario", "cliffs_set_rows_per_warp", "cliffs_adjoint_records",
    "cliffs_adjoint_recorded_records", "cliffs_adjoint_recorded_scenario", "cliffs_diagnostics",
]


class CliffsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("cliffs error %d: %s" % (code, msg))
        self.code = code


class cliffs_nest(C.Structure):
    _fields_ = [("x0", C.c_double), ("y0", C.c_double), ("dx", C.c_double), ("dy", C.c_double),
                ("nx", C.c_int32), ("ny", C.c_int32)]


class cliffs_config(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("batch", C.c_int32), ("coords", C.c_int32),
                ("h_min", C.c_double), ("manning_n2", C.c_double),
                ("itopo", C.c_int32), ("dwall", C.c_double), ("dt", C.c_double),
                ("transverse", C.c_int32), ("solver", C.c_int32), ("alternate", C.c_int32),
                ("maxout", C.c_int32), ("gout", C.c_int32), ("bndout", C.c_int32),
                ("n_gauges", C.c_int32), ("gauge_ixiy", C.POINTER(C.c_int32)),
                ("n_nests", C.c_int32), ("nests", C.POINTER(cliffs_nest)),
                ("stream", C.c_void_p), ("open_edges", C.c_int32)]


_lib = None


def lib():
    """Load libcliffs.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError("libcliffs.so is not built; run paper_1410_0753_gb300._build.build() "
                               "(or __graft_entry__.build()) on a machine with nvcc")
        L = C.CDLL(_build.LIB)
        P, vp, i64p = C.POINTER, C.c_void_p, C.POINTER(C.c_int64)
        sig = {
            "cliffs_grid_create": ([P(cliffs_config), P(vp)], C.c_int),
            "cliffs_set_bathy": ([vp, vp, vp, vp, C.c_int, C.c_double, C.c_double], C.c_int),
            "cliffs_read_depth": ([vp, vp], C.c_int),
            "cliffs_set_initial": ([vp, C.c_int, vp, vp, vp, C.c_int], C.c_int),
            "cliffs_set_durations": ([vp, vp], C.c_int),
            "cliffs_step_n": ([vp, C.c_int64], C.c_int),
            "cliffs_run_persistent": ([vp, C.c_int64], C.c_int),
            "cliffs_adjoint_n": ([vp, C.c_int64, C.c_int32, vp, vp], C.c_int),
            "cliffs_adjoint_scenario": ([vp, C.c_int32, C.c_int64, C.c_int32, vp, vp], C.c_int),
            "cliffs_set_rows_per_warp": ([vp, C.c_int32], C.c_int),
            "cliffs_adjoint_records": ([vp, C.c_int32, C.c_int64, C.c_int32, vp, vp], C.c_int),
            "cliffs_adjoint_recorded_records": ([vp, vp, vp], C.c_int),
            "cliffs_adjoint_recorded_scenario": ([vp, C.c_int32, C.c_int32, vp, vp], C.c_int),
            "cliffs_diagnostics": ([vp, C.c_int, vp], C.c_int),
            "cliffs_adjoint_record": ([vp, C.c_int32], C.c_int),
            "cliffs_state_ptrs": ([vp, C.c_int, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp),
                                   C.POINTER(C.c_int64)], C.c_int),
            "cliffs_adjoint_recorded": ([vp, vp, vp], C.c_int),
            "cliffs_adjoint_velocity": ([vp, vp, vp], C.c_int),
            "cliffs_set_boundary_input": ([vp, C.c_int, vp, C.c_int64, vp], C.c_int),
            "cliffs_set_boundary_clock": ([vp, C.c_double, C.c_int, C.POINTER(C.c_double)], C.c_int),
            "cliffs_set_initial_interp": ([vp, C.c_int, vp, C.c_int32, vp, C.c_int32, vp, vp, vp, C.c_int], C.c_int),
            "cliffs_steps_done": ([vp, i64p], C.c_int),
            "cliffs_read_gauges": ([vp, C.c_int, vp, i64p], C.c_int),
            "cliffs_read_maxwave": ([vp, C.c_int, vp, vp], C.c_int),
            "cliffs_read_boundary": ([vp, C.c_int, C.c_int, vp, i64p], C.c_int),
            "cliffs_read_state": ([vp, C.c_int, vp, vp, vp], C.c_int),
            "cliffs_kernel_time": ([vp, C.c_int, P(C.c_double), i64p], C.c_int),
            "cliffs_destroy": ([vp], None),
            "cliffs_last_error": ([], C.c_char_p),
            "cliffs_abi_version": ([], C.c_int),
            "cliffs_depth_filter_noalloc": ([vp, vp, C.c_int32, C.c_int32, C.c_double, C.c_double,
                                             vp, C.POINTER(C.c_int32)], C.c_int),
            "cliffs_inject_wait_expiry": ([vp, C.c_int64], C.c_int),
            "cliffs_autotune": ([vp, C.c_int, vp, vp, C.POINTER(C.c_int32)], C.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def cliffs_last_error() -> str:
    return lib().cliffs_last_error().decode()


def cliffs_abi_version() -> int:
    return lib().cliffs_abi_version()


def _check(rc):
    if rc != OK:
        raise CliffsError(rc, cliffs_last_error())


def _ptr(a, dtype):
    """(pointer, keep-alive) for a NumPy array (host) or a torch tensor (host or CUDA)."""
    if a is None:
        return None, None
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        import torch
        want = {np.float32: torch.float32, np.float64: torch.float64, np.int64: torch.int64,
                np.int32: torch.int32}[dtype]
        t = a.contiguous()
        if t.dtype != want:
            t = t.to(want)
        return C.c_void_p(t.data_ptr()), t
    arr = np.ascontiguousarray(a, dtype=dtype)
    return C.c_void_p(arr.ctypes.data), arr


# ------------------------------------------------------------------ C ABI, same names

def cliffs_grid_create(cfg: cliffs_config) -> C.c_void_p:
    h = C.c_void_p()
    _check(lib().cliffs_grid_create(C.byref(cfg), C.byref(h)))
    return h


def cliffs_set_bathy(g, x, y, depth, apply_filter=1, alpha=2.0, min_depth=0.1):
    px, kx = _ptr(x, np.float64)
    py, ky = _ptr(y, np.float64)
    pd, kd = _ptr(depth, np.float64)
    _check(lib().cliffs_set_bathy(g, px, py, pd, int(apply_filter), float(alpha), float(min_depth)))


def cliffs_read_depth(g, out):
    _check(lib().cliffs_read_depth(g, _out_ptr(out)))


def cliffs_set_initial(g, scenario, eta, u=None, v=None, quake=0):
    pe, ke = _ptr(eta, np.float32)
    pu, ku = _ptr(u, np.float32)
    pv, kv = _ptr(v, np.float32)
    _check(lib().cliffs_set_initial(g, int(scenario), pe, pu, pv, int(quake)))


def cliffs_set_initial_interp(g, scenario, sx, sy, eta, u=None, v=None, quake=0):
    px, kx = _ptr(sx, np.float64)
    py, ky = _ptr(sy, np.float64)
    pe, ke = _ptr(eta, np.float32)
    pu, ku = _ptr(u, np.float32)
    pv, kv = _ptr(v, np.float32)
    _check(lib().cliffs_set_initial_interp(g, int(scenario), px, len(sx), py, len(sy), pe, pu, pv, int(quake)))


def cliffs_set_durations(g, steps):
    p, k = _ptr(steps, np.int64)
    _check(lib().cliffs_set_durations(g, p))


def cliffs_step_n(g, n):
    _check(lib().cliffs_step_n(g, int(n)))


def cliffs_run_persistent(g, n):
    _check(lib().cliffs_run_persistent(g, int(n)))


def cliffs_steps_done(g) -> int:
    n = C.c_int64()
    _check(lib().cliffs_steps_done(g, C.byref(n)))
    return n.value


def _out_ptr(out):
    if out is None:
        return None
    if isinstance(out, np.ndarray):
        assert out.flags.c_contiguous
        return C.c_void_p(out.ctypes.data)
    return C.c_void_p(out.data_ptr())


def cliffs_adjoint_n(g, n, checkpoint_every, dL_dgauges, out):
    """dL/d eta_0 into ``out`` ([ny][nx] float32, NumPy or torch, host or CUDA) for the
    gauge-eta adjoint seed ``dL_dgauges`` ([n // gout + 1][G] float32, or None)."""
    ps, ks = _ptr(dL_dgauges, np.float32)
    _check(lib().cliffs_adjoint_n(g, int(n), int(checkpoint_every), ps, _out_ptr(out)))


def cliffs_adjoint_scenario(g, scenario, n, checkpoint_every, dL_dgauges, out):
    """cliffs_adjoint_n for one scenario of a batched grid."""
    ps, ks = _ptr(dL_dgauges, np.float32)
    _check(lib().cliffs_adjoint_scenario(g, int(scenario), int(n), int(checkpoint_every), ps, _out_ptr(out)))


def cliffs_adjoint_records(g, scenario, n, checkpoint_every, dL_drecords, out):
    """The adjoint for dL/d (eta, u, v) of the gauge records ([n // gout + 1][G][3])."""
    ps, ks = _ptr(dL_drecords, np.float32)
    _check(lib().cliffs_adjoint_records(g, int(scenario), int(n), int(checkpoint_every), ps, _out_ptr(out)))


def cliffs_adjoint_recorded_records(g, dL_drecords, out):
    ps, ks = _ptr(dL_drecords, np.float32)
    _check(lib().cliffs_adjoint_recorded_records(g, ps, _out_ptr(out)))


def cliffs_adjoint_recorded_scenario(g, scenario, components, dL, out):
    ps, ks = _ptr(dL, np.float32)
    _check(lib().cliffs_adjoint_recorded_scenario(g, int(scenario), int(components), ps, _out_ptr(out)))


def cliffs_diagnostics(g, scenario=0):
    """(volume m^3, wet nodes, max |eta| m, max speed m/s) of the current state over wet nodes."""
    out = np.zeros(4, np.float64)
    _check(lib().cliffs_diagnostics(g, int(scenario), C.c_void_p(out.ctypes.data)))
    return dict(volume=float(out[0]), wet=int(out[1]), eta_abs_max=float(out[2]), speed_max=float(out[3]))


def cliffs_state_ptrs(g, scenario):
    """(eta, u, v device addresses, pitch in floats) of a scenario's current state."""
    e, u, v = C.c_void_p(), C.c_void_p(), C.c_void_p()
    p = C.c_int64()
    _check(lib().cliffs_state_ptrs(g, int(scenario), C.byref(e), C.byref(u), C.byref(v), C.byref(p)))
    return e.value, u.value, v.value, p.value


class _DeviceArray:
    """A [ny][nx] FP32 view of library-owned device memory (CUDA array interface)."""

    def __init__(self, ptr, ny, nx, pitch, owner):
        self.__cuda_array_interface__ = {"shape": (ny, nx), "strides": (4 * pitch, 4), "typestr": "<f4",
                                         "data": (ptr, False), "version": 2}
        self.owner = owner


def cliffs_adjoint_record(g, checkpoint_every):
    _check(lib().cliffs_adjoint_record(g, int(checkpoint_every)))


def cliffs_adjoint_recorded(g, dL_dgauges, out):
    ps, ks = _ptr(dL_dgauges, np.float32)
    _check(lib().cliffs_adjoint_recorded(g, ps, _out_ptr(out)))


def cliffs_adjoint_velocity(g, du=None, dv=None):
    _check(lib().cliffs_adjoint_velocity(g, _out_ptr(du), _out_ptr(dv)))


def cliffs_set_boundary_input(g, edge, times, vals):
    """Boundary input of one edge (0 W, 1 E, 2 S, 3 N): times[nt], vals[nt][3][np] (u, v, eta);
    times=None removes it."""
    if times is None:
        _check(lib().cliffs_set_boundary_input(g, int(edge), None, 0, None))
        return
    pt, kt = _ptr(times, np.float64)
    pv, kv = _ptr(vals, np.float64)
    _check(lib().cliffs_set_boundary_input(g, int(edge), pt, len(times), pv))


def cliffs_set_boundary_clock(g, cuke=0.0, stop_at_end=0) -> float:
    t = C.c_double()
    _check(lib().cliffs_set_boundary_clock(g, float(cuke), int(stop_at_end), C.byref(t)))
    return t.value


def cliffs_read_gauges(g, scenario, out=None) -> int:
    n = C.c_int64()
    _check(lib().cliffs_read_gauges(g, int(scenario), _out_ptr(out), C.byref(n)))
    return n.value


def cliffs_read_maxwave(g, scenario, eta_max=None, speed_max=None):
    _check(lib().cliffs_read_maxwave(g, int(scenario), _out_ptr(eta_max), _out_ptr(speed_max)))


def cliffs_read_boundary(g, nest, edge, vals=None) -> int:
    n = C.c_int64()
    _check(lib().cliffs_read_boundary(g, int(nest), int(edge), _out_ptr(vals), C.byref(n)))
    return n.value


def cliffs_read_state(g, scenario, eta=None, u=None, v=None):
    _check(lib().cliffs_read_state(g, int(scenario), _out_ptr(eta), _out_ptr(u), _out_ptr(v)))


def cliffs_kernel_time(g, enable):
    ms = C.c_double()
    n = C.c_int64()
    _check(lib().cliffs_kernel_time(g, int(enable), C.byref(ms), C.byref(n)))
    return ms.value, n.value


def cliffs_depth_filter_noalloc(depth, out, nx, ny, alpha=2.0, min_depth=0.1, stream=None) -> int:
    """Depth filter into caller-owned device memory ``out`` with no device allocation (see
    include/cliffs.h). ``out`` must be a contiguous CUDA float64 tensor of nx * ny elements;
    ``depth`` may be host (NumPy) or device data. An in-place call (``out`` is ``depth``)
    needs ``depth`` to be that same contiguous CUDA float64 tensor: a converted copy would be
    filtered instead of the caller's array. Returns the passes made."""
    import torch
    n_cells = int(nx) * int(ny)
    if not (isinstance(out, torch.Tensor) and out.is_cuda and out.dtype == torch.float64
            and out.is_contiguous() and out.numel() == n_cells):
        raise CliffsError(ERR_ARG, "out must be a contiguous CUDA float64 tensor of nx * ny = %d "
                                   "elements" % n_cells)
    if isinstance(depth, torch.Tensor) and depth.data_ptr() == out.data_ptr():
        if not (depth.is_cuda and depth.dtype == torch.float64 and depth.is_contiguous()):
            raise CliffsError(ERR_ARG, "an in-place call needs depth to be out itself")
    elif (depth.numel() if isinstance(depth, torch.Tensor) else np.size(depth)) != n_cells:
        raise CliffsError(ERR_ARG, "depth must have nx * ny = %d elements" % n_cells)
    pd, kd = _ptr(depth, np.float64)
    n = C.c_int32()
    _check(lib().cliffs_depth_filter_noalloc(pd, C.c_void_p(out.data_ptr()), int(nx), int(ny), float(alpha),
                                             float(min_depth), C.c_void_p(stream) if stream else None,
                                             C.byref(n)))
    return n.value


def cliffs_autotune(g, trials=3):
    """Time the candidate tile shapes on the current state and keep the fastest; returns
    {rows_per_warp: microseconds}."""
    cand = np.zeros(16, np.int32)
    us = np.zeros(16, np.float64)
    n = C.c_int32()
    _check(lib().cliffs_autotune(g, int(trials), C.c_void_p(cand.ctypes.data),
                                 C.c_void_p(us.ctypes.data), C.byref(n)))
    return {int(cand[i]): float(us[i]) for i in range(n.value)}


def cliffs_set_rows_per_warp(g, rows):
    _check(lib().cliffs_set_rows_per_warp(g, int(rows)))


def cliffs_inject_wait_expiry(g, cycles):
    _check(lib().cliffs_inject_wait_expiry(g, int(cycles)))


def cliffs_destroy(g):
    if g:
        lib().cliffs_destroy(g)


# ------------------------------------------------------------------ convenience wrapper

class CliffsGrid:
    """One grid (optionally a batch of scenarios on shared bathymetry).

    Parameters mirror ``cliffs_config``; ``gauges`` is a sequence of (ix, iy); ``nests`` a
    sequence of objects with x0, y0, dx, dy, nx, ny."""

    def __init__(self, nx, ny, dt, *, batch=1, coords=1, h_min=0.01, manning_n2=0.0, itopo=1,
                 dwall=0.0, transverse=1, solver=2, alternate=0, maxout=1, gout=1, bndout=1,
                 gauges: Sequence = (), nests: Sequence = (), stream: Optional[int] = None,
                 open_edges=0):
        g = np.ascontiguousarray(np.asarray(gauges, np.int32).reshape(-1))
        self._gauges = g
        ns = (cliffs_nest * max(1, len(nests)))()
        for k, n in enumerate(nests):
            ns[k] = cliffs_nest(n.x0, n.y0, n.dx, n.dy, n.nx, n.ny)
        self._nests = ns
        cfg = cliffs_config(nx, ny, batch, coords, h_min, manning_n2, itopo, dwall, dt, transverse,
                            solver, alternate, maxout, gout, bndout, len(g) // 2,
                            g.ctypes.data_as(C.POINTER(C.c_int32)) if len(g) else None,
                            len(nests), ns if len(nests) else None,
                            C.c_void_p(stream) if stream else None, int(open_edges))
        self.cfg = cfg
        self.nx, self.ny, self.batch = nx, ny, batch
        self.n_gauges = len(g) // 2
        self.run_id = 0                 # changes with every set_initial and step through this object
        self.nest_shapes = [(n.nx, n.ny) for n in nests]
        self.h = cliffs_grid_create(cfg)

    @classmethod
    def from_workload(cls, w, stream=None, **kw):
        opts = dict(batch=w.batch, coords=w.coords, h_min=w.h_min, manning_n2=w.manning_n2,
                    itopo=w.itopo, dwall=w.dwall, transverse=w.transverse, maxout=w.maxout,
                    gout=w.gout, bndout=w.bndout, gauges=[tuple(x) for x in w.gauges],
                    nests=w.nests, stream=stream)
        opts.update(kw)
        return cls(w.nx, w.ny, w.dt, **opts)

    def close(self):
        if self.h:
            cliffs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_bathy(self, x, y, depth, apply_filter=True, alpha=2.0, min_depth=0.1):
        cliffs_set_bathy(self.h, x, y, depth, int(apply_filter), alpha, min_depth)

    def depth(self):
        out = np.empty((self.ny, self.nx), np.float64)
        cliffs_read_depth(self.h, out)
        return out

    def set_initial(self, eta, u=None, v=None, scenario=-1, quake=0):
        cliffs_set_initial(self.h, scenario, eta, u, v, quake)
        self.run_id += 1

    def set_initial_interp(self, sx, sy, eta, u=None, v=None, scenario=-1, quake=0):
        cliffs_set_initial_interp(self.h, scenario, sx, sy, eta, u, v, quake)
        self.run_id += 1

    def set_durations(self, steps):
        cliffs_set_durations(self.h, steps)

    def step(self, n, persistent=False):
        """Advance n steps: one launch per step, or (persistent=True) all n in one
        persistent, graph-captured launch with identical results."""
        self.run_id += 1
        if persistent:
            cliffs_run_persistent(self.h, n)
        else:
            cliffs_step_n(self.h, n)

    @property
    def steps_done(self):
        return cliffs_steps_done(self.h)

    def gauges(self, scenario=0):
        n = cliffs_read_gauges(self.h, scenario)
        out = np.empty((n, self.n_gauges, 3), np.float32)
        if n and self.n_gauges:
            cliffs_read_gauges(self.h, scenario, out)
        return out

    def diagnostics(self, scenario=0):
        return cliffs_diagnostics(self.h, scenario)

    def maxwave(self, scenario=0):
        e = np.empty((self.ny, self.nx), np.float32)
        s = np.empty((self.ny, self.nx), np.float32)
        cliffs_read_maxwave(self.h, scenario, e, s)
        return e, s

    def boundary(self, nest, edge):
        n = cliffs_read_boundary(self.h, nest, edge)
        nxn, nyn = self.nest_shapes[nest]
        np_ = nyn if edge in (EDGE_WEST, EDGE_EAST) else nxn
        out = np.empty((n, 3, np_), np.float64)
        cliffs_read_boundary(self.h, nest, edge, out)
        return out

    def state(self, scenario=0):
        e = np.empty((self.ny, self.nx), np.float32)
        u = np.empty_like(e)
        v = np.empty_like(e)
        cliffs_read_state(self.h, scenario, e, u, v)
        return e, u, v

    def state_views(self, scenario=0):
        """Zero-copy torch views (eta, u, v) of the current state on the device, [ny][nx] with
        row stride pitch; valid until the next step or set_initial (the state buffers
        alternate)."""
        import torch
        e, u, v, p = cliffs_state_ptrs(self.h, scenario)
        return tuple(torch.as_tensor(_DeviceArray(a, self.ny, self.nx, p, self), device="cuda") for a in (e, u, v))

    def kernel_time(self, enable=1):
        return cliffs_kernel_time(self.h, enable)

    def set_rows_per_warp(self, rows):
        cliffs_set_rows_per_warp(self.h, rows)

    def autotune(self, trials=3):
        return cliffs_autotune(self.h, trials)

    def set_boundary_input(self, edge, times, vals):
        cliffs_set_boundary_input(self.h, edge, times, vals)

    def set_boundary_clock(self, cuke=0.0, stop_at_end=False):
        return cliffs_set_boundary_clock(self.h, cuke, int(stop_at_end))

    def adjoint_record(self, checkpoint_every=100):
        """Keep checkpoints of the run from the current initial state (0 stops recording)."""
        cliffs_adjoint_record(self.h, checkpoint_every)

    def adjoint_recorded(self, dL_dgauges, out=None, scenario=0):
        """Gradient for the run recorded since the last set_initial (see adjoint)."""
        if out is None:
            out = np.empty((self.ny, self.nx), np.float32)
        comps = 3 if dL_dgauges is not None and len(getattr(dL_dgauges, "shape", ())) == 3 else 1
        cliffs_adjoint_recorded_scenario(self.h, scenario, comps, dL_dgauges, out)
        return out

    def adjoint_velocity(self):
        """(dL/du0, dL/dv0) of the last adjoint call."""
        du = np.empty((self.ny, self.nx), np.float32)
        dv = np.empty_like(du)
        cliffs_adjoint_velocity(self.h, du, dv)
        return du, dv

    def adjoint(self, n, dL_dgauges, checkpoint_every=100, out=None, scenario=0):
        """Gradient with respect to the current free surface of a loss whose derivative with
        respect to the gauge eta records of the next n steps is ``dL_dgauges`` (of scenario
        ``scenario`` on a batched grid)."""
        if out is None:
            out = np.empty((self.ny, self.nx), np.float32)
        if dL_dgauges is not None and len(getattr(dL_dgauges, "shape", ())) == 3:   # [nrec][G][3]
            cliffs_adjoint_records(self.h, scenario, n, checkpoint_every, dL_dgauges, out)
        else:
            cliffs_adjoint_scenario(self.h, scenario, n, checkpoint_every, dL_dgauges, out)
        return out
