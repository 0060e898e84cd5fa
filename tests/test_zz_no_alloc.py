"""The allocation-free depth filter, cliffs_depth_filter_noalloc, on the GPU.

Some callers of this library cannot allocate device memory when they call it: applications
whose own memory pool owns the whole device and forbids allocations behind its back, and
callers that cannot afford the device-wide synchronisation of cudaFree. For them the library
filters bathymetry into memory the caller owns, using a fixed static scratch array instead of
allocating. Its result must equal the allocating path's (cliffs_set_bathy) bit for bit, the
tolerance every depth-filter test here uses, on consecutive calls that reuse the one scratch
array. Arguments it cannot use are refused before anything is launched.
"""
import ctypes as C

import numpy as np
import pytest

import paper_1410_0753_gb300 as pk
from paper_1410_0753_gb300 import CliffsError, CliffsGrid, ERR_ARG, _build

pytestmark = pytest.mark.gpu


def spiky(seed, ny, nx):
    rng = np.random.default_rng(seed)
    d = 50.0 + 40.0 * rng.standard_normal((ny, nx))
    d[rng.random(d.shape) < 0.05] = 0.05
    d[:, :5] = -2.0
    d[ny // 3: ny // 3 + 8, nx // 2: nx // 2 + 9] = -1.0
    return d


def filtered_by_set_bathy(d):
    ny, nx = d.shape
    g = CliffsGrid(nx, ny, 0.01)
    g.set_bathy(np.arange(nx) * 100.0, np.arange(ny) * 100.0, d, True, 2.0, 0.1)
    out = g.depth()
    g.close()
    return out


def test_noalloc_filter_equals_set_bathy_on_consecutive_calls():
    import torch
    assert torch.cuda.is_available(), "needs a CUDA device"
    _build.build()
    stream = torch.cuda.current_stream().cuda_stream
    cases = [spiky(11, 97, 131), spiky(12, 150, 80)]
    for d in cases + cases[::-1]:                       # back-to-back calls share the scratch
        want = filtered_by_set_bathy(d)
        dev_in = torch.from_numpy(d).cuda()
        dev_out = torch.full_like(dev_in, float("nan"))
        passes = pk.cliffs_depth_filter_noalloc(dev_in, dev_out, d.shape[1], d.shape[0], 2.0, 0.1, stream)
        assert passes > 1
        assert np.array_equal(dev_out.cpu().numpy(), want)
        assert np.array_equal(dev_in.cpu().numpy(), d)  # the input is left alone
    # host input, device output; and in place on the device
    d = cases[0]
    want = filtered_by_set_bathy(d)
    dev_out = torch.empty(d.shape, dtype=torch.float64, device="cuda")
    pk.cliffs_depth_filter_noalloc(d, dev_out, d.shape[1], d.shape[0], 2.0, 0.1, stream)
    assert np.array_equal(dev_out.cpu().numpy(), want)
    inplace = torch.from_numpy(d).cuda()
    pk.cliffs_depth_filter_noalloc(inplace, inplace, d.shape[1], d.shape[0], 2.0, 0.1, stream)
    assert np.array_equal(inplace.cpu().numpy(), want)


def test_noalloc_filter_rejects_grids_beyond_its_scratch():
    import torch
    _build.build()
    n = 1025                                            # 1,050,625 nodes > 2^20
    dev = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    with pytest.raises(CliffsError) as e:
        pk.cliffs_depth_filter_noalloc(dev, dev, n, n, 2.0, 0.1)
    assert e.value.code == ERR_ARG and "at most 1048576" in str(e.value)


def test_noalloc_filter_refuses_unusable_outputs_before_launching():
    """The C entry point itself refuses a host output and partly overlapping arrays (checked
    with the runtime's pointer attributes, before any launch); the Python wrapper refuses
    outputs of the wrong kind, type or size, and an in-place call on a converted copy."""
    import torch
    _build.build()
    d = spiky(13, 40, 50)
    ny, nx = d.shape
    L = pk.lib()
    host_out = np.zeros_like(d)
    rc = L.cliffs_depth_filter_noalloc(C.c_void_p(d.ctypes.data), C.c_void_p(host_out.ctypes.data), nx, ny,
                                       2.0, 0.1, None, None)
    assert rc == ERR_ARG and "device memory" in pk.cliffs_last_error()
    assert np.all(host_out == 0.0)
    buf = torch.zeros(2 * d.size, dtype=torch.float64, device="cuda")
    rc = L.cliffs_depth_filter_noalloc(C.c_void_p(buf.data_ptr()), C.c_void_p(buf.data_ptr() + 8 * 100), nx, ny,
                                       2.0, 0.1, None, None)
    assert rc == ERR_ARG and "overlap" in pk.cliffs_last_error()
    assert torch.count_nonzero(buf).item() == 0
    bad_outs = [host_out, torch.zeros(d.shape, dtype=torch.float32, device="cuda"),
                torch.zeros((ny, nx + 1), dtype=torch.float64, device="cuda"),
                torch.zeros((nx, ny), dtype=torch.float64, device="cuda").t(),
                torch.zeros(d.shape, dtype=torch.float64)]
    for out in bad_outs:
        with pytest.raises(CliffsError) as e:
            pk.cliffs_depth_filter_noalloc(d, out, nx, ny)
        assert e.value.code == ERR_ARG
    f32 = torch.from_numpy(d.astype(np.float32)).cuda()
    with pytest.raises(CliffsError):
        pk.cliffs_depth_filter_noalloc(f32, f32, nx, ny)
