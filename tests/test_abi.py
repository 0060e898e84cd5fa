"""The C ABI (no GPU needed): libcliffs.so builds for sm_103a, loads, exports every function
include/cliffs.h declares, and the ctypes structures match the C layout."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

import paper_1410_0753_gb300 as pk
from paper_1410_0753_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cliffs.h")


@pytest.fixture(scope="module")
def built():
    return _build.build()


def declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\s*\*)\s+(cliffs_\w+)\s*\(", txt, re.M)))


def test_every_declared_symbol_is_exported(built):
    names = declared()
    assert len(names) >= 15
    L = C.CDLL(built)
    for n in names:
        assert hasattr(L, n), n
    assert sorted(pk.EXPORTED) == names                 # the binding covers the whole ABI
    nm = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True).stdout
    for n in names:
        assert re.search(r"\bT %s$" % n, nm, re.M), n


def test_abi_version_without_gpu(built):
    assert pk.cliffs_abi_version() == 2
    assert pk.cliffs_last_error() == ""


def test_struct_layout_matches_c(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "cliffs.h"
#define F(T, m) printf(#T "." #m " %zu\n", offsetof(T, m))
int main(void) {
  printf("cliffs_config %zu\n", sizeof(cliffs_config));
  printf("cliffs_nest %zu\n", sizeof(cliffs_nest));
  F(cliffs_config, nx); F(cliffs_config, ny); F(cliffs_config, batch); F(cliffs_config, coords);
  F(cliffs_config, h_min); F(cliffs_config, manning_n2); F(cliffs_config, itopo);
  F(cliffs_config, dwall); F(cliffs_config, dt); F(cliffs_config, transverse);
  F(cliffs_config, solver); F(cliffs_config, alternate); F(cliffs_config, maxout);
  F(cliffs_config, gout); F(cliffs_config, bndout); F(cliffs_config, n_gauges);
  F(cliffs_config, gauge_ixiy); F(cliffs_config, n_nests); F(cliffs_config, nests);
  F(cliffs_config, stream); F(cliffs_config, open_edges);
  F(cliffs_nest, x0); F(cliffs_nest, y0); F(cliffs_nest, dx); F(cliffs_nest, dy);
  F(cliffs_nest, nx); F(cliffs_nest, ny);
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = dict(l.rsplit(" ", 1) for l in out.strip().splitlines())
    assert int(got["cliffs_config"]) == C.sizeof(pk.cliffs_config)
    assert int(got["cliffs_nest"]) == C.sizeof(pk.cliffs_nest)
    for T, cls in (("cliffs_config", pk.cliffs_config), ("cliffs_nest", pk.cliffs_nest)):
        for name, _ in cls._fields_:
            assert int(got["%s.%s" % (T, name)]) == getattr(cls, name).offset, (T, name)


def test_loading_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(pk, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        pk.lib()


# Argument checks that return before any CUDA call (host logic; nothing is launched).
BAD_GRIDS = [
    (dict(nx=0, ny=10), "need nx, ny >= 1"),
    (dict(nx=10, ny=0), "need nx, ny >= 1"),
    (dict(nx=1, ny=1), "not both 1"),
    (dict(nx=2, ny=10), "at least 3 nodes"),
    (dict(nx=10, ny=2), "at least 3 nodes"),
    (dict(batch=0), "batch"),
    (dict(h_min=0.0), "h_min"),
    (dict(dt=0.0), "dt"),
    (dict(manning_n2=-1e-4), "manning_n2"),
    (dict(maxout=0), "maxout"),
    (dict(gout=0), "maxout, gout and bndout"),
    (dict(solver=3), "solver"),
    (dict(open_edges=16), "open_edges"),
    (dict(alternate=2), "alternate"),
    (dict(gauges=[(10, 3)]), "outside the 10 x 8 grid"),
    (dict(gauges=[(3, -1)]), "outside the 10 x 8 grid"),
    (dict(nx=10, ny=1, nests=[pk.cliffs_nest(0.0, 0.0, 1.0, 1.0, 3, 3)]), "2D master grid"),
    (dict(batch=2, nests=[pk.cliffs_nest(0.0, 0.0, 1.0, 1.0, 3, 3)]), "batch == 1"),
    (dict(nests=[pk.cliffs_nest(0.0, 0.0, 1.0, 1.0, 1, 3)]), "nest 0"),
]


@pytest.mark.parametrize("kw,msg", BAD_GRIDS, ids=[m for _, m in BAD_GRIDS])
def test_grid_create_rejects_bad_arguments_on_the_host(built, kw, msg):
    kw = dict(kw)
    nx, ny, dt = kw.pop("nx", 10), kw.pop("ny", 8), kw.pop("dt", 1.0)
    with pytest.raises(pk.CliffsError) as e:
        pk.CliffsGrid(nx, ny, dt, **kw)
    assert e.value.code == pk.ERR_ARG
    assert msg in str(e.value) and msg in pk.cliffs_last_error()


def test_null_handles_are_argument_errors(built):
    out = (C.c_double * 4)()
    L = pk.lib()
    for rc in (L.cliffs_step_n(None, 1), L.cliffs_run_persistent(None, 1),
               L.cliffs_read_state(None, 0, None, None, None),
               L.cliffs_read_maxwave(None, 0, None, None),
               L.cliffs_diagnostics(None, 0, out), L.cliffs_set_durations(None, None),
               L.cliffs_adjoint_n(None, 1, 1, None, None), L.cliffs_grid_create(None, None)):
        assert rc == pk.ERR_ARG
    assert "null" in pk.cliffs_last_error()
    pk.lib().cliffs_destroy(None)                       # destroying nothing is a no-op


def test_noalloc_filter_wrapper_refuses_bad_outputs_on_the_host(built):
    """The allocation-free filter's binding refuses outputs it cannot write (host memory, a
    CPU tensor, the wrong type or size) before calling into the library; the C entry point's
    own NULL and size checks run without touching a GPU."""
    import torch
    d = np.full((6, 5), 10.0)
    for out in (np.zeros((6, 5)), torch.zeros((6, 5), dtype=torch.float64),
                torch.zeros((6, 5), dtype=torch.float32)):
        with pytest.raises(pk.CliffsError) as e:
            pk.cliffs_depth_filter_noalloc(d, out, 5, 6)
        assert e.value.code == pk.ERR_ARG and "CUDA float64" in str(e.value)
    L = pk.lib()
    assert L.cliffs_depth_filter_noalloc(None, None, 5, 6, 2.0, 0.1, None, None) == pk.ERR_ARG
    buf = (C.c_double * 30)()
    assert L.cliffs_depth_filter_noalloc(buf, buf, 0, 6, 2.0, 0.1, None, None) == pk.ERR_ARG
    assert L.cliffs_depth_filter_noalloc(buf, buf, 2048, 2048, 2.0, 0.1, None, None) == pk.ERR_ARG
    assert "at most 1048576" in pk.cliffs_last_error()
