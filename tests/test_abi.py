"""The C ABI (no GPU needed): libcliffs.so builds for sm_103a, loads, exports every function
include/cliffs.h declares, and the ctypes structures match the C layout."""
import ctypes as C
import os
import re
import subprocess

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
