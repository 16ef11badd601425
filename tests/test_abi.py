"""The C-ABI library builds, loads and exports every entry point declared in
include/bdg.h; argument checks answer with status codes without touching a GPU."""
import ctypes
import os
import re

import pytest

import paper_2102_04656_b300 as bdg
from paper_2102_04656_b300 import build as bdg_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[\w\s\*]*?\b(bdg_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def L():
    bdg_build.build()
    return bdg.lib()


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert "bdg_build_graph" in names and "bdg_search" in names
    for n in names:
        assert hasattr(L, n), n


def test_argument_checks_return_status_codes(L):
    # no device work is enqueued for invalid arguments
    assert L.bdg_route(None, 10, 100, None, 4, 2, None, None, None) == -1   # bits % 64
    assert L.bdg_route(None, 10, 192, None, 4, 2, None, None, None) == -1   # W = 3
    assert L.bdg_route(None, 10, 256, None, 4, 5, None, None, None) == -1   # t > m
    out = ctypes.c_void_p()
    P = bdg._Partitions()
    P.m, P.t = 4, 2
    assert L.bdg_build_graph(ctypes.c_void_p(16), 1, 256, 4, ctypes.byref(P), None,
                             ctypes.byref(out)) == -1  # N < 2
    assert L.bdg_build_graph(ctypes.c_void_p(16), 100, 256, 200, ctypes.byref(P), None,
                             ctypes.byref(out)) == -1  # k > 128
    assert b"k = 200" in L.bdg_last_error()
    assert L.bdg_build_graph(ctypes.c_void_p(16), 100, 256, 8, ctypes.byref(P), None,
                             ctypes.byref(out)) == -1  # no entry sample
    assert L.bdg_rerank(None, 10, 100, None, None, 1, 10, 5, None, None, None) == -5  # D
    assert L.bdg_search(None, None, 1, None, 64, 10, None, None, None, None) == -1


def test_memory_budget_roundtrip(L):
    bdg.set_memory_budget(1 << 30)
    assert bdg.memory_in_use() == 0
    bdg.set_memory_budget(0)


def test_load_rejects_bad_files(L, tmp_path):
    p = tmp_path / "bad.bdg"
    p.write_bytes(b"not a graph")
    out = ctypes.c_void_p()
    assert L.bdg_graph_load(str(p).encode(), ctypes.c_void_p(16), ctypes.byref(out)) == -1
