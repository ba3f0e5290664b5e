"""The C ABI library builds, loads and exports every symbol declared in include/rtproj.h.

CPU only: no compute call is made (there is no GPU here)."""
import ctypes
import os
import re

import pytest

import paper_0912_1135_gb300 as rt
from paper_0912_1135_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(rtproj_\w+)\s*\(", txt)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return ctypes.CDLL(_build.LIB)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_the_abi():
    names = set(declared_functions())
    assert names <= set(rt.EXPORTS)


def test_host_only_entry_points_without_gpu(lib):
    rt.load_library()
    o = rt.default_opts()
    assert o.mode == rt.MODES["mixed"] and o.refine_passes >= 1
    assert rt.load_library().rtproj_status_string(4).decode().startswith("Cholesky")
    # workspace sizing is host arithmetic
    sz = rt.load_library().rtproj_workspace_bytes(64, 2048, 256, 16, ctypes.byref(o))
    assert sz > 64 * 2048 * 8
    assert rt.load_library().rtproj_workspace_bytes(64, 32, 64, 16, ctypes.byref(o)) == 0   # n < m
    assert rt.load_library().rtproj_workspace_bytes(64, 2048, 32, 16, ctypes.byref(o)) == 0  # l < m
    o.sketch_slices = 0
    assert rt.load_library().rtproj_workspace_bytes(64, 2048, 256, 16, ctypes.byref(o)) == 0


def test_create_rejects_bad_arguments_before_touching_the_device(lib):
    L = rt.load_library()
    h = ctypes.c_void_p()
    o = rt.default_opts()
    assert L.rtproj_create(ctypes.byref(h), 8, 4, ctypes.c_void_p(256), 4, 8, 1, ctypes.c_void_p(256), 1 << 30,
                           None, ctypes.byref(o)) == 1          # n < m
    assert L.rtproj_create(ctypes.byref(h), 8, 16, None, 16, 8, 1, ctypes.c_void_p(256), 1 << 30,
                           None, ctypes.byref(o)) == 1          # null A
    assert L.rtproj_create(ctypes.byref(h), 8, 16, ctypes.c_void_p(256), 16, 8, 1, ctypes.c_void_p(256), 16,
                           None, ctypes.byref(o)) == 7          # workspace too small
    assert L.rtproj_create(ctypes.byref(h), 8, 16, ctypes.c_void_p(256), 16, 8, 1, ctypes.c_void_p(257), 1 << 30,
                           None, ctypes.byref(o)) == 1          # misaligned workspace
    assert L.rtproj_precondition(None, 1, 8) == 1
    assert L.rtproj_null_project(None, None, 0, 1, None, 0) == 1


def test_sparse_entry_points_check_arguments_on_the_host(lib):
    """Sparse handles: workspace sizing is host arithmetic, and every argument error is
    returned before the device is touched (no GPU here)."""
    L = rt.load_library()
    o = rt.make_opts("fp64")
    sz = L.rtproj_sparse_workspace_bytes(64, 4096, 5 * 4096, 0, 256, 16, ctypes.byref(o))
    assert sz >= 64 * 4096 * 8 + 5 * 4096 * 12          # D = A^* P^- (n x m) and the CSC copy
    assert L.rtproj_sparse_workspace_bytes(64, 4096, 5 * 4096, 10, 256, 16, ctypes.byref(o)) > sz
    assert L.rtproj_sparse_workspace_bytes(64, 4096, 5 * 4096, 65, 256, 16, ctypes.byref(o)) == 0   # r > 64
    assert L.rtproj_sparse_workspace_bytes(64, 4096, -1, 0, 256, 16, ctypes.byref(o)) == 0
    assert L.rtproj_sparse_workspace_bytes(64, 4096, 10, 0, 256, 70000, ctypes.byref(o)) == 0        # k_max
    h = ctypes.c_void_p()
    p = ctypes.c_void_p(256)
    args = lambda **kw: dict(dict(m=8, n=16, nnz=40, rp=p, ci=p, v=p, r=0, U=None, V=None, l=8, k=1, ws=p,
                                  wsb=1 << 30, o=o), **kw)

    def create(a):
        return L.rtproj_create_sparse(ctypes.byref(h), a["m"], a["n"], a["nnz"], a["rp"], a["ci"], a["v"], a["r"],
                                      a["U"], a["V"], a["l"], a["k"], a["ws"], a["wsb"], None, ctypes.byref(a["o"]))
    assert create(args(rp=None)) == 1
    assert create(args(v=None)) == 1
    assert create(args(r=2)) == 1                        # U, V missing
    assert create(args(n=4)) == 1                        # n < m
    assert create(args(r=9, U=p, V=p)) == 9              # r > m
    assert create(args(k=70000)) == 9
    assert create(args(ws=ctypes.c_void_p(257))) == 1
    assert create(args(wsb=16)) == 7
    o32 = rt.make_opts("fp64")
    o32.dtype = 1
    assert create(args(o=o32)) == 9
