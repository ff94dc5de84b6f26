"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/*.h (no GPU needed: nothing here calls into CUDA)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(graphgp_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_2606_11402_gb300 import build as b
    return b.build()


def test_header_declares_entry_points():
    names = _declared()
    for required in ("graphgp_build_graph", "graphgp_factor", "graphgp_generate",
                     "graphgp_whiten", "graphgp_logdet", "graphgp_generate_backward",
                     "graphgp_whiten_backward", "graphgp_nll", "graphgp_nll_backward"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_library_is_built_for_sm103a():
    """The build compiles every unit and links for sm_103a only (the nvcc
    flags); on a GPU the loaded kernels report that target
    (test_gpu_graph.py::test_kernels_report_sm103)."""
    from paper_2606_11402_gb300 import build as b
    assert b.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_status_strings(libpath):
    lib = ctypes.CDLL(libpath)
    lib.graphgp_status_string.restype = ctypes.c_char_p
    assert lib.graphgp_status_string(0) == b"ok"
    assert b"timed out" in lib.graphgp_status_string(-4)


def test_binding_refuses_missing_library(monkeypatch, tmp_path):
    import paper_2606_11402_gb300 as gg
    monkeypatch.setattr(gg, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(gg, "_lib", None)
    with pytest.raises(ImportError):
        gg.load()


def test_host_side_argument_errors_without_gpu(libpath):
    """Arguments are validated on the host before any CUDA call."""
    import numpy as np
    lib = ctypes.CDLL(libpath)
    out = ctypes.c_void_p()
    lib.graphgp_build_graph.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.graphgp_build_graph(None, 100, 3, 8, None, None, ctypes.byref(out)) == -1
    assert lib.graphgp_selftest_wait_timeout(ctypes.c_int64(0), None) == -1
    # graph import: order must be a permutation and neighbours must precede
    lib.graphgp_graph_import.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    N, k, n0 = 6, 1, 2
    pts = np.zeros((N, 3), np.float32)
    lo = np.array([0, 2, 4, 6], np.int64)
    nbr = np.array([0, 1, 2, 3], np.int32)
    bad_order = np.array([0, 1, 2, 3, 4, 4], np.int32)
    assert lib.graphgp_graph_import(pts.ctypes.data, N, k, n0, bad_order.ctypes.data,
                                    nbr.ctypes.data, lo.ctypes.data, 3, None,
                                    ctypes.byref(out)) == -1
    order = np.arange(N, dtype=np.int32)
    late = np.array([0, 2, 3, 3], np.int32)  # position 3 conditions on 2, same level
    assert lib.graphgp_graph_import(pts.ctypes.data, N, k, n0, order.ctypes.data,
                                    late.ctypes.data, lo.ctypes.data, 3, None,
                                    ctypes.byref(out)) == -1
