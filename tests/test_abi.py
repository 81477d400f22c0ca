"""The C ABI without a GPU: the library builds for sm_103a, loads, and exports
every function that include/polarstroke.h declares; the Python binding names
the same set.  Only host-side entry points are called here."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "polarstroke.h")


def declared():
    names = []
    decl = re.compile(r"^[A-Za-z][A-Za-z_0-9 ]*[ *]+(ps_[a-z0-9_]+)\(")
    with open(HEADER) as f:
        for line in f:
            m = decl.match(line)
            if m:
                names.append(m.group(1))
    return names


@pytest.fixture(scope="module")
def library():
    from paper_2007_00308_gb300 import _build
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_path_calls():
    names = set(declared())
    for n in ("ps_tessellate_strokes", "ps_arclength_scan", "ps_dash", "ps_rasterize_coverage",
              "ps_tessellate_backward", "ps_set_pixel_tolerance"):
        assert n in names
    assert len(names) >= 26


def test_library_exports_every_declared_symbol(library):
    missing = [n for n in declared() if not hasattr(library, n)]
    assert not missing, missing


def test_binding_names_match_the_header():
    import paper_2007_00308_gb300 as ps
    assert sorted(ps.EXPORTS) == sorted(declared())


def test_host_entry_points(library):
    library.ps_error_string.restype = ctypes.c_char_p
    library.ps_error_string.argtypes = [ctypes.c_int]
    assert library.ps_error_string(0)
    bound = ctypes.c_int64(0)
    library.ps_max_ribs.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_float,
                                    ctypes.POINTER(ctypes.c_int64)]
    assert library.ps_max_ribs(10, 2, 0.02, ctypes.byref(bound)) == 0 and bound.value > 0
    assert library.ps_max_ribs(10, 2, -1.0, ctypes.byref(bound)) < 0
    # null context: argument checks fail without touching a device
    library.ps_set_pixel_tolerance.argtypes = [ctypes.c_void_p, ctypes.c_float]
    assert library.ps_set_pixel_tolerance(None, 0.5) < 0
    library.ps_check_wait_timeout.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    assert library.ps_check_wait_timeout(None, 0, None) < 0


def test_static_rib_bound_holds_on_the_workloads(library):
    """ps_max_ribs (host only) bounds the oracle's rib count on samples of every
    workload and on degenerate and pivot-heavy inputs: callers size their rib
    buffers with it."""
    import numpy as np
    import oracle
    from paper_2007_00308_gb300 import workloads as W
    library.ps_max_ribs.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_float,
                                    ctypes.POINTER(ctypes.c_int64)]
    cusp = [[[0, 0], [1, 1], [0, 1], [1, 0]]]
    batches = [W.c1_plain_small(), W.c2_batching(n_paths=200), W.c3_large_path(n_seg=300),
               W.c4_precision(n=500), W.c5_differentiation(n_paths=8),
               W.single([W.CUBIC], cusp, width=4.0, dtheta_deg=0.5),
               W.single([W.CONIC], [[[0, 0], [50, 80], [50, 80], [100, 0]]], w=-0.9,
                        width=6.0, dtheta_deg=1.0)]
    for b in batches:
        bound = ctypes.c_int64(0)
        assert library.ps_max_ribs(len(b.seg_type), len(b.path_width), float(b.dtheta),
                                   ctypes.byref(bound)) == 0
        r = len(oracle.tessellate(b)["s"])
        assert r <= bound.value, (b.name, r, bound.value)
