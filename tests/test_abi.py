"""The C-ABI library loads on a machine without a GPU and exports every function include/*.h declares,
and the host-side argument checks reject bad input without touching the device."""
import ctypes as C
import glob
import os
import re

import pytest

from conftest import ROOT


def _declared():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(digs_\w+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    path = os.path.join(ROOT, "paper_2506_22280_gb300", "libdigs.so")
    if not os.path.exists(path):
        from paper_2506_22280_gb300 import build
        build.build()
    return C.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "digs_project_fwd" in names and "digs_step" in names and "digs_ffd_eval" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_host_checks(lib):
    lib.digs_status_string.restype = C.c_char_p
    assert lib.digs_status_string(0) == b"ok"
    assert b"workspace" in lib.digs_status_string(3)
    lib.digs_workspace_size.restype = C.c_size_t
    lib.digs_workspace_size.argtypes = [C.c_int] * 5 + [C.c_longlong, C.c_void_p]
    assert lib.digs_workspace_size(100, 4, 64, 64, 2, 1000, None) > 0
    assert lib.digs_workspace_size(100, 4, 64, 64, 9, 1000, None) == 0  # R above DIGS_MAX_R
    assert lib.digs_workspace_size(-1, 4, 64, 64, 2, 1000, None) == 0
    # workspace grows with the pair capacity
    assert lib.digs_workspace_size(100, 4, 64, 64, 2, 10 ** 6, None) > lib.digs_workspace_size(100, 4, 64, 64, 2, 0, None)
    lib.digs_ffd_eval.restype = C.c_int
    lib.digs_ffd_eval.argtypes = [C.c_void_p] * 3 + [C.c_int] + [C.c_void_p] * 3
    assert lib.digs_ffd_eval(None, None, None, 0, None, None, None) == 1  # DIGS_ERR_ARG, no launch


def test_binding_marshals_views_and_lattice():
    import numpy as np
    import synth
    from paper_2506_22280_gb300 import digs
    wl = synth.tiny()
    arr = digs.views_array(wl.views[:3])
    assert arr[1].nu == 64 and abs(arr[1].src[0] - wl.views[1]["src"][0]) < 1e-12
    lat = digs.lattice_struct(wl.lattice)
    assert (lat.nx, lat.ny, lat.nz, lat.R) == (8, 8, 8, 2) and abs(lat.origin[0] + 35) < 1e-6
    assert C.sizeof(digs.DigsView) == 8 * 16 + 4 * 3 + 4  # 16 doubles, 3 ints, tail padding


def test_gemm_and_cnn_input_host_checks(lib):
    """The tensor-core GEMM and the CNN input step reject bad sizes before any launch."""
    P, I = C.c_void_p, C.c_int
    f = lib.digs_gemm_bf16
    f.restype = I
    f.argtypes = [I, I, I, I, I, P, I, P, I, P, I, P, I, I, P, P, P]
    dummy = C.c_void_p(16)
    assert f(0, 0, -1, 4, 4, dummy, 4, dummy, 4, None, 0, dummy, 4, 1, None, None, None) == 1   # M < 0
    assert f(0, 0, 4, 4, 4, dummy, 4, dummy, 4, None, 0, dummy, 2, 1, None, None, None) == 1    # ldc < N
    assert f(0, 0, 4, 4, 8, dummy, 4, dummy, 4, None, 0, dummy, 4, 1, None, None, None) == 1    # lda < K
    assert f(0, 0, 4, 4, 4, dummy, 4, dummy, 4, None, 0, dummy, 4, 2, None, None, None) == 1    # split, no scratch
    assert f(0, 0, 4, 4, 4, dummy, 4, dummy, 4, None, 0, dummy, 4, 65, dummy, None, None) == 1  # splits > 64
    assert f(0, 0, 0, 4, 4, None, 4, None, 4, None, 0, None, 4, 1, None, None, None) == 0       # empty: nothing to do
    g = lib.digs_cnn_prepare_input
    g.restype = I
    g.argtypes = [P, I, I, I, C.c_float, P, P]
    assert g(dummy, 2, 64, 64, 1.0, dummy, None) == 1     # only 256 x 256 or 128 x 128 projections
    assert g(dummy, 2, 256, 128, 1.0, dummy, None) == 1
