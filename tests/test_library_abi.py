"""Host-side checks of the C-ABI library that need no GPU: it loads, it exports every function
include/aiwcrf.h declares, and argument validation that runs before any CUDA call rejects bad
input with the documented codes."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1811_00156_gb300 import aiwcrf as A

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "aiwcrf.h")


def _lib():
    if not os.path.exists(A.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return A.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(aiwcrf_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("aiwcrf_fit", "aiwcrf_predict", "aiwcrf_select_device"):
        assert must in names


def test_library_exports_every_declared_symbol():
    L = _lib()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    assert sorted(A.EXPORTS) == declared_functions()


def test_struct_layouts_match_header():
    assert C.sizeof(A.FitParams) == 40
    assert A.FitParams.first_tree.offset == 32
    assert C.sizeof(A.FitStats) == 10 * 8 + 16


def test_param_validation_without_gpu():
    L = _lib()
    X = np.zeros((4, 10), np.float32)
    y = np.zeros(10, np.int64)
    h = C.c_void_p()
    bad = [A.params(0, 2, 1), A.params(3, 0, 1), A.params(3, 2, 0), A.params(3, 2, 1, max_depth=-1)]
    for p in bad:
        rc = L.aiwcrf_fit(C.byref(p), X.ctypes.data, y.ctypes.data, 10, 4, None, C.byref(h))
        assert rc == -1, rc
        assert b"aiwcrf error -1" in L.aiwcrf_last_error()
    p = A.params(3, 2, 1)
    assert L.aiwcrf_fit(C.byref(p), X.ctypes.data, y.ctypes.data, 0, 4, None, C.byref(h)) == -1
    assert L.aiwcrf_fit(C.byref(p), X.ctypes.data, y.ctypes.data, 1 << 22, 4, None, C.byref(h)) == -8
    assert L.aiwcrf_fit(C.byref(p), X.ctypes.data, y.ctypes.data, 10, 129, None, C.byref(h)) == -1
    assert L.aiwcrf_fit(C.byref(p), None, y.ctypes.data, 10, 4, None, C.byref(h)) == -1


def test_deserialize_rejects_corrupt_blobs_without_gpu():
    L = _lib()
    h = C.c_void_p()
    for blob in [b"", b"NOTAFOREST" + b"\0" * 40, b"AIWCRF01" + b"\0" * 24]:
        buf = C.create_string_buffer(blob, max(len(blob), 1))
        assert L.aiwcrf_forest_deserialize(buf, len(blob), C.byref(h)) == -7
    # a split pointing backwards is rejected
    hdr = b"AIWCRF01" + np.array([1, 2], np.uint32).tobytes() + np.array([1, 2], np.int64).tobytes()
    off = np.array([0, 2], np.int64).tobytes()
    nodes = np.array([(0 << 56) | (0 << 32), 0], np.uint64).tobytes()
    blob = hdr + off + nodes
    buf = C.create_string_buffer(blob, len(blob))
    assert L.aiwcrf_forest_deserialize(buf, len(blob), C.byref(h)) == -7


def test_profile_names():
    L = _lib()
    n = L.aiwcrf_profile_num_classes()
    names = [L.aiwcrf_profile_name(k).decode() for k in range(n)]
    assert "level_big" in names and "predict" in names
    assert L.aiwcrf_profile_name(n) == b""


def test_plan_and_gate_layouts():
    assert C.sizeof(A.FitSchedule) == 16
    assert C.sizeof(A.GateParams) == 16
    assert C.sizeof(A.GateStats) == 32


def test_server_layouts_and_validation_without_gpu():
    assert C.sizeof(A.ServerParams) == 40
    assert C.sizeof(A.ServerCounters) == 23 * 8
    assert C.sizeof(A.BatchTrace) == 64
    assert C.sizeof(A.LoadReport) == 15 * 8
    L = _lib()
    F, N, D = 4, 10, 3
    X = np.zeros((F, N), np.float32)
    y = np.zeros(N, np.int64)
    dev = np.arange(D, dtype=np.int32)
    fp = A.params(3, 2, 1)
    h = C.c_void_p()

    def create(sp, X=X, y=y, F=F, N=N, D=D):
        return L.aiwcrf_server_create(C.byref(sp), C.byref(fp), X.ctypes.data, y.ctypes.data, N, F,
                                      dev.ctypes.data, D, C.byref(h))

    for sp in [A.server_params(n_streams=0), A.server_params(n_streams=17), A.server_params(max_request_kernels=0),
               A.server_params(max_request_kernels=128, batch_kernels=64), A.server_params(max_pending=0),
               A.server_params(refit_every=-1), A.server_params(arena_bytes=1024)]:
        assert create(sp) == -1, sp
    assert create(A.server_params(), F=2) == -1
    assert create(A.server_params(), D=0) == -1
    Xn = X.copy()
    Xn[1, 3] = np.nan
    assert create(A.server_params(), X=Xn) == -2
    yb = y.copy()
    yb[0] = (1 << 40) + 1
    assert create(A.server_params(), y=yb) == -8
    assert L.aiwcrf_server_destroy(None) == 0
    # the gated entry points check their arguments before touching a device
    t = C.c_int64()
    kf = np.zeros((F - 2, 1), np.float32)
    assert L.aiwcrf_server_set_surrogate(None, None, None) == -1
    # the tuner checks its arguments before fitting
    tp, best, mse = A.tune_params(), A.FitParams(), C.c_double()
    assert L.aiwcrf_tune_sa(None, C.byref(fp), X.ctypes.data, y.ctypes.data, N, F, None, None, C.byref(best),
                            C.byref(mse)) == -1
    for badtp in (A.tune_params(trees=(0, 4)), A.tune_params(node=(3, 2)), A.tune_params(cooling=0.0)):
        assert L.aiwcrf_tune_sa(C.byref(badtp), C.byref(fp), X.ctypes.data, y.ctypes.data, N, F, None, None,
                                C.byref(best), C.byref(mse)) == -1
    assert C.sizeof(A.TuneParams) == 56 and C.sizeof(A.TuneStep) == 24
    assert L.aiwcrf_server_submit_gated(None, kf.ctypes.data, 1, 0, C.byref(t)) == -1
    assert L.aiwcrf_server_wait_gated(None, 1, 0, None, None, None, None) == -1
    rep = A.LoadReport()
    assert L.aiwcrf_server_run_load_gated(None, kf.ctypes.data, 1, None, None, None, None, 1, 1.0, 1, 0, None, None,
                                          None, C.byref(rep)) == -1
