"""Thin ctypes binding of libaiwcrf.so (include/aiwcrf.h). Argument marshalling only: every
step of fit, predict and device selection runs in the library's CUDA kernels.

Arrays may be torch tensors (CUDA or CPU) or numpy arrays. CUDA tensors are passed by device
pointer on torch's current stream; host arrays are staged by the library itself.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# AIWCRF_LIB=debug selects the bounds-checking build (libaiwcrf_debug.so), for tests;
# AIWCRF_LIB_PATH names another build of the same library (for example one compiled with other
# tuning macros)
LIB_PATH = os.environ.get("AIWCRF_LIB_PATH") or os.path.join(
    _HERE, "libaiwcrf_debug.so" if os.environ.get("AIWCRF_LIB") == "debug" else "libaiwcrf.so")

AIWCRF_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "NAN_INPUT", -3: "BAD_POINTER", -4: "OOM", -5: "CUDA",
          -6: "TIMEOUT", -7: "CORRUPT", -8: "LIMIT"}


class AiwcrfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class FitParams(C.Structure):
    _fields_ = [("num_trees", C.c_int32), ("mtry", C.c_int32), ("min_node_size", C.c_int32),
                ("max_depth", C.c_int32), ("seed", C.c_uint64), ("bootstrap", C.c_int32),
                ("ctas_per_sm", C.c_int32), ("first_tree", C.c_int64)]


class TuneParams(C.Structure):
    _fields_ = [("steps", C.c_int32), ("trees_min", C.c_int32), ("trees_max", C.c_int32), ("mtry_min", C.c_int32),
                ("mtry_max", C.c_int32), ("node_min", C.c_int32), ("node_max", C.c_int32), ("reserved", C.c_int32),
                ("t0", C.c_double), ("cooling", C.c_double), ("seed", C.c_uint64)]


class TuneStep(C.Structure):
    _fields_ = [("num_trees", C.c_int32), ("mtry", C.c_int32), ("min_node_size", C.c_int32),
                ("accepted", C.c_int32), ("oob_mse", C.c_double)]


class SurrogateParams(C.Structure):
    _fields_ = [("epochs", C.c_int32), ("batch", C.c_int32), ("lr", C.c_float), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float), ("seed", C.c_uint64), ("n_devices", C.c_int32),
                ("n_sizes", C.c_int32)]


class SurrogateStats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("first_batch_loss", C.c_float), ("last_batch_loss", C.c_float)]


class FitStats(C.Structure):
    _fields_ = [("num_trees", C.c_int64), ("total_nodes", C.c_int64), ("levels", C.c_int64),
                ("groups", C.c_int64), ("entries_evaluated", C.c_int64), ("entries_partitioned", C.c_int64),
                ("nodes_evaluated", C.c_int64), ("nodes_small", C.c_int64),
                ("entries_evaluated_small", C.c_int64), ("entries_partitioned_small", C.c_int64),
                ("n_features", C.c_int32), ("mtry", C.c_int32), ("rank_bytes", C.c_int32),
                ("grower", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerParams(C.Structure):
    _fields_ = [("n_streams", C.c_int32), ("max_request_kernels", C.c_int32), ("batch_kernels", C.c_int32),
                ("max_pending", C.c_int32), ("arena_bytes", C.c_int64), ("refit_every", C.c_int64),
                ("refit_rows", C.c_int64)]


class ServerCounters(C.Structure):
    _fields_ = [(k, C.c_int64) for k in (
        "submitted", "rejected", "completed", "failed", "batches", "batch_kernels_total", "batch_kernels_max",
        "arena_waits", "arena_bytes", "arena_peak_bytes", "refits", "refit_failures", "generation",
        "training_rows", "appended_rows", "forest_bytes", "refit_us_total", "refit_us_max", "gated_kernels",
        "gated_fallback", "gated_fallback_ood", "gated_fallback_var", "surrogate_bytes")]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class LoadReport(C.Structure):
    _fields_ = [("n_requests", C.c_int64), ("n_kernels", C.c_int64), ("offered_rate", C.c_double),
                ("wall_s", C.c_double), ("requests_per_s", C.c_double), ("kernels_per_s", C.c_double),
                ("p50_us", C.c_double), ("p99_us", C.c_double), ("mean_us", C.c_double), ("max_us", C.c_double),
                ("batches", C.c_int64), ("mean_batch_kernels", C.c_double), ("refits", C.c_int64),
                ("failed", C.c_int64), ("rejected", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class GateParams(C.Structure):
    _fields_ = [("var_trees", C.c_int32), ("z", C.c_float), ("ood", C.c_int32), ("tau", C.c_float)]


class GateStats(C.Structure):
    _fields_ = [("kernels", C.c_int64), ("fallback", C.c_int64), ("fallback_ood", C.c_int64),
                ("fallback_var", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class FitSchedule(C.Structure):
    _fields_ = [("level_big_ctas_per_sm", C.c_int32), ("level_small_ctas_per_sm", C.c_int32), ("ms", C.c_float),
                ("reserved", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class BatchTrace(C.Structure):
    _fields_ = [("t_formed_ns", C.c_int64), ("t_enqueued_ns", C.c_int64), ("t_done_ns", C.c_int64),
                ("kernels", C.c_int32), ("generation", C.c_int32), ("enqueue_cpu_ns", C.c_int64),
                ("enqueue_voluntary_switches", C.c_int32), ("enqueue_involuntary_switches", C.c_int32),
                ("poll_gap_max_ns", C.c_int64), ("gated_kernels", C.c_int32), ("fallback_kernels", C.c_int32)]


class RefitTrace(C.Structure):
    _fields_ = [("t_start_ns", C.c_int64), ("t_staged_ns", C.c_int64), ("t_fitted_ns", C.c_int64),
                ("t_swapped_ns", C.c_int64), ("rows", C.c_int64), ("generation", C.c_int64)]


EXPORTS = ["aiwcrf_fit", "aiwcrf_fit_subsets", "aiwcrf_predict", "aiwcrf_predict_sum", "aiwcrf_oob",
           "aiwcrf_oob_error",
           "aiwcrf_round_mean", "aiwcrf_select_device", "aiwcrf_forest_stats", "aiwcrf_forest_info",
           "aiwcrf_forest_serialize", "aiwcrf_forest_deserialize", "aiwcrf_forest_free",
           "aiwcrf_last_error", "aiwcrf_profile_enable", "aiwcrf_profile_read",
           "aiwcrf_profile_name", "aiwcrf_profile_num_classes", "aiwcrf_launch_count",
           "aiwcrf_select_device_noalloc", "aiwcrf_tc_gemm_bf16", "aiwcrf_surrogate_fit",
           "aiwcrf_surrogate_predict", "aiwcrf_surrogate_grad", "aiwcrf_surrogate_create", "aiwcrf_surrogate_export",
           "aiwcrf_surrogate_stats", "aiwcrf_surrogate_num_params", "aiwcrf_surrogate_free",
           "aiwcrf_server_create", "aiwcrf_server_submit", "aiwcrf_server_wait", "aiwcrf_server_append",
           "aiwcrf_server_refit", "aiwcrf_server_pause", "aiwcrf_server_stats", "aiwcrf_server_run_load",
           "aiwcrf_server_trace", "aiwcrf_server_destroy", "aiwcrf_select_device_gated",
           "aiwcrf_server_set_surrogate", "aiwcrf_server_submit_gated", "aiwcrf_server_wait_gated",
           "aiwcrf_server_run_load_gated", "aiwcrf_tune_sa",
           "aiwcrf_fit_plan_create", "aiwcrf_fit_plan_run", "aiwcrf_fit_plan_tune", "aiwcrf_fit_plan_set_schedule",
           "aiwcrf_fit_plan_free", "aiwcrf_profile_classes", "aiwcrf_set_grower", "aiwcrf_debug_bounds"]

_lib = None
_lock = threading.Lock()
_vp = C.c_void_p


def load():
    """Load the library. Raises if it has not been built: there is no fallback."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        L.aiwcrf_fit.argtypes = [C.POINTER(FitParams), _vp, _vp, C.c_int64, C.c_int32, _vp, C.POINTER(_vp)]
        L.aiwcrf_fit_subsets.argtypes = [C.POINTER(FitParams), _vp, _vp, C.c_int64, C.c_int32, _vp, _vp,
                                         C.c_int32, _vp, C.POINTER(_vp)]
        L.aiwcrf_predict.argtypes = [_vp, _vp, C.c_int64, _vp, _vp, _vp]
        L.aiwcrf_predict_sum.argtypes = [_vp, _vp, C.c_int64, _vp, _vp]
        L.aiwcrf_round_mean.argtypes = [_vp, C.c_int64, C.c_int64, _vp, _vp]
        L.aiwcrf_oob.argtypes = [_vp, _vp, C.c_int64, _vp, _vp, _vp]
        L.aiwcrf_oob_error.argtypes = [_vp, _vp, _vp, C.c_int64, _vp, C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                       _vp]
        L.aiwcrf_surrogate_fit.argtypes = [C.POINTER(SurrogateParams), _vp, _vp, C.c_int64, C.c_int32, _vp,
                                           C.POINTER(_vp)]
        L.aiwcrf_surrogate_predict.argtypes = [_vp, _vp, C.c_int64, _vp, _vp]
        L.aiwcrf_surrogate_grad.argtypes = [_vp, _vp, _vp, C.c_int32, _vp, _vp, _vp]
        L.aiwcrf_surrogate_create.argtypes = [C.c_int32, C.c_int32, C.c_int32, _vp, _vp, _vp, _vp, C.POINTER(_vp)]
        L.aiwcrf_surrogate_export.argtypes = [_vp, _vp, _vp, _vp, _vp]
        L.aiwcrf_surrogate_stats.argtypes = [_vp, C.POINTER(SurrogateStats)]
        L.aiwcrf_surrogate_num_params.restype = C.c_int32
        L.aiwcrf_surrogate_free.argtypes = [_vp]
        L.aiwcrf_tc_gemm_bf16.argtypes = [_vp, C.c_int32, C.c_int32, _vp, C.c_int32, C.c_int32, _vp, C.c_int32,
                                          C.c_int32, C.c_int32, C.c_int32, _vp]
        L.aiwcrf_select_device.argtypes = [_vp, _vp, C.c_int32, C.c_int32, _vp, C.c_int32, _vp, _vp, _vp]
        L.aiwcrf_select_device_noalloc.argtypes = [_vp, _vp, C.c_int32, C.c_int32, _vp, C.c_int32, _vp, _vp, _vp]
        L.aiwcrf_forest_stats.argtypes = [_vp, C.POINTER(FitStats)]
        L.aiwcrf_forest_info.argtypes = [_vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int32)]
        L.aiwcrf_forest_serialize.argtypes = [_vp, _vp, C.c_size_t, C.POINTER(C.c_size_t)]
        L.aiwcrf_forest_deserialize.argtypes = [_vp, C.c_size_t, C.POINTER(_vp)]
        L.aiwcrf_forest_free.argtypes = [_vp]
        L.aiwcrf_last_error.restype = C.c_char_p
        L.aiwcrf_profile_enable.argtypes = [C.c_int32]
        L.aiwcrf_profile_classes.argtypes = [C.c_uint32]
        L.aiwcrf_profile_read.argtypes = [C.c_int32, _vp, _vp]
        L.aiwcrf_profile_name.argtypes = [C.c_int32]
        L.aiwcrf_profile_name.restype = C.c_char_p
        L.aiwcrf_profile_num_classes.restype = C.c_int32
        L.aiwcrf_set_grower.argtypes = [C.c_int32]
        L.aiwcrf_debug_bounds.restype = C.c_int64
        L.aiwcrf_launch_count.restype = C.c_int64
        L.aiwcrf_server_create.argtypes = [C.POINTER(ServerParams), C.POINTER(FitParams), _vp, _vp, C.c_int64,
                                           C.c_int32, _vp, C.c_int32, C.POINTER(_vp)]
        L.aiwcrf_server_submit.argtypes = [_vp, _vp, C.c_int32, C.c_int32, C.POINTER(C.c_int64)]
        L.aiwcrf_server_wait.argtypes = [_vp, C.c_int64, C.c_int32, _vp, _vp, C.POINTER(C.c_int64)]
        L.aiwcrf_server_append.argtypes = [_vp, _vp, _vp, C.c_int64]
        L.aiwcrf_server_refit.argtypes = [_vp, C.c_int32]
        L.aiwcrf_server_pause.argtypes = [_vp, C.c_int32]
        L.aiwcrf_server_stats.argtypes = [_vp, C.POINTER(ServerCounters)]
        L.aiwcrf_server_run_load.argtypes = [_vp, _vp, C.c_int64, _vp, _vp, _vp, C.c_int64, C.c_double,
                                             C.c_uint64, C.c_int32, _vp, _vp, _vp, C.POINTER(LoadReport)]
        L.aiwcrf_server_destroy.argtypes = [_vp]
        L.aiwcrf_fit_plan_create.argtypes = [C.POINTER(FitParams), _vp, _vp, C.c_int64, C.c_int32, _vp, _vp,
                                             C.c_int32, _vp, C.POINTER(_vp)]
        L.aiwcrf_fit_plan_run.argtypes = [_vp, _vp, _vp]
        L.aiwcrf_fit_plan_tune.argtypes = [_vp, C.c_int32, _vp, _vp, C.c_int32, C.POINTER(C.c_int32),
                                           C.POINTER(FitSchedule)]
        L.aiwcrf_fit_plan_set_schedule.argtypes = [_vp, C.POINTER(FitSchedule)]
        L.aiwcrf_fit_plan_free.argtypes = [_vp]
        L.aiwcrf_select_device_gated.argtypes = [_vp, _vp, C.POINTER(GateParams), _vp, C.c_int32, C.c_int32, _vp,
                                                 C.c_int32, _vp, _vp, _vp, C.POINTER(GateStats), _vp]
        L.aiwcrf_server_trace.argtypes = [_vp, _vp, C.c_int64, C.POINTER(C.c_int64), _vp, C.c_int64,
                                          C.POINTER(C.c_int64)]
        L.aiwcrf_server_set_surrogate.argtypes = [_vp, _vp, C.POINTER(GateParams)]
        L.aiwcrf_tune_sa.argtypes = [C.POINTER(TuneParams), C.POINTER(FitParams), _vp, _vp, C.c_int64, C.c_int32, _vp,
                                     _vp, C.POINTER(FitParams), C.POINTER(C.c_double)]
        L.aiwcrf_server_submit_gated.argtypes = [_vp, _vp, C.c_int32, C.c_int32, C.POINTER(C.c_int64)]
        L.aiwcrf_server_wait_gated.argtypes = [_vp, C.c_int64, C.c_int32, _vp, _vp, _vp, C.POINTER(C.c_int64)]
        L.aiwcrf_server_run_load_gated.argtypes = [_vp, _vp, C.c_int64, _vp, _vp, _vp, _vp, C.c_int64, C.c_double,
                                                   C.c_uint64, C.c_int32, _vp, _vp, _vp, C.POINTER(LoadReport)]
        for name in EXPORTS:
            if name not in ("aiwcrf_last_error", "aiwcrf_profile_name", "aiwcrf_profile_num_classes",
                            "aiwcrf_launch_count", "aiwcrf_surrogate_num_params"):
                getattr(L, name).restype = C.c_int
        _lib = L
        return L


def _check(rc: int):
    if rc != AIWCRF_OK:
        msg = load().aiwcrf_last_error().decode(errors="replace")
        raise AiwcrfError(rc, msg)


def _ptr(a):
    """Pointer of a torch tensor or numpy array (must be contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return a.ctypes.data
    if not a.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return a.data_ptr()


def _stream(stream=None):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    import torch
    return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0


def _shape(a):
    return tuple(a.shape)


class Forest:
    """A fitted forest owned by the library (freed on garbage collection)."""

    def __init__(self, handle: int):
        self._h = _vp(handle)

    def __del__(self):
        self.free()

    def free(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().aiwcrf_forest_free(self._h)
        self._h = None

    @property
    def handle(self):
        return self._h

    def info(self):
        T, nn, F = C.c_int64(), C.c_int64(), C.c_int32()
        _check(load().aiwcrf_forest_info(self._h, C.byref(T), C.byref(nn), C.byref(F)))
        return dict(num_trees=T.value, num_nodes=nn.value, n_features=F.value)

    def stats(self) -> dict:
        st = FitStats()
        _check(load().aiwcrf_forest_stats(self._h, C.byref(st)))
        return st.as_dict()

    def serialize(self) -> bytes:
        need = C.c_size_t()
        _check(load().aiwcrf_forest_serialize(self._h, None, 0, C.byref(need)))
        buf = C.create_string_buffer(need.value)
        _check(load().aiwcrf_forest_serialize(self._h, buf, need.value, C.byref(need)))
        return buf.raw


def aiwcrf_fit(params: FitParams, X, y, stream=None) -> Forest:
    F, N = _shape(X)
    h = _vp()
    _check(load().aiwcrf_fit(C.byref(params), _ptr(X), _ptr(y), N, F, _stream(stream), C.byref(h)))
    return Forest(h.value)


def aiwcrf_fit_subsets(params: FitParams, X, y, offsets, rows, stream=None) -> list:
    F, N = _shape(X)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    G = int(offsets.size - 1)
    hs = (_vp * G)()
    _check(load().aiwcrf_fit_subsets(C.byref(params), _ptr(X), _ptr(y), N, F, offsets.ctypes.data,
                                     _ptr(rows), G, _stream(stream), hs))
    return [Forest(hs[g]) for g in range(G)]


def aiwcrf_predict(forest: Forest, Xq, out_pred, out_var=None, stream=None):
    F, Q = _shape(Xq)
    _check(load().aiwcrf_predict(forest.handle, _ptr(Xq), Q, _ptr(out_pred), _ptr(out_var), _stream(stream)))
    return out_pred


def aiwcrf_predict_sum(forest: Forest, Xq, out_sum, stream=None):
    F, Q = _shape(Xq)
    _check(load().aiwcrf_predict_sum(forest.handle, _ptr(Xq), Q, _ptr(out_sum), _stream(stream)))
    return out_sum


def aiwcrf_oob(forest: Forest, X, out_sum, out_count, stream=None):
    F, N = _shape(X)
    _check(load().aiwcrf_oob(forest.handle, _ptr(X), N, _ptr(out_sum), _ptr(out_count), _stream(stream)))
    return out_sum, out_count


def aiwcrf_oob_error(forest: Forest, X, y, out_pred=None, stream=None):
    """(mean squared out-of-bag error in the target's units, rows out of bag); fills out_pred
    with the out-of-bag predictions when given."""
    F, N = _shape(X)
    mse = C.c_double(0.0)
    rows = C.c_int64(0)
    _check(load().aiwcrf_oob_error(forest.handle, _ptr(X), _ptr(y), N, _ptr(out_pred),
                                   C.byref(mse), C.byref(rows), _stream(stream)))
    return mse.value, rows.value


class Surrogate:
    """A trained surrogate owned by the library."""

    def __init__(self, handle: int, F: int):
        self._h = _vp(handle)
        self.F = F

    def __del__(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().aiwcrf_surrogate_free(self._h)
        self._h = None

    @property
    def handle(self):
        return self._h

    def predict(self, Xq, out, stream=None):
        F, Q = _shape(Xq)
        _check(load().aiwcrf_surrogate_predict(self._h, _ptr(Xq), Q, _ptr(out), _stream(stream)))
        return out

    def grad(self, X, y, grad, loss, stream=None):
        F, n = _shape(X)
        _check(load().aiwcrf_surrogate_grad(self._h, _ptr(X), _ptr(y), n, _ptr(grad), _ptr(loss), _stream(stream)))
        return grad, loss

    def export(self):
        P = np.zeros(int(load().aiwcrf_surrogate_num_params()), np.float32)
        mu = np.zeros(self.F - 2, np.float32)
        sd = np.zeros(self.F - 2, np.float32)
        lg = np.zeros(self.F - 2, np.uint8)
        _check(load().aiwcrf_surrogate_export(self._h, P.ctypes.data, mu.ctypes.data, sd.ctypes.data, lg.ctypes.data))
        return P, mu, sd, lg

    def stats(self) -> dict:
        st = SurrogateStats()
        _check(load().aiwcrf_surrogate_stats(self._h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in st._fields_}


def surrogate_params(epochs=20, batch=4096, lr=1e-3, seed=156, n_devices=15, n_sizes=4) -> SurrogateParams:
    return SurrogateParams(epochs, batch, lr, 0.9, 0.999, 1e-8, seed, n_devices, n_sizes)


def aiwcrf_surrogate_fit(params: SurrogateParams, teacher: Forest, X, stream=None) -> Surrogate:
    F, n = _shape(X)
    h = _vp()
    _check(load().aiwcrf_surrogate_fit(C.byref(params), teacher.handle, _ptr(X), n, F, _stream(stream), C.byref(h)))
    return Surrogate(h.value, F)


def aiwcrf_surrogate_create(F, n_devices, n_sizes, P, mu, sd, log2_cols) -> Surrogate:
    P = np.ascontiguousarray(P, np.float32)
    mu, sd = np.ascontiguousarray(mu, np.float32), np.ascontiguousarray(sd, np.float32)
    lg = np.ascontiguousarray(log2_cols, np.uint8)
    h = _vp()
    _check(load().aiwcrf_surrogate_create(F, n_devices, n_sizes, P.ctypes.data, mu.ctypes.data, sd.ctypes.data,
                                          lg.ctypes.data, C.byref(h)))
    return Surrogate(h.value, F)


def aiwcrf_tc_gemm_bf16(A, B, C, a_trans=False, b_trans=False, ksplit=1, stream=None):
    """C = A @ B^T on the tensor cores (BF16 in, FP32 out). A: (M, K) or, with a_trans, (K, M)."""
    M = A.shape[1] if a_trans else A.shape[0]
    K = A.shape[0] if a_trans else A.shape[1]
    N = B.shape[1] if b_trans else B.shape[0]
    _check(load().aiwcrf_tc_gemm_bf16(_ptr(A), A.shape[1], int(a_trans), _ptr(B), B.shape[1], int(b_trans), _ptr(C),
                                      M, N, K, int(ksplit), _stream(stream)))
    return C


def aiwcrf_round_mean(sums, total_trees: int, out, stream=None):
    n = int(np.prod(_shape(sums)))
    _check(load().aiwcrf_round_mean(_ptr(sums), n, total_trees, _ptr(out), _stream(stream)))
    return out


def aiwcrf_select_device(forest: Forest, kfeat, size_class: int, device_ids, out_best, out_pred=None,
                         stream=None):
    Fm2, K = _shape(kfeat)
    dev = np.ascontiguousarray(device_ids, dtype=np.int32)
    _check(load().aiwcrf_select_device(forest.handle, _ptr(kfeat), K, int(size_class), dev.ctypes.data,
                                       int(dev.size), _ptr(out_best), _ptr(out_pred), _stream(stream)))
    return out_best


def aiwcrf_select_device_noalloc(forest: Forest, kfeat, size_class: int, device_ids, out_best, out_pred=None,
                                 stream=None):
    """Same as aiwcrf_select_device without any device allocation: kfeat and the outputs must be
    device tensors; the library's static scratch array limits the request size."""
    Fm2, K = _shape(kfeat)
    dev = np.ascontiguousarray(device_ids, dtype=np.int32)
    _check(load().aiwcrf_select_device_noalloc(forest.handle, _ptr(kfeat), K, int(size_class), dev.ctypes.data,
                                               int(dev.size), _ptr(out_best), _ptr(out_pred), _stream(stream)))
    return out_best


def server_params(n_streams=4, max_request_kernels=64, batch_kernels=1024, max_pending=65536,
                  arena_bytes=64 << 20, refit_every=0, refit_rows=0) -> ServerParams:
    return ServerParams(n_streams, max_request_kernels, batch_kernels, max_pending, arena_bytes, refit_every,
                        refit_rows)


class Server:
    """Device-selection server (include/aiwcrf.h): a resident forest answering requests by
    continuous batching, with refits from appended rows. Host numpy arrays throughout."""

    def __init__(self, sparams: ServerParams, fparams: FitParams, X: np.ndarray, y: np.ndarray, device_ids):
        X = np.ascontiguousarray(X, dtype=np.float32)
        y = np.ascontiguousarray(y, dtype=np.int64)
        self.F, N = X.shape
        self.device_ids = np.ascontiguousarray(device_ids, dtype=np.int32)
        self.D = int(self.device_ids.size)
        h = _vp()
        _check(load().aiwcrf_server_create(C.byref(sparams), C.byref(fparams), X.ctypes.data, y.ctypes.data, N,
                                           self.F, self.device_ids.ctypes.data, self.D, C.byref(h)))
        self.handle = h.value

    def close(self):
        if getattr(self, "handle", None):
            load().aiwcrf_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def submit(self, kfeat: np.ndarray, size_class: int, gated: bool = False) -> int:
        """Queue a request (gated: answered through the resident surrogate, see set_surrogate)."""
        kfeat = np.ascontiguousarray(kfeat, dtype=np.float32)
        t = C.c_int64()
        fn = load().aiwcrf_server_submit_gated if gated else load().aiwcrf_server_submit
        _check(fn(self.handle, kfeat.ctypes.data, int(kfeat.shape[1]), int(size_class), C.byref(t)))
        self._k = getattr(self, "_k", {})
        self._k[t.value] = int(kfeat.shape[1])
        return t.value

    def set_surrogate(self, surrogate, gate: "GateParams | None" = None):
        """Keep a copy of surrogate resident for gated requests (None removes it)."""
        _check(load().aiwcrf_server_set_surrogate(self.handle, None if surrogate is None else surrogate.handle,
                                                  None if gate is None else C.byref(gate)))

    def wait_gated(self, ticket: int, timeout_ms: int = -1):
        """(best[K], pred[K, D] float log10 s, fallback[K] uint8, generation) of a gated request."""
        K = self._k[ticket]
        best = np.zeros(K, np.int32)
        pred = np.zeros((K, self.D), np.float32)
        fb = np.zeros(K, np.uint8)
        g = C.c_int64()
        _check(load().aiwcrf_server_wait_gated(self.handle, ticket, timeout_ms, best.ctypes.data, pred.ctypes.data,
                                               fb.ctypes.data, C.byref(g)))
        del self._k[ticket]
        return best, pred, fb, g.value

    def wait(self, ticket: int, timeout_ms: int = -1):
        """(best[K], pred[K, D], generation)."""
        K = self._k[ticket]
        best = np.zeros(K, np.int32)
        pred = np.zeros((K, self.D), np.int64)
        g = C.c_int64()
        _check(load().aiwcrf_server_wait(self.handle, ticket, timeout_ms, best.ctypes.data, pred.ctypes.data,
                                         C.byref(g)))
        del self._k[ticket]
        return best, pred, g.value

    def append(self, X: np.ndarray, y: np.ndarray):
        X = np.ascontiguousarray(X, dtype=np.float32)
        y = np.ascontiguousarray(y, dtype=np.int64)
        _check(load().aiwcrf_server_append(self.handle, X.ctypes.data, y.ctypes.data, int(y.size)))

    def refit(self, wait: bool = True):
        _check(load().aiwcrf_server_refit(self.handle, 1 if wait else 0))

    def pause(self, paused: bool):
        _check(load().aiwcrf_server_pause(self.handle, 1 if paused else 0))

    def stats(self) -> dict:
        c = ServerCounters()
        _check(load().aiwcrf_server_stats(self.handle, C.byref(c)))
        return c.as_dict()

    def trace(self):
        """(batches, refits) as numpy structured arrays, oldest first."""
        bt = (BatchTrace * 65536)()
        rt = (RefitTrace * 256)()
        n, rn = C.c_int64(), C.c_int64()
        _check(load().aiwcrf_server_trace(self.handle, bt, 65536, C.byref(n), rt, 256, C.byref(rn)))
        b = np.ctypeslib.as_array(bt)[:n.value].copy()
        r = np.ctypeslib.as_array(rt)[:rn.value].copy()
        return b, r

    def run_load(self, pool: np.ndarray, first, n_kernels, size_class, rate_per_s: float, seed: int = 1,
                 timeout_ms: int = 120000, gated=None):
        """Open-loop Poisson load (gated: per-request flags, or None for none). Returns (report dict,
        best[sum K], generation[n], latency_ns[n])."""
        pool = np.ascontiguousarray(pool, dtype=np.float32)
        first = np.ascontiguousarray(first, dtype=np.int64)
        nk = np.ascontiguousarray(n_kernels, dtype=np.int32)
        sc = np.ascontiguousarray(size_class, dtype=np.int32)
        n = int(first.size)
        best = np.full(int(nk.sum()), -1, np.int32)
        gen = np.full(n, -1, np.int64)
        lat = np.full(n, -1, np.int64)
        rep = LoadReport()
        if gated is None:
            _check(load().aiwcrf_server_run_load(self.handle, pool.ctypes.data, int(pool.shape[1]), first.ctypes.data,
                                                 nk.ctypes.data, sc.ctypes.data, n, float(rate_per_s), seed,
                                                 timeout_ms, best.ctypes.data, gen.ctypes.data, lat.ctypes.data,
                                                 C.byref(rep)))
        else:
            g = np.ascontiguousarray(gated, dtype=np.uint8)
            _check(load().aiwcrf_server_run_load_gated(self.handle, pool.ctypes.data, int(pool.shape[1]),
                                                       first.ctypes.data, nk.ctypes.data, sc.ctypes.data,
                                                       g.ctypes.data, n, float(rate_per_s), seed, timeout_ms,
                                                       best.ctypes.data, gen.ctypes.data, lat.ctypes.data,
                                                       C.byref(rep)))
        return rep.as_dict(), best, gen, lat


class FitPlan:
    """A fit captured once as a CUDA graph and replayed (include/aiwcrf.h). X, y and subset_rows are
    device tensors the plan reads at every run; keep them alive while the plan lives."""

    def __init__(self, params: FitParams, X, y, subset_offsets=None, subset_rows=None, stream=None):
        F, N = _shape(X)
        self._keep = (X, y, subset_rows)
        off = None if subset_offsets is None else np.ascontiguousarray(subset_offsets, dtype=np.int64)
        G = 0 if off is None else int(off.size - 1)
        h = _vp()
        _check(load().aiwcrf_fit_plan_create(C.byref(params), _ptr(X), _ptr(y), N, F,
                                             None if off is None else off.ctypes.data, _ptr(subset_rows), G,
                                             _stream(stream), C.byref(h)))
        self.handle = h.value
        self.n_forests = max(G, 1)

    def run(self, stream=None) -> list:
        arr = (_vp * self.n_forests)()
        _check(load().aiwcrf_fit_plan_run(self.handle, _stream(stream), arr))
        return [Forest(arr[i]) for i in range(self.n_forests)]

    def tune(self, reps: int = 3, stream=None):
        """(chosen schedule dict, list of every schedule tried)."""
        tried = (FitSchedule * 64)()
        n = C.c_int32()
        chosen = FitSchedule()
        _check(load().aiwcrf_fit_plan_tune(self.handle, reps, _stream(stream), tried, 64, C.byref(n), C.byref(chosen)))
        return chosen.as_dict(), [tried[i].as_dict() for i in range(min(n.value, 64))]

    def set_schedule(self, level_big: int, level_small: int):
        _check(load().aiwcrf_fit_plan_set_schedule(self.handle, C.byref(FitSchedule(level_big, level_small, 0.0, 0))))

    def close(self):
        if getattr(self, "handle", None):
            load().aiwcrf_fit_plan_free(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


def gate_params(var_trees: int = 32, z: float = 1.0, ood: bool = True, tau: float = 0.0) -> GateParams:
    return GateParams(var_trees, z, 1 if ood else 0, tau)


def aiwcrf_select_device_gated(forest: Forest, surrogate, gate: GateParams, kfeat, size_class: int, device_ids,
                               out_best, out_pred=None, out_fallback=None, stream=None) -> dict:
    """Surrogate device selection with forest fallback (device tensors); returns the gate counters."""
    Fm2, K = _shape(kfeat)
    dev = np.ascontiguousarray(device_ids, dtype=np.int32)
    st = GateStats()
    _check(load().aiwcrf_select_device_gated(forest.handle, surrogate.handle, C.byref(gate), _ptr(kfeat), K,
                                             int(size_class), dev.ctypes.data, int(dev.size), _ptr(out_best),
                                             _ptr(out_pred), _ptr(out_fallback), C.byref(st), _stream(stream)))
    return st.as_dict()


def aiwcrf_forest_deserialize(blob: bytes) -> Forest:
    h = _vp()
    buf = C.create_string_buffer(blob, len(blob))
    _check(load().aiwcrf_forest_deserialize(buf, len(blob), C.byref(h)))
    return Forest(h.value)


def aiwcrf_profile_enable(on: bool):
    _check(load().aiwcrf_profile_enable(1 if on else 0))


def aiwcrf_profile_classes(names=None):
    """Time only the named kernel classes (None: all)."""
    L = load()
    if names is None:
        mask = 0xFFFFFFFF
    else:
        idx = {L.aiwcrf_profile_name(k).decode(): k for k in range(int(L.aiwcrf_profile_num_classes()))}
        mask = 0
        for n in names:
            mask |= 1 << idx[n]
    _check(L.aiwcrf_profile_classes(mask))


def aiwcrf_profile_read() -> dict:
    L = load()
    n = int(L.aiwcrf_profile_num_classes())
    launches = np.zeros(n, np.int64)
    ms = np.zeros(n, np.float64)
    _check(L.aiwcrf_profile_read(n, launches.ctypes.data, ms.ctypes.data))
    return {L.aiwcrf_profile_name(k).decode(): (int(launches[k]), float(ms[k])) for k in range(n)}


def aiwcrf_launch_count() -> int:
    return int(load().aiwcrf_launch_count())


GROWER_AUTO, GROWER_LEVEL, GROWER_TREE, GROWER_LISTS = 0, 1, 2, 3


def aiwcrf_debug_bounds() -> int:
    """Bounds-check violations since the last call in a debug build (0 none), -1 in a release build."""
    return int(load().aiwcrf_debug_bounds())


def aiwcrf_set_grower(grower: int):
    """Kernels that grow the trees of the following fits (GROWER_AUTO, GROWER_LEVEL, GROWER_TREE,
    GROWER_LISTS)."""
    _check(load().aiwcrf_set_grower(grower))


def params(num_trees: int, mtry: int, min_node_size: int, max_depth: int = 0, seed: int = 156,
           bootstrap: bool = True, first_tree: int = 0, ctas_per_sm: int = 0) -> FitParams:
    return FitParams(num_trees, mtry, min_node_size, max_depth, seed, 1 if bootstrap else 0, ctas_per_sm, first_tree)


def tune_params(steps=40, trees=(16, 512), mtry=(1, 32), node=(1, 20), t0=0.1, cooling=0.95,
                seed=1) -> TuneParams:
    return TuneParams(steps, trees[0], trees[1], mtry[0], mtry[1], node[0], node[1], 0, t0, cooling, seed)


def aiwcrf_tune_sa(tp: TuneParams, start: FitParams, X, y, stream=None):
    """Simulated-annealing tuning against the out-of-bag error (include/aiwcrf.h). Returns
    (best FitParams, best OOB MSE, trace as a list of dicts)."""
    F, N = _shape(X)
    trace = (TuneStep * (tp.steps + 1))()
    best = FitParams()
    mse = C.c_double()
    _check(load().aiwcrf_tune_sa(C.byref(tp), C.byref(start), _ptr(X), _ptr(y), N, F, _stream(stream), trace,
                                 C.byref(best), C.byref(mse)))
    steps = [{k: getattr(t, k) for k, _ in TuneStep._fields_} for t in trace]
    return best, mse.value, steps


def decode_forest(blob: bytes) -> dict:
    """Parse a serialized forest (layout in include/aiwcrf.h) into numpy arrays."""
    assert blob[:8] == b"AIWCRF01"
    version, F = np.frombuffer(blob, np.uint32, 2, 8)
    T, nn = np.frombuffer(blob, np.int64, 2, 16)
    off = np.frombuffer(blob, np.int64, int(T) + 1, 32)
    nodes = np.frombuffer(blob, np.uint64, int(nn), 32 + 8 * (int(T) + 1))
    return dict(version=int(version), F=int(F), T=int(T), tree_off=off.copy(), nodes=nodes.copy())
