"""CPU oracle for the random-forest path: a ctypes wrapper around aiwcrf_oracle.c.

TEST INFRASTRUCTURE. Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import this package. It shares no code with the CUDA library (``paper_1811_00156_gb300``), and
the library never imports it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aiwcrf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_aiwcrf.so")
_lock = threading.Lock()
_lib = None

_P_F32 = C.POINTER(C.c_float)
_P_I64 = C.POINTER(C.c_int64)
_P_I32 = C.POINTER(C.c_int32)
_P_U32 = C.POINTER(C.c_uint32)
_P_U64 = C.POINTER(C.c_uint64)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, no SIMD intrinsics, no threads)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            L.orc_philox4x32.argtypes = [_P_U32, _P_U32, C.c_int, _P_U32]
            L.orc_philox4x64.argtypes = [_P_U64, _P_U64, C.c_int, _P_U64]
            L.orc_bootstrap_counts.argtypes = [C.c_uint64, C.c_int64, C.c_int64, _P_U32]
            L.orc_mtry_draw.argtypes = [C.c_uint64, C.c_int64, C.c_int64, C.c_int64, C.c_int32,
                                        C.c_int32, _P_I32]
            L.orc_gain_cmp.argtypes = [C.c_int64] * 8
            L.orc_gain_cmp.restype = C.c_int
            L.orc_round_mean.argtypes = [C.c_int64, C.c_int64]
            L.orc_round_mean.restype = C.c_int64
            L.orc_fit.argtypes = [_P_F32, _P_I64, C.c_int64, C.c_int32, C.c_int64, C.c_int64,
                                  C.c_int32, C.c_int32, C.c_int32, C.c_uint64, C.c_int32,
                                  C.POINTER(C.c_void_p)]
            L.orc_fit.restype = C.c_int
            L.orc_forest_free.argtypes = [C.c_void_p]
            L.orc_forest_num_trees.argtypes = [C.c_void_p]
            L.orc_forest_num_trees.restype = C.c_int64
            L.orc_tree_num_nodes.argtypes = [C.c_void_p, C.c_int64]
            L.orc_tree_num_nodes.restype = C.c_int64
            L.orc_tree_export.argtypes = [C.c_void_p, C.c_int64, _P_I32, _P_F32, _P_I64, _P_I64,
                                          _P_I64, _P_I64, _P_I64, _P_I32, _P_I32]
            L.orc_predict.argtypes = [C.c_void_p, _P_F32, C.c_int64, C.c_int64, _P_I64, _P_I64,
                                      _P_U64]
            L.orc_predict.restype = C.c_int
            L.orc_oob.argtypes = [C.c_void_p, _P_F32, C.c_int64, _P_I64, _P_I32]
            L.orc_oob.restype = C.c_int
            L.orc_select_device.argtypes = [C.c_void_p, _P_F32, C.c_int32, C.c_int32, _P_I32,
                                            C.c_int32, _P_I32, _P_I64]
            L.orc_select_device.restype = C.c_int
            _lib = L
    return _lib


def _ptr(a: np.ndarray, typ):
    return a.ctypes.data_as(typ)


def philox4x32(ctr, key, rounds: int = 10) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32(_ptr(c, _P_U32), _ptr(k, _P_U32), rounds, _ptr(out, _P_U32))
    return out


def philox4x64(ctr, key, rounds: int = 10) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64(_ptr(c, _P_U64), _ptr(k, _P_U64), rounds, _ptr(out, _P_U64))
    return out


def bootstrap_counts(seed: int, t: int, n_pool: int) -> np.ndarray:
    out = np.zeros(n_pool, dtype=np.uint32)
    lib().orc_bootstrap_counts(seed, t, n_pool, _ptr(out, _P_U32))
    return out


def mtry_draw(seed: int, t: int, d: int, i: int, F: int, mtry: int) -> np.ndarray:
    out = np.zeros(F, dtype=np.int32)
    lib().orc_mtry_draw(seed, t, d, i, F, mtry, _ptr(out, _P_I32))
    return out[:min(mtry, F)].copy()


def gain_cmp(a, b) -> int:
    """sign(G(a) - G(b)) for candidates given as (nL, SL, nR, SR)."""
    return int(lib().orc_gain_cmp(*[int(v) for v in a], *[int(v) for v in b]))


def round_mean(S: int, n: int) -> int:
    return int(lib().orc_round_mean(S, n))


@dataclass
class Tree:
    """One tree in BFS order. feature == -1 marks a leaf."""
    feature: np.ndarray
    thr: np.ndarray
    left: np.ndarray
    value: np.ndarray
    n: np.ndarray
    S: np.ndarray
    nrows: np.ndarray
    depth: np.ndarray
    evaluated: np.ndarray

    @property
    def num_nodes(self) -> int:
        return int(self.feature.size)


class Forest:
    """Oracle forest for global tree indices [t0, t1)."""

    def __init__(self, handle, t0: int, t1: int, F: int):
        self._h = handle
        self.t0, self.t1, self.F = t0, t1, F

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_forest_free(self._h)
            self._h = None

    @property
    def num_trees(self) -> int:
        return self.t1 - self.t0

    def tree(self, k: int) -> Tree:
        L = lib()
        m = int(L.orc_tree_num_nodes(self._h, k))
        a = dict(feature=np.zeros(m, np.int32), thr=np.zeros(m, np.float32),
                 left=np.zeros(m, np.int64), value=np.zeros(m, np.int64),
                 n=np.zeros(m, np.int64), S=np.zeros(m, np.int64), nrows=np.zeros(m, np.int64),
                 depth=np.zeros(m, np.int32), evaluated=np.zeros(m, np.int32))
        L.orc_tree_export(self._h, k, _ptr(a["feature"], _P_I32), _ptr(a["thr"], _P_F32),
                          _ptr(a["left"], _P_I64), _ptr(a["value"], _P_I64),
                          _ptr(a["n"], _P_I64), _ptr(a["S"], _P_I64), _ptr(a["nrows"], _P_I64),
                          _ptr(a["depth"], _P_I32), _ptr(a["evaluated"], _P_I32))
        return Tree(**a)

    def trees(self):
        return [self.tree(k) for k in range(self.num_trees)]

    def predict(self, Xq: np.ndarray, total_trees: int | None = None, want_var: bool = False):
        """Returns (pred, sum[, var]) with var as Python ints."""
        Xq = np.ascontiguousarray(Xq, dtype=np.float32)
        Q = int(Xq.shape[1])
        T = self.num_trees if total_trees is None else int(total_trees)
        s = np.zeros(Q, np.int64)
        p = np.zeros(Q, np.int64)
        v = np.zeros(2 * Q, np.uint64) if want_var else None
        lib().orc_predict(self._h, _ptr(Xq, _P_F32), Q, T, _ptr(s, _P_I64), _ptr(p, _P_I64),
                          _ptr(v, _P_U64) if want_var else None)
        if want_var:
            var = [int(v[2 * q]) | (int(v[2 * q + 1]) << 64) for q in range(Q)]
            return p, s, var
        return p, s

    def oob(self, X: np.ndarray):
        """(out_sum, out_count) of every training row over the trees that did not draw it."""
        X = np.ascontiguousarray(X, dtype=np.float32)
        N = int(X.shape[1])
        s = np.zeros(N, np.int64)
        c = np.zeros(N, np.int32)
        if lib().orc_oob(self._h, _ptr(X, _P_F32), N, _ptr(s, _P_I64), _ptr(c, _P_I32)) != 0:
            raise ValueError("X is not the training matrix")
        return s, c

    def oob_error(self, X: np.ndarray, y: np.ndarray):
        """Out-of-bag predictions (0 for rows in every tree's bootstrap), the mean squared error
        over the rows out of bag for some tree (in the target's units, from the exact rational
        mean of the Q32.32 differences, rounded once) and their number (Sec. III-B)."""
        s, c = self.oob(X)
        y = np.asarray(y, np.int64)
        pred = np.zeros(len(s), np.int64)
        tot, rows = 0, 0
        for r in range(len(s)):
            if c[r] > 0:
                pred[r] = (2 * int(s[r]) + int(c[r])) // (2 * int(c[r]))
                tot += (int(pred[r]) - int(y[r])) ** 2
                rows += 1
        mse = float(Fraction(tot, rows * 2 ** 64)) if rows else 0.0
        return pred, mse, rows

    def select_device(self, kfeat: np.ndarray, size_class: int, device_ids):
        kfeat = np.ascontiguousarray(kfeat, dtype=np.float32)
        K = int(kfeat.shape[1])
        dev = np.ascontiguousarray(device_ids, dtype=np.int32)
        D = int(dev.size)
        best = np.zeros(K, np.int32)
        pred = np.zeros(K * D, np.int64)
        lib().orc_select_device(self._h, _ptr(kfeat, _P_F32), K, size_class, _ptr(dev, _P_I32), D,
                                _ptr(best, _P_I32), _ptr(pred, _P_I64))
        return best, pred.reshape(K, D)


def fit(X: np.ndarray, y: np.ndarray, num_trees: int, mtry: int, min_node_size: int,
        max_depth: int = 0, seed: int = 156, bootstrap: bool = True, t0: int = 0,
        t1: int | None = None) -> Forest:
    """Grow trees with global indices [t0, t1) (default [0, num_trees))."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.int64)
    F, N = int(X.shape[0]), int(X.shape[1])
    if t1 is None:
        t1 = t0 + num_trees
    if np.isnan(X).any():
        raise ValueError("NaN in X")
    h = C.c_void_p()
    rc = lib().orc_fit(_ptr(X, _P_F32), _ptr(y, _P_I64), N, F, t0, t1, mtry, min_node_size,
                       max_depth, seed, 1 if bootstrap else 0, C.byref(h))
    if rc != 0:
        raise ValueError(f"orc_fit failed ({rc})")
    return Forest(h, t0, t1, F)
