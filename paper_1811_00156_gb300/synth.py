"""Seeded synthetic AIWC-shaped workloads.

The paper fits its model on AIWC metrics of the 37 OpenDwarfs-Extended kernels at 4 problem sizes,
timed on 15 devices (Sec. III, Sec. III-A, Table I, Table II). That table and those timings are
not available, so every workload here is synthetic with the same shape:

* 30 AIWC-like feature columns, drawn once per (kernel, size) pair and shared by all devices
  (the features are architecture independent, Sec. I), in four families:
  columns 0-9 instruction/opcode counts, lognormal(mu=12, sigma=3);
  columns 10-17 memory/branch entropies, uniform[0, 32] bits;
  columns 18-23 ratios, uniform[0, 1];
  columns 24-29 unique-address / work-item counts, 2**k with k uniform on {4..24} (exact in f32).
* column 30: device id 0..14 (Table II has 15 devices); column 31: size class 0..3.
* target: log10 runtime from a hidden seeded piecewise-linear function per device, plus noise,
  quantised once to Q32.32 int64 (value * 2**32, round half to even).

This module only produces inputs. It holds none of the method's arithmetic, and both the CUDA
path and the CPU oracle read what it returns.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

N_KERNELS = 37
N_DEVICES = 15
N_SIZES = 4
N_AIWC = 30
N_FEATURES = N_AIWC + 2          # + device id + size class
COL_DEVICE = N_AIWC
COL_SIZE = N_AIWC + 1
Q32 = float(1 << 32)

DATA_SEED = 1811
FOREST_SEED = 156
QUERY_SEED = 7

_COUNT_COLS = list(range(0, 10)) + list(range(24, 30))


@dataclass
class Workload:
    """Column-major inputs: X is float32 [F][N] (row n of feature f at X[f, n]); y is int64 Q32.32."""
    X: np.ndarray
    y: np.ndarray
    name: str
    meta: dict = field(default_factory=dict)

    @property
    def n_rows(self) -> int:
        return int(self.X.shape[1])

    @property
    def n_features(self) -> int:
        return int(self.X.shape[0])


def aiwc_features(rng: np.random.Generator, m: int) -> np.ndarray:
    """m draws of the 30 AIWC-like columns, float32 [30][m]."""
    out = np.empty((N_AIWC, m), dtype=np.float32)
    out[0:10] = rng.lognormal(mean=12.0, sigma=3.0, size=(10, m)).astype(np.float32)
    out[10:18] = rng.uniform(0.0, 32.0, size=(8, m)).astype(np.float32)
    out[18:24] = rng.uniform(0.0, 1.0, size=(6, m)).astype(np.float32)
    out[24:30] = np.exp2(rng.integers(4, 25, size=(6, m))).astype(np.float32)
    return out


class _HiddenRuntime:
    """Seeded piecewise-linear log10-runtime model per device (the synthetic response)."""

    def __init__(self, rng: np.random.Generator, pop: np.ndarray):
        z = self._raw(pop)
        self.mu = z.mean(axis=1, keepdims=True)
        self.sd = z.std(axis=1, keepdims=True) + 1e-12
        self.b = rng.uniform(-4.5, -2.5, size=N_DEVICES)
        self.gamma = np.cumsum(rng.uniform(0.3, 0.9, size=N_SIZES)) - 0.3
        self.J = np.stack([rng.choice(N_AIWC, 4, replace=False) for _ in range(N_DEVICES)])
        self.K = np.stack([rng.choice(N_AIWC, 4, replace=False) for _ in range(N_DEVICES)])
        self.a = rng.uniform(0.05, 0.45, size=(N_DEVICES, 4))
        self.a2 = rng.uniform(0.05, 0.45, size=(N_DEVICES, 4))
        self.beta = rng.normal(0.0, 0.7, size=(N_DEVICES, 4))
        self.beta2 = rng.normal(0.0, 0.7, size=(N_DEVICES, 4))

    @staticmethod
    def _raw(feat: np.ndarray) -> np.ndarray:
        z = feat.astype(np.float64).copy()
        z[_COUNT_COLS] = np.log2(np.maximum(z[_COUNT_COLS], 1.0))
        return z

    def __call__(self, feat: np.ndarray, dev: np.ndarray, size: np.ndarray) -> np.ndarray:
        z = (self._raw(feat) - self.mu) / self.sd
        m = feat.shape[1]
        cols = np.arange(m)
        out = self.b[dev] + self.gamma[size]
        for k in range(4):
            zj = z[self.J[dev, k], cols]
            out = out + self.a[dev, k] * np.maximum(0.0, zj - self.beta[dev, k])
            zk = z[self.K[dev, k], cols]
            out = out - self.a2[dev, k] * np.maximum(0.0, self.beta2[dev, k] - zk)
        return out


def quantise(y: np.ndarray) -> np.ndarray:
    """Q32.32 int64, round half to even, applied once."""
    return np.rint(np.asarray(y, dtype=np.float64) * Q32).astype(np.int64)


def _population(seed: int):
    rng = np.random.default_rng(seed)
    pop = aiwc_features(rng, N_KERNELS * N_SIZES)      # one vector per (kernel, size)
    model = _HiddenRuntime(rng, pop)
    return rng, pop, model


def _grid_rows(pop: np.ndarray):
    """Rows ordered (kernel, device, size): row = (k*15 + d)*4 + s."""
    k, d, s = np.meshgrid(np.arange(N_KERNELS), np.arange(N_DEVICES), np.arange(N_SIZES),
                          indexing="ij")
    k, d, s = k.ravel(), d.ravel(), s.ravel()
    X = np.empty((N_FEATURES, k.size), dtype=np.float32)
    X[:N_AIWC] = pop[:, k * N_SIZES + s]
    X[COL_DEVICE] = d.astype(np.float32)
    X[COL_SIZE] = s.astype(np.float32)
    return X, k, d, s


def plain_forest_workload(seed: int = DATA_SEED) -> Workload:
    """2,220 rows = 37 kernels x 15 devices x 4 sizes; log10 runtime + N(0, 0.02)."""
    rng, pop, model = _population(seed)
    X, k, d, s = _grid_rows(pop)
    y = model(pop[:, k * N_SIZES + s], d, s) + rng.normal(0.0, 0.02, size=k.size)
    return Workload(X=np.ascontiguousarray(X), y=quantise(y), name="aiwc-2220",
                    meta=dict(seed=seed, kernel=k, device=d, size=s))


def scaled_forest_workload(seed: int = DATA_SEED, replicates: int = 50) -> Workload:
    """111,000 rows: every (kernel, device, size) cell repeated 50x; each replicate adds
    lognormal 3 % run noise, i.e. N(0, 0.03/ln 10) in log10."""
    base = plain_forest_workload(seed)
    rng = np.random.default_rng(seed + 1)
    n0 = base.n_rows
    X = np.repeat(base.X, replicates, axis=1)
    ylog = np.repeat(base.y.astype(np.float64) / Q32, replicates)
    ylog = ylog + rng.normal(0.0, 0.03 / math.log(10.0), size=n0 * replicates)
    meta = {key: np.repeat(val, replicates) for key, val in base.meta.items() if key != "seed"}
    meta["seed"] = seed
    return Workload(X=np.ascontiguousarray(X), y=quantise(ylog), name=f"aiwc-{n0 * replicates}",
                    meta=meta)


def per_row_forest_workload(seed: int = DATA_SEED, replicates: int = 50) -> Workload:
    """The 111,000-row workload read with features per row: the same (kernel, device, size)
    grid and replicate count as scaled_forest_workload, but every row draws its own AIWC vector
    from the feature distributions (no two rows share one), with the target from the same hidden
    model on the row's own features plus N(0, 0.02) and the 3 % run noise. The continuous
    columns then hold about one distinct value per row."""
    rng, pop, model = _population(seed)
    X0, k, d, s = _grid_rows(pop)
    n = k.size * replicates
    rng2 = np.random.default_rng(seed + 3)
    X = np.empty((N_FEATURES, n), dtype=np.float32)
    X[:N_AIWC] = aiwc_features(rng2, n)
    dev = np.repeat(d, replicates)
    size = np.repeat(s, replicates)
    X[COL_DEVICE] = dev.astype(np.float32)
    X[COL_SIZE] = size.astype(np.float32)
    ylog = model(X[:N_AIWC], dev, size) + rng2.normal(0.0, 0.02, size=n)
    ylog = ylog + rng2.normal(0.0, 0.03 / math.log(10.0), size=n)
    return Workload(X=np.ascontiguousarray(X), y=quantise(ylog), name=f"aiwc-{n}-per-row",
                    meta=dict(seed=seed, kernel=np.repeat(k, replicates), device=dev, size=size))


def queries(q: int, seed: int = QUERY_SEED) -> np.ndarray:
    """q fresh query rows from the same feature distributions (continuous, off the training
    grid); device and size class uniform. float32 [32][q]."""
    rng = np.random.default_rng(seed)
    Xq = np.empty((N_FEATURES, q), dtype=np.float32)
    Xq[:N_AIWC] = aiwc_features(rng, q)
    Xq[COL_DEVICE] = rng.integers(0, N_DEVICES, size=q).astype(np.float32)
    Xq[COL_SIZE] = rng.integers(0, N_SIZES, size=q).astype(np.float32)
    return Xq


def kernel_neighbours(K: int, size: int, jitter: float = 0.05, seed: int = QUERY_SEED,
                      data_seed: int = DATA_SEED) -> np.ndarray:
    """K kernels near the training kernels: the AIWC vector of a random training kernel at this
    size class, each count column scaled by exp(N(0, jitter)), each entropy and ratio column moved
    by N(0, jitter) times its range and kept inside it. float32 [30][K]."""
    _, pop, _ = _population(data_seed)
    rng = np.random.default_rng(seed)
    k = rng.integers(0, N_KERNELS, size=K)
    out = pop[:, k * N_SIZES + size].astype(np.float64)
    out[_COUNT_COLS] *= np.exp(rng.normal(0.0, jitter, size=(len(_COUNT_COLS), K)))
    ent = list(range(10, 18))
    out[ent] = np.clip(out[ent] + rng.normal(0.0, 32.0 * jitter, size=(len(ent), K)), 0.0, 32.0)
    rat = list(range(18, 24))
    out[rat] = np.clip(out[rat] + rng.normal(0.0, jitter, size=(len(rat), K)), 0.0, 1.0)
    return np.ascontiguousarray(out.astype(np.float32))


def neighbour_queries(q: int, jitter: float = 0.05, seed: int = QUERY_SEED) -> np.ndarray:
    """q query rows near the training kernels: kernel_neighbours' AIWC vectors, the size class
    uniform (each size's vectors drawn at that size), the device uniform. float32 [32][q]."""
    rng = np.random.default_rng(seed)
    size = rng.integers(0, N_SIZES, size=q)
    Xq = np.empty((N_FEATURES, q), dtype=np.float32)
    for s in range(N_SIZES):
        idx = np.nonzero(size == s)[0]
        if idx.size:
            Xq[:N_AIWC, idx] = kernel_neighbours(int(idx.size), s, jitter=jitter, seed=seed * N_SIZES + s + 1)
    Xq[COL_DEVICE] = rng.integers(0, N_DEVICES, size=q).astype(np.float32)
    Xq[COL_SIZE] = size.astype(np.float32)
    return Xq


def loko_folds(seed: int = DATA_SEED):
    """Leave-one-kernel-out folds over the 2,220-row workload.

    Fold k holds out a seeded coverage subset of kernel k (1-4 size classes x 5-15 devices) and
    trains on every other row, so training sets are uneven (2,160-2,215 rows). Returns
    (workload, [(train_rows, test_rows)] * 37) with row indices in increasing order."""
    wl = plain_forest_workload(seed)
    rng = np.random.default_rng(seed + 2)
    k, d, s = wl.meta["kernel"], wl.meta["device"], wl.meta["size"]
    folds = []
    for kern in range(N_KERNELS):
        ns = int(rng.integers(1, N_SIZES + 1))
        nd = int(rng.integers(5, N_DEVICES + 1))
        sizes = rng.choice(N_SIZES, ns, replace=False)
        devs = rng.choice(N_DEVICES, nd, replace=False)
        test = (k == kern) & np.isin(s, sizes) & np.isin(d, devs)
        folds.append((np.flatnonzero(~test).astype(np.int64), np.flatnonzero(test).astype(np.int64)))
    return wl, folds


def small_case(seed: int, n: int, f: int, card: int | None = None, y_scale: float = 4.0,
               y_levels: int | None = None) -> Workload:
    """Small random case for parity and pin tests: f columns, n rows.

    card: number of distinct values per column (None = continuous, tie-free in practice).
    y_levels: number of distinct target values (None = continuous)."""
    rng = np.random.default_rng(seed)
    if card is None:
        X = rng.normal(0.0, 1.0, size=(f, n)).astype(np.float32)
    else:
        levels = np.sort(rng.normal(0.0, 3.0, size=(f, card)).astype(np.float32), axis=1)
        X = np.take_along_axis(levels, rng.integers(0, card, size=(f, n)), axis=1)
    if y_levels is None:
        y = rng.uniform(-y_scale, y_scale, size=n)
    else:
        y = rng.integers(-y_levels, y_levels + 1, size=n) * (y_scale / max(y_levels, 1))
    return Workload(X=np.ascontiguousarray(X.astype(np.float32)), y=quantise(y),
                    name=f"small-{seed}-{n}x{f}", meta=dict(seed=seed))
