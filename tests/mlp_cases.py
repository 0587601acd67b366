"""Shared inputs of the surrogate tests: a random network and a seeded batch encoded the way
the surrogate standardises its inputs (mean and deviation of the batch's own columns)."""
import numpy as np

from oracle import mlp as M
from paper_1811_00156_gb300 import synth


def model(seed=0, n=512, query_seed=3):
    rng = np.random.default_rng(seed)
    P = rng.normal(0.0, 0.08, M.N_PARAMS).astype(np.float32)
    P[M.OW1:M.OB1].reshape(M.HID, M.K_IN)[:, 49:] = 0.0
    P[M.OB3] = -2.0
    X = synth.queries(n, seed=query_seed)
    lg = np.zeros(30, np.uint8)
    lg[:10] = 1
    lg[24:] = 1
    T = np.where(lg[:, None] == 1, np.log2(np.maximum(X[:30].astype(np.float64), 1.0)), X[:30].astype(np.float64))
    mu = T.mean(1).astype(np.float32)
    sd = (T.std(1) + 1e-3).astype(np.float32)
    y = np.random.default_rng(seed + 4).normal(-3.0, 1.0, n).astype(np.float32)
    return P, X, mu, sd, lg, y


BLOCKS = [("W1", M.OW1, M.OB1), ("b1", M.OB1, M.OW2), ("W2", M.OW2, M.OB2), ("b2", M.OB2, M.OW3),
          ("w3", M.OW3, M.OB3), ("b3", M.OB3, M.N_PARAMS)]


def violations(g_dev, g_ref, bound):
    """Per block: (elements outside the bound, largest |error| / bound)."""
    out = {}
    for name, a, b in BLOCKS:
        err = np.abs(np.asarray(g_dev[a:b], np.float64) - g_ref[a:b])
        bd = bound[a:b]
        ratio = np.where(err > 0, err / np.maximum(bd, 1e-300), 0.0)
        out[name] = (int(np.sum(err > bd)), float(np.max(ratio)))
    return out
