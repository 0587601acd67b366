"""Pins of the surrogate's FP64 oracle: the analytic gradient of the unrounded network equals
central finite differences of its loss; BF16 rounding matches torch's own BF16 conversion."""
import numpy as np
import pytest

from oracle import mlp as M


def _params(rng, scale=0.1):
    P = rng.normal(0.0, scale, M.N_PARAMS)
    P[M.OB3] = 0.3
    return P


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(0).normal(0, 100, 20000)
    x = np.concatenate([x, [1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -0.0, 65504.0]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.bf16(x), ref)


def test_gradient_equals_finite_differences():
    rng = np.random.default_rng(1)
    P = _params(rng)
    xin = rng.normal(size=(16, M.K_IN))
    y = rng.normal(size=16)
    _, g = M.loss_and_grad(P, xin, y, rounding=False)
    h = 1e-6
    idx = np.concatenate([rng.choice(np.arange(M.OW1, M.OB1), 12), rng.choice(np.arange(M.OB1, M.OW2), 6),
                          rng.choice(np.arange(M.OW2, M.OB2), 12), rng.choice(np.arange(M.OB2, M.OW3), 6),
                          rng.choice(np.arange(M.OW3, M.OB3), 6), [M.OB3]])
    for i in idx:
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        fd = (M.loss_and_grad(Pp, xin, y, False)[0] - M.loss_and_grad(Pm, xin, y, False)[0]) / (2 * h) / 16
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), i


def test_encode_layout():
    X = np.array([[1.0, 8.0], [3.0, 5.0], [2.0, 14.0], [0.0, 3.0]], np.float32)      # 2 AIWC, device, size
    e = M.encode(X, mu=[1.0, 4.0], sd=[2.0, 1.0], log2_cols=[1, 0], n_dev=15, n_size=4)
    assert e.shape == (2, 64)
    assert e[0, 0] == (0.0 - 1.0) / 2.0 and e[1, 0] == (3.0 - 1.0) / 2.0       # log2 of 1 and of 8
    assert e[0, 1] == -1.0 and e[1, 1] == 1.0
    assert e[0, 2 + 2] == 1.0 and e[1, 2 + 14] == 1.0 and e[0, 2:17].sum() == 1.0
    assert e[0, 17 + 0] == 1.0 and e[1, 17 + 3] == 1.0 and e[:, 21:].sum() == 0.0
