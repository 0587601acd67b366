"""Pins of the surrogate's FP64 oracle and of its device tolerance.

* The unrounded network (forward, GELU, loss and gradient) equals torch's own float64 operators
  and autograd element by element, and central finite differences of its loss.
* BF16 rounding matches torch's own BF16 conversion.
* The element-wise tolerance (grad_tolerance, forward_tolerance) admits an independent FP32
  evaluation of the rounded network written here with numpy float32 operations, and rejects
  planted mistakes, among them a 5 % error in one W2 gradient entry."""
import numpy as np
import pytest
from scipy.special import erf

from oracle import mlp as M
from tests.mlp_cases import BLOCKS, model, violations


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


def test_gelu_matches_torch_float64():
    torch = pytest.importorskip("torch")
    z = np.concatenate([np.linspace(-12.0, 12.0, 4001), np.random.default_rng(5).normal(0, 3, 4000)])
    zt = torch.tensor(z, dtype=torch.float64, requires_grad=True)
    gt = torch.nn.functional.gelu(zt, approximate="none")
    (dg,) = torch.autograd.grad(gt.sum(), zt)
    ref, dref = gt.detach().numpy(), dg.numpy()
    assert np.all(np.abs(M.gelu(z) - ref) <= 1e-12 * np.maximum(np.abs(ref), 1e-300) + 1e-300)
    assert np.all(np.abs(M.gelu_grad(z) - dref) <= 1e-12 * np.maximum(np.abs(dref), 1e-300) + 1e-300)


def _torch_net(torch, P, xin, y):
    Pt = torch.tensor(P, dtype=torch.float64, requires_grad=True)
    W1 = Pt[M.OW1:M.OB1].reshape(M.HID, M.K_IN)
    W2 = Pt[M.OW2:M.OB2].reshape(M.HID, M.HID)
    x = torch.tensor(xin, dtype=torch.float64)
    gelu = torch.nn.functional.gelu
    h1 = gelu(x @ W1.T + Pt[M.OB1:M.OW2], approximate="none")
    h2 = gelu(h1 @ W2.T + Pt[M.OB2:M.OW3], approximate="none")
    out = h2 @ Pt[M.OW3:M.OB3] + Pt[M.OB3]
    loss = 0.5 * ((out - torch.tensor(y, dtype=torch.float64)) ** 2).sum()
    (g,) = torch.autograd.grad(loss / len(y), Pt)
    return out.detach().numpy(), float(loss.detach()), g.numpy()


def test_forward_and_gradient_match_torch_autograd():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    P = _params(rng)
    xin = rng.normal(size=(64, M.K_IN))
    y = rng.normal(size=64)
    out_t, loss_t, g_t = _torch_net(torch, P, xin, y)
    out, _ = M.forward(P, xin, rounding=False)
    loss, g = M.loss_and_grad(P, xin, y, rounding=False)
    assert np.all(np.abs(out - out_t) <= 1e-12 * np.abs(out_t) + 1e-15)
    assert abs(loss - loss_t) <= 1e-12 * abs(loss_t)
    # element by element; the absolute floor is float64 summation noise on the block's scale
    for name, a, b in BLOCKS:
        scale = np.abs(g_t[a:b]).max()
        assert np.all(np.abs(g[a:b] - g_t[a:b]) <= 1e-12 * np.abs(g_t[a:b]) + 1e-14 * scale), name


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


# ------------------------------------------------------------------------------------------
# the device tolerance
# ------------------------------------------------------------------------------------------
def _f32(a):
    return np.asarray(a, np.float32)


def _gelu32(z):
    z = _f32(z)
    return _f32(np.float32(0.5) * z * (np.float32(1.0) + _f32(erf(z * np.float32(0.70710678118654752)))))


def _gelu_grad32(z):
    z = _f32(z)
    a = _f32(np.float32(0.5) * (np.float32(1.0) + _f32(erf(z * np.float32(0.70710678118654752)))))
    return _f32(a + z * np.float32(0.39894228040143268) * _f32(np.exp(np.float32(-0.5) * z * z)))


def _bf16_32(a):
    return _f32(M.bf16(_f32(a)))


def fp32_evaluation(P, X, mu, sd, lg, y):
    """The rounded network evaluated with numpy float32 operations only (float32 encoding,
    float32 matrix products, BF16 rounding of inputs, weights, the first activation and the two
    back-propagated pre-activation gradients). Returns (out, loss, grad)."""
    P = _f32(P)
    n = X.shape[1]
    W1, b1 = P[M.OW1:M.OB1].reshape(M.HID, M.K_IN), P[M.OB1:M.OW2]
    W2, b2 = P[M.OW2:M.OB2].reshape(M.HID, M.HID), P[M.OB2:M.OW3]
    w3, b3 = P[M.OW3:M.OB3], P[M.OB3]
    enc = np.zeros((n, M.K_IN), np.float32)
    for f in range(30):
        x = _f32(X[f])
        if lg[f]:
            x = np.log2(np.maximum(x, np.float32(1.0)))
        enc[:, f] = (x - np.float32(mu[f])) / np.float32(sd[f])
    for d in range(15):
        enc[:, 30 + d] = X[30] == d
    for s in range(4):
        enc[:, 45 + s] = X[31] == s
    x = _bf16_32(enc)
    W1b, W2b = _bf16_32(W1), _bf16_32(W2)
    z1 = x @ W1b.T + b1
    h1 = _bf16_32(_gelu32(z1))
    z2 = h1 @ W2b.T + b2
    h2 = _gelu32(z2)
    out = h2 @ w3 + b3
    d = out - _f32(y)
    dout = d / np.float32(n)
    loss = np.sum(np.float32(0.5) * d * d, dtype=np.float32)
    g = np.zeros(M.N_PARAMS, np.float32)
    g[M.OW3:M.OB3] = h2.T @ dout
    g[M.OB3] = np.sum(dout, dtype=np.float32)
    dz2 = dout[:, None] * w3[None, :] * _gelu_grad32(z2)
    g[M.OB2:M.OW3] = np.sum(dz2, axis=0, dtype=np.float32)
    dz2b = _bf16_32(dz2)
    g[M.OW2:M.OB2] = (dz2b.T @ h1).ravel()
    dz1 = (dz2b @ W2b) * _gelu_grad32(z1)
    g[M.OB1:M.OW2] = np.sum(dz1, axis=0, dtype=np.float32)
    g[M.OW1:M.OB1] = (_bf16_32(dz1).T @ x).ravel()
    return out, float(loss), g


@pytest.fixture(scope="module")
def case():
    P, X, mu, sd, lg, y = model()
    tol = M.grad_tolerance(P.astype(np.float64), X, mu, sd, lg, 15, 4, y.astype(np.float64))
    return P, X, mu, sd, lg, y, tol


def test_tolerance_admits_an_fp32_evaluation(case):
    P, X, mu, sd, lg, y, (loss, g, lb, gb) = case
    out32, loss32, g32 = fp32_evaluation(P, X, mu, sd, lg, y)
    assert abs(loss32 - loss) <= lb
    assert all(v[0] == 0 for v in violations(g32, g, gb).values()), violations(g32, g, gb)
    out, eo = M.forward_tolerance(P.astype(np.float64), X, mu, sd, lg, 15, 4)
    assert np.all(np.abs(out32 - out) <= eo)


def test_tolerance_is_tight_on_w2(case):
    """The bound is a small fraction of the gradient itself: a 5 % error in a typical W2 entry
    is outside it."""
    _, _, _, _, _, _, (_, g, _, gb) = case
    r = gb[M.OW2:M.OB2] / np.abs(g[M.OW2:M.OB2])
    assert np.median(r) < 0.05 and np.mean(r < 0.05) > 0.6


def _planted(P, xin, y, mistake):
    """loss_and_grad(rounding=True) with one planted mistake."""
    W1, b1, W2, b2, w3, b3 = M.unpack(P)
    R = M.bf16
    n = xin.shape[0]
    out, (x, z1, h1, z2, h2) = M.forward(P, xin, True)
    d = out - y
    dout = d if mistake == "dout_not_divided_by_n" else d / n
    g = np.zeros(M.N_PARAMS)
    g[M.OW3:M.OB3] = h2.T @ dout
    g[M.OB3] = dout.sum()
    gg2 = 0.5 * (1.0 + erf(z2 / np.sqrt(2.0))) if mistake == "gelu_grad_without_z_phi" else M.gelu_grad(z2)
    dz2 = dout[:, None] * w3[None, :] * gg2
    g[M.OB2:M.OW3] = dz2.sum(0)
    dz2r = R(dz2)
    if mistake == "w2_transposed":
        g[M.OW2:M.OB2] = (dz2r.T @ h1).T.ravel()
    elif mistake == "w2_last_row_dropped":
        g[M.OW2:M.OB2] = (dz2r[:-1].T @ h1[:-1]).ravel()
    else:
        g[M.OW2:M.OB2] = (dz2r.T @ h1).ravel()
    dh1 = dz2r @ R(W2)
    dz1 = dh1 * M.gelu_grad(z1)
    g[M.OB1:M.OW2] = (dh1 if mistake == "b1_without_gelu_grad" else dz1).sum(0)
    g[M.OW1:M.OB1] = (R(dz1).T @ x).ravel()
    if mistake == "w2_entry_5pct":
        k = M.OW2 + int(np.argmax(np.abs(g[M.OW2:M.OB2])))
        g[k] *= 1.05
    if mistake == "w2_median_entry_5pct":
        blk = np.abs(g[M.OW2:M.OB2])
        k = M.OW2 + int(np.argsort(blk)[len(blk) // 2])
        g[k] *= 1.05
    return g


@pytest.mark.parametrize("mistake", ["w2_entry_5pct", "w2_median_entry_5pct", "w2_transposed", "w2_last_row_dropped",
                                     "gelu_grad_without_z_phi", "b1_without_gelu_grad", "dout_not_divided_by_n"])
def test_tolerance_rejects_planted_mistakes(case, mistake):
    P, X, mu, sd, lg, y, (loss, g, lb, gb) = case
    xin = M.encode(X, mu, sd, lg, 15, 4)
    gp = _planted(P.astype(np.float64), xin, y.astype(np.float64), "none")
    assert np.array_equal(gp, g)                    # the copy without a mistake is the oracle
    gm = _planted(P.astype(np.float64), xin, y.astype(np.float64), mistake)
    assert sum(v[0] for v in violations(gm, g, gb).values()) > 0
