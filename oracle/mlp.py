"""FP64 restatement of the learned surrogate's forward and backward pass (numpy).

TEST INFRASTRUCTURE: only tests and benchmark baselines use it. The surrogate is a multilayer
perceptron 64 -> 256 -> 256 -> 1 with GELU (erf form), BF16 weights and activations and FP32
accumulation on the GPU. This oracle computes in float64 and applies BF16 rounding (round to
nearest even) at the points where the GPU path stores BF16: the encoded inputs, both weight
matrices, the first hidden activation and the two back-propagated pre-activation gradients that
feed the tensor-core GEMMs. With rounding=False it is the plain float64 network, whose gradient
the tests pin with central finite differences and with torch's float64 autograd.

forward_tolerance and grad_tolerance give, element by element, how far an evaluation of the same
rounded network in FP32 arithmetic (FP32 accumulation of exact BF16 products) may lie from this
oracle: a running error analysis from the unit roundoff of FP32, the documented ulp bounds of
log2f, erff and expf, and the monotonicity of rounding to BF16 (derivation beside the code).

Parameter vector: W1[256][64], b1[256], W2[256][256], b2[256], w3[256], b3.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

K_IN, HID = 64, 256
OW1 = 0
OB1 = OW1 + HID * K_IN
OW2 = OB1 + HID
OB2 = OW2 + HID * HID
OW3 = OB2 + HID
OB3 = OW3 + HID
N_PARAMS = OB3 + 1


def bf16(x: np.ndarray) -> np.ndarray:
    """Round to BF16 (nearest, ties to even) through the float32 bit pattern; back as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def encode(X: np.ndarray, mu, sd, log2_cols, n_dev: int, n_size: int) -> np.ndarray:
    """(n, 64) inputs: standardised AIWC columns (log2 first where flagged), one-hot device,
    one-hot size class, zeros. X is F x n, column-major like the library's inputs."""
    F, n = X.shape
    na = F - 2
    out = np.zeros((n, K_IN))
    for f in range(na):
        x = X[f].astype(np.float64)
        if log2_cols[f]:
            x = np.log2(np.maximum(x, 1.0))
        out[:, f] = (x - mu[f]) / sd[f]
    dev, size = X[na], X[na + 1]
    for d in range(n_dev):
        out[:, na + d] = (dev == d)
    for s in range(n_size):
        out[:, na + n_dev + s] = (size == s)
    return out


def unpack(P):
    P = np.asarray(P, np.float64)
    return (P[OW1:OB1].reshape(HID, K_IN), P[OB1:OW2], P[OW2:OB2].reshape(HID, HID), P[OB2:OW3], P[OW3:OB3],
            P[OB3])


def forward(P, xin, rounding=True):
    W1, b1, W2, b2, w3, b3 = unpack(P)
    R = bf16 if rounding else (lambda a: np.asarray(a, np.float64))
    x = R(xin)
    z1 = x @ R(W1).T + b1
    h1 = R(gelu(z1))
    z2 = h1 @ R(W2).T + b2
    h2 = gelu(z2)
    out = h2 @ w3 + b3
    return out, (x, z1, h1, z2, h2)


def loss_and_grad(P, xin, y, rounding=True):
    """Loss sum((out - y)^2 / 2) and the gradient of that loss divided by n."""
    W1, b1, W2, b2, w3, b3 = unpack(P)
    R = bf16 if rounding else (lambda a: np.asarray(a, np.float64))
    n = xin.shape[0]
    out, (x, z1, h1, z2, h2) = forward(P, xin, rounding)
    d = out - y
    loss = 0.5 * np.sum(d * d)
    dout = d / n
    g = np.zeros(N_PARAMS)
    g[OW3:OB3] = h2.T @ dout
    g[OB3] = dout.sum()
    dz2 = dout[:, None] * w3[None, :] * gelu_grad(z2)
    g[OB2:OW3] = dz2.sum(0)
    dz2r = R(dz2)
    g[OW2:OB2] = (dz2r.T @ h1).ravel()
    dh1 = dz2r @ R(W2)
    dz1 = dh1 * gelu_grad(z1)
    g[OB1:OW2] = dz1.sum(0)
    g[OW1:OB1] = (R(dz1).T @ x).ravel()
    return loss, g


# ------------------------------------------------------------------------------------------
# Element-wise tolerance for a BF16/FP32 evaluation of loss_and_grad (running error analysis)
# ------------------------------------------------------------------------------------------
# A device evaluates the same network with FP32 arithmetic and FP32 tensor-core accumulation of
# exact BF16 x BF16 products, rounding to BF16 where loss_and_grad(rounding=True) does. Each
# intermediate q of that evaluation differs from this oracle's float64 value by at most E_q,
# propagated step by step with these facts (u = 2^-24, the FP32 unit roundoff):
#   * one FP32 operation (+, *, /) errs by at most u relative to its result;
#   * log2f errs by at most 1 ulp, erff and expf by at most 2 ulp (CUDA's documented bounds);
#     one FP32 ulp is at most 2u relative, so these are taken as 2u, 4u and 4u relative;
#   * a K-term FP32 accumulation (tensor core or loop, any order, FMA or not) errs by at most
#     2 K u times the sum of the absolute terms, which allows truncating rather than rounding
#     accumulation as well;
#   * an error E in the argument of GELU moves it by at most (|GELU'(z)| + 0.7979 E) E, and
#     GELU' by at most (|GELU''(z)| + 0.7788 E) E (Taylor with the global maxima 0.7979 of
#     |GELU''| and 0.7788 of |GELU'''|);
#   * rounding to BF16 is monotone: if the device's value lies in [v - E, v + E] around the
#     oracle's v, both rounded values lie in [bf16(v - E), bf16(v + E)], so after rounding the
#     error is at most bf16(v + E) - bf16(v - E) (zero when no rounding boundary is in between);
#   * products of perturbed factors: |ab - a'b'| <= |a| E_b + |b| E_a + E_a E_b.
# The oracle's own float64 rounding (relative 2^-52 per step) is covered by a 1e-12 relative
# margin on every sum of absolute terms.
_U = 2.0 ** -24
_MAX_GELU_D2 = 0.7979          # max |GELU''| = 2 phi(0)
_MAX_GELU_D3 = 0.7788          # max |phi(z) (z^3 - 4 z)|


def _gelu_d2(z):
    return np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi) * (2.0 - z * z)


def _gelu_moved(z, E):
    """Bound on |GELU(z') - GELU(z)| for |z' - z| <= E."""
    return (np.abs(gelu_grad(z)) + _MAX_GELU_D2 * E) * E


def _gelu_grad_moved(z, E):
    """Bound on |GELU'(z') - GELU'(z)| for |z' - z| <= E."""
    return (np.abs(_gelu_d2(z)) + _MAX_GELU_D3 * E) * E


def _acc(K):
    return 2.0 * K * _U + 1e-12


def _round_err(v, E):
    """Bound on |bf16(v') - bf16(v)| for every v' within E of v."""
    return bf16(v + E) - bf16(v - E)


def _gelu_f32_err(z, erf_err=None):
    """Bound on |GELU evaluated in FP32 (0.5 z (1 + erf(z c)), c = fl(1/sqrt 2)) - GELU(z)| at
    an exact FP32 argument z: the argument z c errs by 1.42 u |z| (c and the product), erf's
    slope is at most 2/sqrt(pi) exp(-z^2/2), the erf evaluation adds erf_err (absolute; default
    4u, CUDA's erff), the sum and the product u each."""
    a = np.abs(z)
    e0 = 4.0 * _U if erf_err is None else erf_err
    d_erf = e0 + 1.13 * 1.42 * _U * a * np.exp(-0.5 * z * z)
    return 0.5 * a * (d_erf + _U * np.abs(1.0 + erf(z / np.sqrt(2.0)))) + 2.0 * _U * np.abs(gelu(z))


def _gelu_grad_f32_err(z):
    """Bound on |GELU' evaluated in FP32 (0.5 (1 + erff(z c)) + z c2 expf(-0.5 z z)) - GELU'(z)|:
    the first term as in _gelu_f32_err; the exponent -z^2/2 errs by u z^2/2 (relative error of
    exp), expf adds 4u, c2 and the two products 3u, the final sum u."""
    a = np.abs(z)
    d_erf = 4.0 * _U + 1.13 * 1.42 * _U * a * np.exp(-0.5 * z * z)
    t2 = a * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)
    return 0.5 * (d_erf + _U * np.abs(1.0 + erf(z / np.sqrt(2.0)))) + t2 * (0.5 * _U * z * z + 7.0 * _U) + \
        2.0 * _U * np.abs(gelu_grad(z))


def _mm_err(A, EA, B, EB, K):
    """Error of the accumulated product A @ B when A and B are known within EA and EB:
    propagated factor errors plus the accumulation bound on the sum of absolute terms."""
    aA, aB = np.abs(A), np.abs(B)
    return EA @ aB + aA @ EB + EA @ EB + _acc(K) * (aA @ aB)


def encode_error(X, mu, sd, log2_cols, n_dev: int, n_size: int):
    """Bound on |FP32 encoding - encode()| per input: log2f (2u), the subtraction (u) and the
    division (u); the one-hot and padding inputs are exact."""
    F, n = X.shape
    na = F - 2
    E = np.zeros((n, K_IN))
    for f in range(na):
        x = X[f].astype(np.float64)
        el = 0.0
        if log2_cols[f]:
            x = np.log2(np.maximum(x, 1.0))
            el = 2.0 * _U * np.abs(x)
        e = (x - mu[f]) / sd[f]
        E[:, f] = (el + _U * np.abs(x - mu[f])) / sd[f] * (1.0 + _U) + _U * np.abs(e) + 1e-12 * np.abs(e)
    return E


def _forward_bounds(P, X, mu, sd, log2_cols, n_dev: int, n_size: int, erf_err=None):
    """Forward pass with rounding and the error bound of every intermediate (dict); erf_err: the
    absolute error of the evaluation's erf (None: CUDA's erff)."""
    W1, b1, W2, b2, w3, b3 = unpack(P)
    r = {}
    xin = encode(X, mu, sd, log2_cols, n_dev, n_size)
    r["xin"] = xin
    r["W1r"], r["W2r"] = bf16(W1), bf16(W2)          # FP32 weights rounded once: the same values
    r["x"] = x = bf16(xin)
    r["Ex"] = Ex = _round_err(xin, encode_error(X, mu, sd, log2_cols, n_dev, n_size))
    r["z1"] = z1 = x @ r["W1r"].T + b1
    r["Ez1"] = Ez1 = _mm_err(x, Ex, r["W1r"].T, 0.0 * W1.T, K_IN + 1) + _acc(1) * np.abs(b1) + _U * np.abs(z1)
    r["h1"] = h1 = bf16(gelu(z1))
    r["Eh1"] = Eh1 = _round_err(gelu(z1), _gelu_moved(z1, Ez1) + _gelu_f32_err(z1, erf_err))
    r["z2"] = z2 = h1 @ r["W2r"].T + b2
    r["Ez2"] = Ez2 = _mm_err(h1, Eh1, r["W2r"].T, 0.0 * W2.T, HID + 1) + _acc(1) * np.abs(b2) + _U * np.abs(z2)
    r["h2"] = h2 = gelu(z2)
    r["Eh2"] = Eh2 = _gelu_moved(z2, Ez2) + _gelu_f32_err(z2, erf_err)
    r["out"] = h2 @ w3 + b3
    r["Eout"] = Eh2 @ np.abs(w3) + _acc(HID + 1) * (np.abs(h2) @ np.abs(w3) + abs(b3))
    return r


def forward_tolerance(P, X, mu, sd, log2_cols, n_dev: int, n_size: int, erf_err=None):
    """The rounded forward pass's outputs and the bound on how far an FP32/BF16 evaluation of
    the same network may lie from each of them, its erf within erf_err (absolute; None: CUDA's
    erff). Returns (out, out_bound)."""
    r = _forward_bounds(P, X, mu, sd, log2_cols, n_dev, n_size, erf_err)
    return r["out"], r["Eout"]


def grad_tolerance(P, X, mu, sd, log2_cols, n_dev: int, n_size: int, y):
    """Oracle loss and gradient (loss_and_grad with rounding) and element-wise bounds on how far
    an FP32/BF16 evaluation of the same network may lie from them. Returns
    (loss, grad, loss_bound, grad_bound)."""
    W1, b1, W2, b2, w3, b3 = unpack(P)
    y = np.asarray(y, np.float64)
    n = X.shape[1]
    r = _forward_bounds(P, X, mu, sd, log2_cols, n_dev, n_size)
    loss, g = loss_and_grad(P, r["xin"], y, rounding=True)
    x, Ex, z1, Ez1, h1, Eh1 = r["x"], r["Ex"], r["z1"], r["Ez1"], r["h1"], r["Eh1"]
    z2, Ez2, h2, Eh2, W2r = r["z2"], r["Ez2"], r["h2"], r["Eh2"], r["W2r"]
    d = r["out"] - y
    Ed = r["Eout"] + _U * np.abs(d)
    dout = d / n
    Edout = Ed / n + _U * np.abs(dout)
    loss_bound = np.sum(np.abs(d) * Ed + 0.5 * Ed * Ed) + _acc(n) * loss
    gb = np.zeros(N_PARAMS)
    # w3 and b3
    gb[OW3:OB3] = _mm_err(h2.T, Eh2.T, dout[:, None], Edout[:, None], n)[:, 0]
    gb[OB3] = Edout.sum() + _acc(n) * np.abs(dout).sum()
    # dz2 = dout w3 GELU'(z2): two FP32 products
    gg2 = gelu_grad(z2)
    Egg2 = _gelu_grad_moved(z2, Ez2) + _gelu_grad_f32_err(z2)
    a2 = np.abs(dout)[:, None] * np.abs(w3)[None, :]
    Ea2 = Edout[:, None] * np.abs(w3)[None, :] + _U * a2
    dz2 = dout[:, None] * w3[None, :] * gg2
    Edz2 = a2 * Egg2 + Ea2 * np.abs(gg2) + Ea2 * Egg2 + _U * np.abs(dz2)
    gb[OB2:OW3] = Edz2.sum(0) + _acc(n) * np.abs(dz2).sum(0)
    dz2r = bf16(dz2)
    Edz2r = _round_err(dz2, Edz2)
    gb[OW2:OB2] = _mm_err(dz2r.T, Edz2r.T, h1, Eh1, n + 16).ravel()
    # dh1 = dz2r W2r, dz1 = dh1 GELU'(z1)
    dh1 = dz2r @ W2r
    Edh1 = _mm_err(dz2r, Edz2r, W2r, 0.0 * W2r, HID)
    gg1 = gelu_grad(z1)
    Egg1 = _gelu_grad_moved(z1, Ez1) + _gelu_grad_f32_err(z1)
    dz1 = dh1 * gg1
    Edz1 = np.abs(dh1) * Egg1 + Edh1 * np.abs(gg1) + Edh1 * Egg1 + _U * np.abs(dz1)
    gb[OB1:OW2] = Edz1.sum(0) + _acc(n) * np.abs(dz1).sum(0)
    dz1r = bf16(dz1)
    Edz1r = _round_err(dz1, Edz1)
    gb[OW1:OB1] = _mm_err(dz1r.T, Edz1r.T, x, Ex, n + 16).ravel()
    return loss, g, loss_bound, gb
