"""FP64 restatement of the learned surrogate's forward and backward pass (numpy).

TEST INFRASTRUCTURE: only tests and benchmark baselines use it. The surrogate is a multilayer
perceptron 64 -> 256 -> 256 -> 1 with GELU (erf form), BF16 weights and activations and FP32
accumulation on the GPU. This oracle computes in float64 and applies BF16 rounding (round to
nearest even) at the points where the GPU path stores BF16: the encoded inputs, both weight
matrices, the first hidden activation and the two back-propagated pre-activation gradients that
feed the tensor-core GEMMs. With rounding=False it is the plain float64 network, whose gradient
the tests pin with central finite differences.

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
