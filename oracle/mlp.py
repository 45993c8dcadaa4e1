"""FP64 oracle of the learned VSamp proposal's network (test infrastructure only).

Not part of the paper: VSamp (Algorithm 4) draws vertices uniformly; the
library can instead draw from a mixture whose learned half follows the scores
of a small network.  This module restates that network in plain float64
numpy so the CUDA kernels can be checked against it:
  features  - the six per-vertex features, from the edge list
  bf16      - round-to-nearest-even of float32 values to bfloat16
  forward   - 6 -> 64 -> 64 -> 1 with GELU (erf form) after each hidden layer
  grad      - gradient of the mean squared error, by the chain rule
Parameter vector layout: W1[6][64], b1[64], W2[64][64], b2[64], W3[64], b3.
"""
from __future__ import annotations

import math

import numpy as np

F, H = 6, 64
OFF_W1 = 0
OFF_B1 = OFF_W1 + F * H
OFF_W2 = OFF_B1 + H
OFF_B2 = OFF_W2 + H * H
OFF_W3 = OFF_B2 + H
OFF_B3 = OFF_W3 + H
NPARAM = OFF_B3 + 1

_erf = np.vectorize(math.erf, otypes=[np.float64])


def bf16(w32: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest, ties to even); returned as float64."""
    b = np.ascontiguousarray(w32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> np.uint64(16)) & np.uint64(1)
    r = ((b + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def unpack(p: np.ndarray):
    p = np.asarray(p, dtype=np.float64)
    return (p[OFF_W1:OFF_B1].reshape(F, H), p[OFF_B1:OFF_W2], p[OFF_W2:OFF_B2].reshape(H, H), p[OFF_B2:OFF_W3],
            p[OFF_W3:OFF_B3], p[OFF_B3])


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    cdf = 0.5 * (1.0 + _erf(z / math.sqrt(2.0)))
    pdf = np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)
    return cdf + z * pdf


def forward(p: np.ndarray, X: np.ndarray) -> np.ndarray:
    W1, b1, W2, b2, W3, b3 = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    h1 = gelu(X @ W1 + b1)
    h2 = gelu(h1 @ W2 + b2)
    return h2 @ W3 + b3


def loss_and_grad(p: np.ndarray, X: np.ndarray, T: np.ndarray):
    """(mean (y - t)^2, its gradient with respect to the parameter vector)."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    n = X.shape[0]
    z1 = X @ W1 + b1
    h1 = gelu(z1)
    z2 = h1 @ W2 + b2
    h2 = gelu(z2)
    y = h2 @ W3 + b3
    e = y - T
    loss = float(np.mean(e * e))
    dy = 2.0 * e / n
    g = np.zeros(NPARAM)
    g[OFF_W3:OFF_B3] = h2.T @ dy
    g[OFF_B3] = dy.sum()
    dz2 = np.outer(dy, W3) * gelu_grad(z2)
    g[OFF_W2:OFF_B2] = (h1.T @ dz2).ravel()
    g[OFF_B2:OFF_W3] = dz2.sum(axis=0)
    dz1 = (dz2 @ W2.T) * gelu_grad(z1)
    g[OFF_W1:OFF_B1] = (X.T @ dz1).ravel()
    g[OFF_B1:OFF_W2] = dz1.sum(axis=0)
    return loss, g


def features(u, v, nU: int, nV: int) -> np.ndarray:
    """Per-vertex features, rows U then V, from the definitions:
    log1p(d)/8, log1p(sum of neighbour degrees)/16, log1p(sum (d_u - 1))/16,
    log1p(C(d, 2))/16, side, log1p(max neighbour degree)/16."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    dU = np.bincount(u, minlength=nU).astype(np.float64)
    dV = np.bincount(v, minlength=nV).astype(np.float64)
    out = np.zeros((nU + nV, F))
    for side, (a, b, da, db, n) in enumerate(((u, v, dU, dV, nU), (v, u, dV, dU, nV))):
        s1 = np.zeros(n)
        np.add.at(s1, a, db[b])
        mx = np.zeros(n)
        np.maximum.at(mx, a, db[b])
        rows = out[side * nU: side * nU + n]
        rows[:, 0] = np.log1p(da) / 8
        rows[:, 1] = np.log1p(s1) / 16
        rows[:, 2] = np.log1p(s1 - da) / 16
        rows[:, 3] = np.log1p(da * (da - 1) / 2) / 16
        rows[:, 4] = side
        rows[:, 5] = np.log1p(mx) / 16
    return out


def score_weights(scores: np.ndarray) -> np.ndarray:
    """Integer proposal weights max(1, floor(2^24 exp(s - max s))) (float64 arithmetic)."""
    s = np.asarray(scores, dtype=np.float64)
    e = np.exp(np.minimum(s - s.max(), 0.0)) * 16777216.0
    return np.maximum(1, np.floor(np.minimum(e, 16777216.0))).astype(np.uint64)
