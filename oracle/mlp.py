"""Plain CPU reference of the warm-start network (test infrastructure only).

Not part of the paper's method: the paper's iteration starts from the zero
vector, and Lemma 1 (section 2.1) makes any start legitimate because the
feasibility of the kept triplet is checked directly.  This module is the
float64 restatement that the GPU forward and backward kernels are checked
against.

Network (sigma = d = 2): features of a state of length h -> 256 -> 256 -> 1,
GELU (erf form) after the two hidden layers.
Features (49): for positions p < 12 of each string j, a one-hot of the letter
(feature 4p + 2j + letter), zero for p >= h; feature 48 = h / 16.  Positions
from 12 on are not encoded.  A state is first replaced by the smallest index
of its orbit under complement and string swap, so the prediction has the
iterate's exact symmetries.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

H_IN = 12
N_FEAT = 4 * H_IN + 1
HIDDEN = 256


def canonical(x: np.ndarray, h: int) -> np.ndarray:
    """Smallest index of each state's orbit under complement and string swap (interleaved index)."""
    x = np.asarray(x, dtype=np.int64)
    n = 1 << (2 * h)
    c = (n - 1) - x
    w = ((x >> 1) & 0x5555555555555555) | ((x & 0x5555555555555555) << 1)
    wc = (n - 1) - w
    return np.minimum(np.minimum(x, c), np.minimum(w, wc))


def features(x: np.ndarray, h: int) -> np.ndarray:
    """The 49 input features of states x (length h), after canonicalisation."""
    x = canonical(x, h)
    X = np.zeros((x.size, N_FEAT))
    for p in range(min(h, H_IN)):
        pair = (x >> (2 * (h - 1 - p))) & 3  # bits of position p: string 0 high, string 1 low
        a, b = pair >> 1, pair & 1
        X[np.arange(x.size), 4 * p + 0 + a] = 1.0
        X[np.arange(x.size), 4 * p + 2 + b] = 1.0
    X[:, N_FEAT - 1] = h / 16.0
    return X


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def forward(params, X):
    W1, b1, W2, b2, w3, b3 = (params[k] for k in ("W1", "b1", "W2", "b2", "w3", "b3"))
    Z1 = X @ W1.T + b1
    A1 = gelu(Z1)
    Z2 = A1 @ W2.T + b2
    A2 = gelu(Z2)
    y = A2 @ w3 + b3
    return y, (X, Z1, A1, Z2, A2)


def loss_and_grads(params, X, t):
    """Mean squared error and its gradient with respect to every parameter."""
    y, (X, Z1, A1, Z2, A2) = forward(params, X)
    n = X.shape[0]
    r = y - t
    loss = float(np.mean(r * r))
    dy = 2.0 * r / n
    g = {}
    g["w3"] = A2.T @ dy
    g["b3"] = np.array(dy.sum())
    dZ2 = np.outer(dy, params["w3"]) * gelu_grad(Z2)
    g["W2"] = dZ2.T @ A1
    g["b2"] = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ params["W2"]) * gelu_grad(Z1)
    g["W1"] = dZ1.T @ X
    g["b1"] = dZ1.sum(axis=0)
    return loss, g


def to_bf16(a: np.ndarray) -> np.ndarray:
    """Round to bfloat16 (round to nearest, ties to even) through float32; returns float64."""
    f = np.asarray(a, dtype=np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    bits = (bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16(params, X):
    """BF16 inference as the tensor-core path defines it: the first layer and
    GELU in full precision, its output and W2 rounded to bfloat16, the 256 x 256
    product accumulated exactly (float64 here), then bias, GELU and head in
    full precision."""
    W1, b1, W2, b2, w3, b3 = (params[k] for k in ("W1", "b1", "W2", "b2", "w3", "b3"))
    A1 = to_bf16(gelu(X @ W1.T + b1))
    Z2 = A1 @ to_bf16(W2).T + b2
    return gelu(Z2) @ w3 + b3
